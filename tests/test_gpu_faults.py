"""Failure detection with faults made on the host, never on the GPU: an allocator that fails
gives LBM_ERR_OOM and leaks nothing; a non-finite field gives LBM_ERR_DIVERGED at the next
step, the handle stays usable, and a checkpoint taken before restores the solve."""
import ctypes as C

import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _solver_with_failing_allocator(cfg, fail_at):
    import torch

    blocks, stats = {}, dict(n=0, freed=0)

    def _alloc(nbytes, stream, ctx):
        stats["n"] += 1
        if stats["n"] == fail_at:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        blocks[t.data_ptr()] = t
        return t.data_ptr()

    def _free(ptr, stream, ctx):
        stats["freed"] += 1
        blocks.pop(int(ptr), None)

    hooks = (pkg.ALLOC_FN(_alloc), pkg.FREE_FN(_free))
    c = pkg._config_struct(cfg)
    c.dev_alloc, c.dev_free = hooks
    h = C.c_void_p()
    lib = pkg.library()
    assert lib.lbm_create(C.byref(c), C.byref(h)) == 0
    return lib, h, blocks, stats, (hooks, c)


@pytest.mark.parametrize("fail_at", [1, 7, 25])
def test_allocator_failure_is_reported_and_leaks_nothing(fail_at):
    pkg.build()
    cfg, loops = W.naca0012_small(levels=4)
    xy, off = pkg._loops_arrays(loops)
    lib, h, blocks, stats, keep = _solver_with_failing_allocator(cfg, fail_at)
    rc = lib.lbm_set_geometry(h, pkg._dp(xy), pkg._ip(off), len(loops))
    assert rc == -2 and b"allocation" in lib.lbm_last_error(h)
    # every block it got was returned (the allocations of the failing stage are all attempted)
    assert not blocks and stats["freed"] == stats["n"] - 1
    assert lib.lbm_step(h, 1) == -4                          # no geometry: a clean error
    lib.lbm_destroy(h)
    assert stats["freed"] == stats["n"] - 1


def test_non_finite_state_is_detected_and_a_checkpoint_recovers():
    pkg.build()
    cfg, loops = W.naca0012_small(levels=4)
    L = cfg["levels"]
    s = pkg.Solver(cfg)
    s.set_geometry(loops)
    s.step(5)
    blob = s.get_state()
    s.step(5)
    want = [s.get_populations(l) for l in range(L)]
    f = s.get_fields(L - 1)
    rho = f["rho"].copy()
    j, i = np.argwhere(f["mask"] == 1)[len(np.argwhere(f["mask"] == 1)) // 2]
    rho[j, i] = np.nan                                        # the fault, injected on the host
    s.set_fields(L - 1, rho=rho)
    with pytest.raises(pkg.LBMError) as e:
        s.step(1)
    assert e.value.code == -6
    assert s.get_fields(0)["rho"].shape[0] > 0                 # the handle still answers queries
    s.set_state(blob)                                          # recovery from the checkpoint
    s.step(5)
    for l in range(L):
        assert np.array_equal(s.get_populations(l), want[l], equal_nan=True), l
