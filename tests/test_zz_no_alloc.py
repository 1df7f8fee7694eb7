"""lbm_level_mass_noalloc: the level mass and finiteness check that allocates nothing.

It serves callers that cannot call cudaMalloc (inside another framework's stream
capture, real-time loops with a fixed memory plan).  Its scratch is a fixed device
array shared by every call, so the checks here run two calls in a row and compare
both with the mass that lbm_get_loads reports for the same state.  The file is
collected last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg

pytestmark = pytest.mark.gpu


def _level_arrays(solver, level):
    """Dense device arrays of one level built from lbm_get_fields: flags 1 (active
    fluid) where the mask is 1 or 2, else 0; rho - 1, u, chi as FP32."""
    import torch

    F = solver.get_fields(level)
    act = (F["mask"] == 1) | (F["mask"] == 2)
    flags = np.where(act, 1, 0).astype(np.int32).ravel()
    arr = {}
    for key, src in (("drho", F["rho"] - 1.0), ("ux", F["ux"]), ("uy", F["uy"]), ("chi", F["chi"])):
        arr[key] = torch.tensor(np.where(act, src, 0.0).astype(np.float32).ravel(), device="cuda")
    arr["flags"] = torch.tensor(flags, device="cuda")
    return arr, int(flags.size)


def _outputs():
    import torch

    return torch.zeros(1, dtype=torch.float64, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda")


def _mass_noalloc(arrays, levels, outs=None):
    import torch

    out_m, out_f = outs if outs is not None else _outputs()
    total, bad = 0.0, 0
    stream = torch.cuda.current_stream().cuda_stream
    for level, (a, n) in enumerate(arrays):
        area = float(4 ** (levels - 1 - level))
        rc = pkg.level_mass_noalloc(a["flags"].data_ptr(), a["drho"].data_ptr(), a["ux"].data_ptr(),
                                    a["uy"].data_ptr(), a["chi"].data_ptr(), n, area, out_m.data_ptr(),
                                    out_f.data_ptr(), stream)
        assert rc == 0, rc
        torch.cuda.synchronize()
        total += float(out_m.item())
        bad |= int(out_f.item())
    return total, bad


def test_noalloc_mass_matches_get_loads_twice():
    import torch

    import __graft_entry__

    pkg.build()
    torch.cuda.set_device(0)
    cfg, loops = __graft_entry__.smoke_case()
    s = pkg.Solver(cfg)
    s.set_geometry(loops)
    s.step(5)
    ref = s.get_loads()["mass"]
    arrays = [_level_arrays(s, l) for l in range(cfg["levels"])]
    outs = _outputs()
    m1, b1 = _mass_noalloc(arrays, cfg["levels"], outs)
    # after that first call (which looks up the scratch address on this device) a call
    # leaves the device's free memory unchanged: it allocates nothing
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    m2, b2 = _mass_noalloc(arrays, cfg["levels"], outs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert b1 == 0 and b2 == 0
    # same FP64 sum of the same FP32 values, different summation order
    assert abs(m1 - ref) <= 1e-12 * ref, (m1, ref)
    assert abs(m2 - ref) <= 1e-12 * ref, (m2, ref)
    # a later state: the shared scratch keeps no result of the earlier calls
    s.step(3)
    ref2 = s.get_loads()["mass"]
    arrays2 = [_level_arrays(s, l) for l in range(cfg["levels"])]
    m3, _ = _mass_noalloc(arrays2, cfg["levels"])
    assert abs(m3 - ref2) <= 1e-12 * ref2, (m3, ref2)
    # a non-finite velocity in an active cell is reported
    a0 = arrays2[0][0]
    k = int(torch.nonzero(a0["flags"])[0])
    a0["ux"][k] = float("nan")
    _, bad = _mass_noalloc(arrays2, cfg["levels"])
    assert bad == 1
    s.close()


def test_noalloc_rejects_oversized_input():
    import torch

    torch.cuda.set_device(0)
    buf = torch.zeros(4, device="cuda")
    rc = pkg.level_mass_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                (1 << 26) + 1, 1.0, buf.data_ptr(), buf.data_ptr(), 0)
    assert rc == -1
