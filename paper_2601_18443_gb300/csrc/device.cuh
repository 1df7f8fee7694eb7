// device.cuh -- device-side views of the tiled levels and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.hpp"
#include "../../include/lbm.h"

namespace lbmdev {

// One level of the sparse tiled grid (device pointers).  Slot indices are 32-bit:
// the host rejects levels with 9 * n_slots >= 2^31.
struct LevelView {
    int ntiles;
    int ns;                       // cell slots = ntiles * 256
    int n_wall_tiles;             // tiles [0, n_wall_tiles) hold boundary nodes
    const int *tile_x, *tile_y;   // tile coordinates (global, in tiles)
    const int *nbr;               // 9 per tile, D2Q9 order, -1 absent
    const int *child;             // 4 per tile: tiles of level l+1, index b * 2 + a
    const int *parent;            // tile of level l-1 holding the parents, or -1
    const int *band_tiles;        // tiles with band cells
    int n_band_tiles;
    const int *work_tiles;        // tiles with active or ghost fluid cells (the level kernel's grid),
                                  // those with boundary nodes first, then with band or coalescing
                                  // cells, then other active cells, then ghosts only
    int n_work_tiles;
    const int *work_warps;        // tile * 8 + w for each warp w (work shape 0) of a work tile that
    int n_work_warps;             // holds an active or ghost fluid cell (the warp-list schedule)
    const uint32_t *flags;        // per slot
    const float *inv_d2;          // 1 / d^2, d the wall distance in level lattice units (SA-neg)
    const int *aux;               // per slot: wall record of a B node (finest level), band index of a
                                  // band cell, 4 * (parent's band index) + child index of a ghost, or -1
    void *f;                      // populations f - w, [d * ns + slot], one lattice in the AA layout
                                  // (storage type: store); see the level kernel for the layout
    int store;                    // 0 FP32, 1 FP16, 2 BF16 population storage (arithmetic is FP32)
    float *ebuf;                  // 9 per band cell: its last post-collision f - w (the explosion)
    float *gbuf;                  // 36 per band cell: f - w its four ghost children pulled in the
                                  // fine level's second sub-step (the coalescence)
    int n_band;                   // band cells
    float *drho[2], *ux[2], *uy[2];  // macroscopic fields (rho - 1, u) at the two time levels
    float *chi[2];                // nu_tilde / nu at the two time levels
    float nu;                     // lattice viscosity of the level
};

// Wall records (finest level), structure of arrays.
struct RecView {
    int n;
    const int *bslot;             // slot of the boundary node
    const int *ns;                // reference stencil size
    const int *st_slot;           // 16 per record
    const float *st_wr;           // 16 per record: inverse-distance weights of rho at R (normalised)
    const float *st_wu;           // 16 per record: weights of u at R (intercept row of the linear LSQ, or the IDW weights)
    const float *nx, *ny, *dwb;   // unit normal (wall -> fluid), wall distance of B
    const float *q;               // 9 per record: wall fraction of cut pulled directions
    const int *loop;
    const float *slip;            // prescribed slip per loop (wall model 2), 2 per loop
    float *drhoW, *uWx, *uWy, *utau, *chiB, *tx, *ty, *ut;
    float *utau_start;            // Newton start of the next step (written by the step only)
    float *fpost;                 // 9 per record: post-collision f - w of the boundary node, last step
    const uint32_t *nfluid;       // per record: bit q set where the node B + c_q is active fluid
                                  // (present and not solid), for eq 27's interpolation
    const float *yc;              // 18 per record: 1 / (1 + q_c) and q_c / (1 + q_c) per direction
                                  // (eq 27's interpolation weights)
};

struct StepConsts {
    int level0_edges;   // level 0 of a non-periodic box
    int nx0, ny0, ntx0; // level-0 cells and tiles per row
    int turbulence;
    int wall_model;
    int sa_convection;  // 0 Lax-Wendroff, 1 first-order upwind
    int outlet;         // 0 linear extrapolation (Yu), 1 zero gradient
    float U;            // inlet lattice velocity
    float chi_inf;
    float d_wr, d_wv;
    int sms;            // streaming multiprocessors of the device
    float pshift[9];    // 16-bit storage holds g_q - pshift_q (pshift = f_eq(1, U, 0) - w); 0 for FP32
    float *obuf;        // level-0 outlet: [2 parities][2 columns N-1, N-2][directions 2, 6, 8][ny0]
                        // post-collision f - w; a step at parity p reads [p] and writes [p ^ 1]
};

// device status word bits (lbm_step maps them to lbm_status codes).  TIMEOUT is reserved
// for a kernel that waits on a flag with an iteration limit; no kernel here waits.
#define LBM_STATUS_NONFINITE 1
#define LBM_STATUS_TIMEOUT 2
#define LBM_STATUS_BOUNDS 4     // a table-derived index left its buffer (LBM_BOUNDS_CHECK builds)

// What one launch of the fused level kernel does besides the level's own update.
struct LevelStep {
    int p;              // time level of this level (reads [p], writes [p ^ 1]); also the parity of
                        // the in-place population update (0 even, 1 odd)
    int has_child;      // level l+1 exists
    int is_level0;      // level 0 (box-edge conditions may apply)
    int wall;           // this level holds the wall records (finest level)
    int restrict_up;    // write the restriction of this level's new fields into level l-1
    int pp;             // time level of level l-1 (restriction writes [pp ^ 1])
    int shape;          // cells of a warp: 0 a 16 x 2 block, 1 a 32 x 1 row of the tile
    int *status;        // device status word (LBM_STATUS_* bits)
    unsigned long long *tl;  // launch timeline (lbm_set_timeline): 3 clock readings a block from
    int tl_base;             // record tl_base + blockIdx.x, or null
};

// Launch variant of a level's kernels (chosen by lbm_autotune): the register budget of the
// fused level kernel, as the minimum resident blocks per SM (5 or 6), whether its blocks
// persist over several tiles, the cells a warp covers within the tile, and whether
// launches use programmatic dependent launch.  Every variant computes the same numbers
// up to FP32 rounding.
struct LevelTune {
    int min_blocks;
    int pdl;
    int sched;          // LBM_SCHED_TILE: one block per work tile; LBM_SCHED_PERSIST: a grid of
                        // 2 x SMs x min_blocks blocks striding over the work tiles;
                        // LBM_SCHED_WARPS: two-warp blocks over the work-warp list (shape 0)
    int shape;          // work shape of a warp (LevelStep::shape)
};


// launchers (kernels.cu); all enqueue on the given stream
void launch_level(cudaStream_t st, const LevelView &P, const LevelView *F, const LevelView *C, const RecView &R,
                  const StepConsts &k, const LevelStep &ls, const LevelTune &tu);
void launch_prolong(cudaStream_t st, const LevelView &P, const LevelView &F, int p, int pdl,
                    unsigned long long *tl = nullptr, int tl_base = 0);
void launch_wallfn(cudaStream_t st, const LevelView &P, int p, const RecView &R, const StepConsts &k);
void launch_restrict(cudaStream_t st, const LevelView &P, const LevelView &F, int pp, int pf);
void launch_init_feq(cudaStream_t st, const LevelView &P, const float *feq9, float U, float chi_inf);
void launch_fill9(cudaStream_t st, float *buf, long long n, const float *g9);
// the in-place layout <-> logical post-collision populations (f - w) of the active cells,
// [q * ns + slot] on the device; p is the parity of the level's next step; C (gather) is
// the parent level (ghosts report its exploded values)
void launch_gather_post(cudaStream_t st, const LevelView &P, const LevelView *C, const RecView &R, const StepConsts &k,
                        int p, int is_level0, float *out);
void launch_store_post(cudaStream_t st, const LevelView &P, const RecView &R, const StepConsts &k, int p, int is_level0,
                       const float *in);
void launch_explode(cudaStream_t st, const LevelView &P, const LevelView &F, const RecView &R, const StepConsts &k,
                    const float *post);

// Batched launches: one launch advances the same level of up to LBM_BATCH_MAX resident
// solves.  Each solve's views travel in the kernel's parameter block; a block finds its
// solve from its index (the solve's blocks are consecutive from first_block).
#define LBM_BATCH_MAX 24
struct SolveDesc {
    LevelView P, F, C;   // the level, its finer level (or P) and its coarser level (or P)
    RecView R;
    StepConsts k;
    LevelStep ls;
    int kind;            // 0 no finer level, 1 with a finer level, 2 finest level with wall records
    int first_block;
};
struct BatchArgs {
    int n;               // solves in this launch
    SolveDesc d[LBM_BATCH_MAX];
};
struct ProlongDesc {
    LevelView P, F;
    int p, first_block;
};
struct ProlongBatchArgs {
    int n;
    unsigned long long *tl;   // launch timeline (as LevelStep::tl), or null
    int tl_base;
    ProlongDesc d[LBM_BATCH_MAX];
};
void launch_level_batch(cudaStream_t st, const BatchArgs &a, int store, unsigned grid, int pdl);
void launch_prolong_batch(cudaStream_t st, const ProlongBatchArgs &a, unsigned grid, int pdl);

struct LoadsView {
    int nseg;
    const int *b1, *b2;
    const double *w1, *w2, *tx, *ty, *nx, *ny, *ds;
    double *cp, *cf;
};
void launch_loads(cudaStream_t st, const LoadsView &S, const RecView &R, float U, double *acc4);
void launch_mass(cudaStream_t st, const LevelView &P, int p, double area, double *acc, int *status);
void launch_hist_push(cudaStream_t st, const double *acc, double *ring, int slot, long long step, double chord);

}  // namespace lbmdev
