// device.cuh -- device-side views of the tiled levels and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.hpp"

namespace lbmdev {

// One level of the sparse tiled grid (device pointers).
struct LevelView {
    int ntiles;
    long long ns;                 // cell slots = ntiles * 256
    const int *tile_x, *tile_y;   // tile coordinates (global, in tiles)
    const int *nbr;               // 9 per tile, D2Q9 order, -1 absent
    const int *child;             // 4 per tile: tiles of level l+1, index b * 2 + a
    const uint32_t *flags;        // per slot
    const float *dist;            // wall distance (level lattice units)
    const int *rec;               // wall record of a B node (finest level) or nullptr
    float *f[2];                  // populations f - w, [q * ns + slot]
    float *drho, *ux, *uy;        // macroscopic fields at the level's current time (rho - 1)
    float *chi[2];                // nu_tilde / nu
    float nu;                     // lattice viscosity of the level
};

// Wall records (finest level), structure of arrays.
struct RecView {
    int n;
    const int *bslot;             // slot of the boundary node
    const int *ns;                // reference stencil size
    const int *st_slot;           // 16 per record
    const float *st_dx, *st_dy;   // stencil cell centre minus R (finest cells)
    const float *nx, *ny, *dwb;   // unit normal (wall -> fluid), wall distance of B
    const float *q;               // 9 per record: wall fraction of cut pulled directions
    const int *loop;
    const float *slip;            // prescribed slip per loop (wall model 2), 2 per loop
    float *drhoW, *uWx, *uWy, *utau, *chiB, *tx, *ty, *ut;
};

struct StepConsts {
    int level0_edges;   // level 0 of a non-periodic box
    int nx0, ny0, ntx0; // level-0 cells and tiles per row
    int turbulence;
    int wall_model;
    float U;            // inlet lattice velocity
    float chi_inf;
    float d_wr, d_wv;
};

// launchers (kernels.cu); all enqueue on the given stream
void launch_stream_collide(cudaStream_t st, const LevelView &P, const LevelView *F, int cur, int fcur, int fchicur,
                           const RecView &R, const StepConsts &k, int is_level0);
void launch_sa(cudaStream_t st, const LevelView &P, const LevelView *F, int cur, const RecView &R,
               const StepConsts &k, int is_level0);
void launch_wallfn(cudaStream_t st, const LevelView &P, const RecView &R, const StepConsts &k);
void launch_restrict(cudaStream_t st, const LevelView &P, const LevelView &F, int pchi, int fchi);
void launch_explode_prolong(cudaStream_t st, const LevelView &P, const LevelView &F, int cur, int fcur,
                            const StepConsts &k);
void launch_init_feq(cudaStream_t st, const LevelView &P, const float *feq9, float U, float chi_inf);

struct LoadsView {
    int nseg;
    const int *b1, *b2;
    const double *w1, *w2, *tx, *ty, *nx, *ny, *ds;
    double *cp, *cf;
};
void launch_loads(cudaStream_t st, const LoadsView &S, const RecView &R, float U, double *acc4);
void launch_mass(cudaStream_t st, const LevelView &P, double area, double *acc, int *status);

}  // namespace lbmdev
