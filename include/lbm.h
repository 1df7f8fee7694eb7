/*
 * lbm.h -- C ABI of the GB300 (sm_103a) LBM-RANS library.
 *
 * One time step of the lattice Boltzmann RANS method of Ponsin & Lozano,
 * "Enhanced Wall Boundary Modeling for Turbulent Flows Using the Lattice
 * Boltzmann Method with Adaptive Cartesian Grids" (arXiv 2601.18443):
 * D2Q9 central-moment stream-collide relaxing with nu + nu_t (Sec 2.1, eqs 1-10),
 * virtual-node slip-velocity interpolated bounce-back on cut wall links
 * (Sec 2.3, eqs 24-28), SA-neg finite-difference update of nu_tilde (Sec 2.2,
 * eqs 11-17), Rohde explosion/coalescence between 2:1 levels with level
 * sub-cycling (Sec 2.1), and surface loads (Sec 3.1.3, eqs 29-30).
 *
 * Conventions (every entry point):
 *  - Status codes, never exceptions or aborts.  After an error the handle stays
 *    valid for lbm_get_* / lbm_last_error / lbm_destroy.
 *  - All pointer arguments are HOST pointers owned by the caller; inputs are
 *    copied during the call, outputs are written into caller-allocated buffers
 *    whose capacity is passed in.  The handle owns all device memory.
 *  - Coordinates returned for geometry are in finest-level lattice units
 *    measured from the box origin (x0, y0): x_lat = (x - x0) / h_finest.  Level-l
 *    cell (i, j) has its centre at ((i + 0.5) 2^(L-1-l), (j + 0.5) 2^(L-1-l)).
 *  - Field arrays are row-major over the level's present-cell box returned by
 *    lbm_get_level_box: element (j - j0) * nx + (i - i0).
 *  - Every call runs on the solver's CUDA stream (cfg->cuda_stream or a stream
 *    the library creates) and is synchronous unless its name ends in _async.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_solver lbm_solver;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = -1,
    LBM_ERR_OOM = -2,
    LBM_ERR_CUDA = -3,
    LBM_ERR_NO_GEOMETRY = -4,
    LBM_ERR_GEOMETRY = -5,
    LBM_ERR_DIVERGED = -6,
    LBM_ERR_TIMEOUT = -7    /* a device-side wait reached its limit (reserved: no kernel waits) */
} lbm_status;

typedef struct {
    int levels;             /* L >= 1 levels of 2:1 refinement, level 0 coarsest (Sec 2.1)          */
    int nx0, ny0;           /* level-0 cells                                                         */
    double x0, y0, h0;      /* box origin and level-0 cell size, chord units                         */
    int layers;             /* refinement band width in cells of each level (Sec 2.1), >= 3          */
    double chord, Re, Ma;   /* reference chord, Reynolds number on the chord, Mach number            */
    double chi_inf;         /* inlet and initial nu_tilde / nu (Sec 3.1.1: 3)                        */
    double d_wr, d_wv;      /* reference / virtual node wall distances in finest cells (Sec 2.3: 2, 1) */
    int turbulence;         /* 0 laminar, 1 SA-neg                                                   */
    int wall_model;         /* 0 virtual-node slip (Sec 2.3), 1 Nishimura slip (Sec 3.1.5, eq 31; use
                               d_wr = 1.75), 2 prescribed slip per loop, 3 no-slip                   */
    int periodic;           /* 1: periodic level-0 box without domain BCs (nx0 % 32 == 0, ny0 % 8 == 0) */
    int solid_walls;        /* 1: loops are walls; 0: loops only drive the refinement                */
    int store;              /* population storage, FP32 arithmetic: 0 FP32 (f - w_i); 1 FP16, 2 BF16
                               (f - f_eq(1, U, 0), the free-stream equilibrium)                      */
    int sa_convection;      /* SA-neg convection: 0 Lax-Wendroff (Sec 2.2), 1 first-order upwind (Sec 3.3) */
    int outlet;             /* level-0 outlet (Sec 3.1.1), on the post-stream values of the three
                               populations entering from outside: 0 Yu's linear extrapolation
                               f_q(N-1) = 2 f_q(N-2) - f_q(N-3), the form the paper names; 1 the
                               zero-gradient copy f_q(N-1) = f_q(N-2), which lets wake vortices leave
                               (the linear form amplifies them as they cross the last columns)    */
    void *cuda_stream;      /* cudaStream_t to run on, or NULL for a library-owned stream            */
    void *(*dev_alloc)(size_t bytes, void *stream, void *ctx); /* optional device allocator          */
    void (*dev_free)(void *ptr, void *stream, void *ctx);      /* its matching free                  */
    void *alloc_ctx;        /* passed back to dev_alloc / dev_free                                   */
} lbm_config;

typedef struct {
    double CL, CD, CDp, CDf; /* eq 30: lift, drag, pressure and friction drag                        */
    double mass;             /* sum over levels of h_l^2 sum_active rho (finest-cell area units)     */
    double dCL;              /* CL minus the CL of the previous lbm_get_loads call (0 on the first)  */
    long long step;          /* coarse steps taken since lbm_set_geometry                            */
} lbm_loads;

typedef struct {
    int levels;
    long long cells_active[16];   /* active fluid cells per level                                    */
    long long cells_present[16];  /* present cells (active, covered, ghost, solid) per level         */
    long long slots[16];          /* device cell slots per level (tiles x 256)                       */
    long long node_updates_per_step; /* sum_l active_l * 2^l per coarse step                         */
    long long wall_records, cut_links, surface_segments;
    long long kernels_per_step;   /* kernel launches issued per coarse step                          */
    double bytes_per_node_update; /* bytes the fused level step moves per node update (populations, flag
                                     word, chi, rho and u; with SA-neg also chi written, u and 1/d^2 read) */
    double device_bytes;          /* device memory held by the handle                                */
    long long work_tiles[16];     /* tiles per level holding an active or ghost fluid cell           */
    long long work_warps[16];     /* 16 x 2-cell warps of those tiles that hold one (LBM_SCHED_WARPS) */
} lbm_info;

/* Per-kernel-class timing of eagerly launched steps (CUDA events on the solver stream). */
typedef struct {
    int n_classes;
    char name[8][32];
    double total_ms[8];
    long long launches[8];
    long long cells[8];           /* cell slots processed by all launches of the class               */
} lbm_kernel_times;

/* Create a solver from a level/box specification (Sec 2.1, Sec 3.1.1).  No device work
 * beyond creating the stream.  Errors: LBM_ERR_INVALID_ARG for a bad spec, LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_config *cfg, lbm_solver **out);

/* Create a host-only handle: no CUDA call is ever made on it (it runs on machines
 * without a GPU).  lbm_set_geometry builds the grid tables on the host exactly as on a
 * device handle and allocates nothing on a device.  The host-table queries work:
 * lbm_get_level_box, lbm_get_fields with only the mask requested (all field pointers
 * NULL), lbm_get_wall_distance, lbm_get_cut_links, lbm_get_wall_records.  Every other
 * call returns LBM_ERR_NO_GEOMETRY.  cuda_stream and the allocator hooks of cfg are
 * ignored.  Release with lbm_destroy.  Errors: LBM_ERR_INVALID_ARG, LBM_ERR_OOM. */
lbm_status lbm_create_host(const lbm_config *cfg, lbm_solver **out);

/* Build the multilevel grid, cut links and wall records from closed wall polylines
 * (Sec 2.1 pre-processor, Sec 2.3 preprocessing), upload them and initialise the state
 * to the equilibrium of rho = 1, u = (U, 0), chi = chi_inf.  xy: 2 * n_points doubles
 * (x, y) in chord units; loop_offsets: n_loops + 1 ints, loop k = points
 * [loop_offsets[k], loop_offsets[k+1]), first vertex not repeated, any orientation.
 * Errors: LBM_ERR_GEOMETRY (a loop with fewer than 3 vertices or zero area, wall
 * segments that cross, refinement that breaks 2:1 nesting or reaches the box edge, a
 * wall touching a non-finest cell, a reference stencil leaving the finest level),
 * LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_set_geometry(lbm_solver *s, const double *xy, const int *loop_offsets, int n_loops);

/* Memory plan of a geometry without a GPU: builds the grid on the host exactly as
 * lbm_set_geometry does and reports the device bytes a solver would hold (allocations
 * rounded to 256 bytes) and the active cells per level.  No CUDA call is made; all
 * arguments are host memory.  Used to admit solves against a device-memory budget.
 * Errors: as lbm_create and lbm_set_geometry (LBM_ERR_INVALID_ARG, LBM_ERR_GEOMETRY);
 * on error, reason holds the message lbm_last_error would give (NUL-terminated). */
typedef struct {
    int levels;
    long long cells_active[16];     /* active fluid cells per level                     */
    long long node_updates_per_step;/* sum over levels of cells_active[l] * 2^l         */
    long long wall_records;         /* boundary nodes of the finest level               */
    double device_bytes;            /* device memory the solver would allocate           */
    char reason[128];               /* error message, empty on success                  */
} lbm_plan;
lbm_status lbm_plan_geometry(const lbm_config *cfg, const double *xy, const int *loop_offsets, int n_loops,
                             lbm_plan *out);

/* Host threads that grid builds started from the calling thread may use (the size of
 * their OpenMP teams); n <= 0 restores the process default (OMP_NUM_THREADS, else every
 * processor).  Callers that build several grids at once on their own threads give each a
 * share of the processors. */
void lbm_set_host_threads(int n);

/* Digest of the host-built grid, without a GPU: 64-bit FNV-1a over every per-cell level
 * table (kind, solid, band, boundary node, coalescence and cut-link bits, wall distance,
 * record index), the tile tables, the wall records and the surface-segment tables, built
 * exactly as lbm_set_geometry builds them.  The builder runs on host threads; the digest
 * of an input does not depend on their number.  *digest (host) is set to 0 on error.
 * Errors: as lbm_plan_geometry (LBM_ERR_INVALID_ARG, LBM_ERR_GEOMETRY). */
lbm_status lbm_grid_digest(const lbm_config *cfg, const double *xy, const int *loop_offsets, int n_loops,
                           unsigned long long *digest);

/* Prescribed wall slip velocity per loop for wall_model 2 (lattice units): uw_xy holds
 * 2 * n_loops doubles.  Errors: LBM_ERR_INVALID_ARG, LBM_ERR_NO_GEOMETRY. */
lbm_status lbm_set_wall_slip(lbm_solver *s, const double *uw_xy, int n_loops);

/* Advance n_coarse_steps level-0 steps (each: 2^l sub-steps of level l, Sec 2.1).
 * Synchronous: returns after the work completes; checks the device status word and
 * the non-finite flag.  Errors: LBM_ERR_NO_GEOMETRY, LBM_ERR_DIVERGED, LBM_ERR_CUDA. */
lbm_status lbm_step(lbm_solver *s, int n_coarse_steps);

/* Enqueue n_coarse_steps on the solver stream without waiting (no status check);
 * pair with lbm_synchronize. */
lbm_status lbm_step_async(lbm_solver *s, int n_coarse_steps);

/* Wait for enqueued work and check the status word (as lbm_step). */
lbm_status lbm_synchronize(lbm_solver *s);

/* Present-cell box of a level: cells i in [i0, i0 + nx), j in [j0, j0 + ny).  Works on
 * host-only handles. */
lbm_status lbm_get_level_box(lbm_solver *s, int level, int *i0, int *j0, int *nx, int *ny);

/* Copy a level's macroscopic fields to the host (any pointer may be NULL).  cap is the
 * element capacity of each array (>= nx * ny).  rho, ux, uy in lattice units; nu_tilde_ratio
 * is nu_tilde / nu (chi).  Cells without values hold NaN.  mask: 0 absent, 1 active fluid,
 * 2 boundary node B, 3 covered, 4 ghost, 5 solid.  On a host-only handle only the mask
 * may be requested (LBM_ERR_NO_GEOMETRY otherwise). */
lbm_status lbm_get_fields(lbm_solver *s, int level, double *rho, double *ux, double *uy,
                          double *nu_tilde_ratio, unsigned char *mask, int cap);

/* Copy a level's populations f_i (eq 1, index i = 0..8 in the order of eq 2) to the host:
 * pop[i * nx * ny + (j - j0) * nx + (i - i0)] over the box of lbm_get_level_box, the
 * post-collision values the next step streams.  Cells without populations of their own
 * (absent, solid, covered) hold NaN, and so do the values the in-place layout does not
 * keep because no step reads them (populations leaving across the inlet or the outlet, or
 * towards a cell without a tile).  Ghost cells report the values they relay next: their
 * parent's exploded populations at a coarse-step boundary.  cap: element capacity
 * (>= 9 nx ny).  The device scratch of the query goes through dev_alloc when given. */
lbm_status lbm_get_populations(lbm_solver *s, int level, double *pop, long long cap);

/* One launch of the level schedule of Sec 2.1, for element-wise checks of single launches
 * against an independent implementation: kind 0 the fused step of `level` (wall function on
 * the finest level, SA-neg, stream with coalescence and cut links, collide, explode), kind 1
 * the same with the restriction of its new fields into the covered cells of level - 1 (the
 * second of two sub-steps), kind 2 the prolongation of level's fields into the ghosts of
 * level + 1.  Synchronous; the status word is checked as in lbm_step.  Afterwards the levels
 * are out of the recursive schedule: lbm_step and lbm_step_async return
 * LBM_ERR_INVALID_ARG until lbm_set_state restores a checkpoint.  No paper counterpart.
 * Errors: LBM_ERR_INVALID_ARG (bad level or kind: kind 2 on the finest level),
 * LBM_ERR_NO_GEOMETRY, LBM_ERR_CUDA, LBM_ERR_DIVERGED. */
lbm_status lbm_step_launch(lbm_solver *s, int level, int kind);

/* The coalescence inputs of a level's band cells (Rohde, Sec 2.1): for band cell b (the
 * active cells of `level` beside a covered one, in row-major order of the level's box) its
 * global cell indices ij[2 b], ij[2 b + 1] and, for each child m = 2 by + bx and direction i,
 * vals[36 b + 9 m + i]: the population f_i its ghost child pulled in the fine level's last
 * odd sub-step (the parent's exploded value where the child keeps its own).  With ij NULL
 * only *n is set.  Errors: LBM_ERR_INVALID_ARG (level without a finer level, capacity),
 * LBM_ERR_NO_GEOMETRY, LBM_ERR_CUDA. */
lbm_status lbm_get_ghost_relay(lbm_solver *s, int level, int *ij, double *vals, int cap, int *n);

/* Set the macroscopic fields of the active fluid cells of a level (NULL = keep) and
 * reset their populations to the equilibrium of eq 4; the interfaces are re-synchronised
 * (restriction, explosion, ghost reconstruction).  Arrays as in lbm_get_fields. */
lbm_status lbm_set_fields(lbm_solver *s, int level, const double *rho, const double *ux,
                          const double *uy, const double *nu_tilde_ratio);

/* Surface loads (eqs 29-30) from the wall function evaluated on the current state.
 * cp_seg / cf_seg (may be NULL) receive per-segment C_p and signed C_f, n_seg_cap their
 * capacity; *n_seg the number of surface segments. */
lbm_status lbm_get_loads(lbm_solver *s, lbm_loads *out, double *cp_seg, double *cf_seg,
                         int n_seg_cap, int *n_seg);

/* Geometry tables (host copies, for inspection and bit-exact comparison).
 * cut links (finest level, ordered by (j, i, dir)): ij_dir[3k] = i, j, pulled direction
 * 1..8 (paper index 2..9), q[k] = wall fraction of eq 27.  Wall records (ordered by
 * (j, i)): ij[2r]; geo[9r] = IW x, IW y, n x, n y, d_WB, R x, R y, loop, segment;
 * nstencil[r] = reference-stencil size.  Wall state (wall function on the current
 * state): st[8r] = rho_W, u_W x, u_W y, u_tau, chi_B, t x, t y, |u_Rt|.  Any pointer
 * may be NULL to query the count.  Cut links and wall records also work on host-only
 * handles; the wall state needs the device state. */
lbm_status lbm_get_cut_links(lbm_solver *s, int *ij_dir, double *q, int cap, int *n);
lbm_status lbm_get_wall_records(lbm_solver *s, int *ij, double *geo, int *nstencil, int cap, int *n);
lbm_status lbm_get_wall_state(lbm_solver *s, double *st, int cap, int *n);

/* Reference-point stencils of the wall records (step 1 of Sec 2.3), in record order:
 * for record r and entry m < 16, sij[32r + 2m] = i, sij[32r + 2m + 1] = j of the
 * finest-level stencil cell (-1 past the record's stencil size), and the FP64 weights
 * the device applies: rho_R = sum wr[16r + m] rho_m (inverse squared distance, normalised)
 * and u_R = sum wu[16r + m] u_m (intercept row of the linear least-squares fit, or the
 * inverse-distance weights where the fit is undefined); 0 past the stencil size.  cap is
 * the record capacity; sij NULL queries the count.  Works on host-only handles. */
lbm_status lbm_get_wall_stencils(lbm_solver *s, int *sij, double *wr, double *wu, int cap, int *n);

/* Surface-element map of the loads (Sec 3.1.3, eqs 29-30): for wall segment k (in loop
 * order, zero-length segments of coincident snapped vertices dropped), mid[2k], mid[2k+1]
 * = its midpoint in finest lattice units from the box origin; b12[2k], b12[2k+1] = the
 * two nearest wall records (boundary-node centres; ties to the lower record index, -1
 * if none) and w12 their inverse squared distances, the weights of the segment's C_p and
 * C_f.  cap is the segment capacity; b12 NULL queries the count.  Works on host-only
 * handles. */
lbm_status lbm_get_segment_map(lbm_solver *s, double *mid, int *b12, double *w12, int cap, int *n);

/* The 32-bit flag word the level kernel reads for each cell of a level's box (0 where the
 * cell has no slot): bits 0-1 kind (0 absent, 1 active, 2 covered, 3 ghost), bit 2 solid,
 * bit 3 band (active, with ghost children on the next level), bit 4 boundary node,
 * bits 5-12 coalesced pulled directions 1..8, bits 13-20 cut pulled directions 1..8,
 * bits 21-24 level-0 inlet, outlet, bottom and top columns/rows (non-periodic boxes).
 * Element (j - j0) * nx + (i - i0); cap >= nx * ny.  Works on host-only handles. */
lbm_status lbm_get_flags(lbm_solver *s, int level, unsigned int *flags, int cap);

/* Wall distance of the active fluid cells of a level (level lattice units, NaN elsewhere).
 * Works on host-only handles. */
lbm_status lbm_get_wall_distance(lbm_solver *s, int level, double *d, int cap);

/* Sizes, counts and the algorithmic bytes per node update. */
lbm_status lbm_get_info(lbm_solver *s, lbm_info *out);

/* Run n_coarse_steps with every kernel launched eagerly and bracketed by CUDA events on
 * the solver stream; accumulate device time per kernel class.  Same results as lbm_step. */
lbm_status lbm_time_kernels(lbm_solver *s, int n_coarse_steps, lbm_kernel_times *out);

/* Grid schedules of the fused level kernel (lbm_autotune, lbm_set_launch_variant). */
#define LBM_SCHED_TILE 0      /* one 256-thread block per work tile                              */
#define LBM_SCHED_PERSIST 1   /* a grid of 2 x SMs x budget blocks striding over the work tiles  */
#define LBM_SCHED_WARPS 2     /* two-warp blocks over the list of work warps (16 x 2 cells each
                                 of a work tile that hold an active or ghost fluid cell; shape 0),
                                 ordered warps with boundary nodes, with band or coalescing cells,
                                 with other active cells, with ghosts only                      */
#define LBM_SCHED_WARPS4 3    /* four-warp blocks over the same list (shape 0)                    */

/* Launch autotuner.  Not part of the paper's method (Sec 2.1 gives the level schedule, not
 * its mapping to a GPU).  For each level it picks one of LBM_TUNE_CANDIDATES launch forms
 * of the fused level kernel: a register budget of at most 48 or 40 registers a thread (at
 * least 5 or 6 resident 256-thread blocks per SM), each with one of the grid schedules
 * LBM_SCHED_* and, for the tile schedules, one of two work shapes of a warp within the
 * 32 x 8 cell tile (shape 0: a 16 x 2 block of cells; shape 1: a 32-cell row, whose
 * accesses shifted by one cell touch fewer sectors and whose restriction goes through
 * shared memory).  The choice comes from per-launch CUDA-event timings of `steps` eager
 * coarse steps per candidate, and is kept only if `steps` coarse steps through the step
 * graphs confirm it (against the same choice with one block per tile where it picked a
 * persistent grid, against the form before tuning, and against each candidate on every
 * level; the fastest of these is kept), since launches overlap inside the
 * graphs.  Then it picks whether launches use programmatic dependent launch, from the time
 * of `steps` coarse steps through the step graphs each way, and recaptures the graphs with
 * the choice.  The variants compute the same numbers up to FP32 rounding (the compiler
 * schedules and contracts the arithmetic differently per variant); the timed steps are real
 * steps of the solve (steps_taken of them).
 * Synchronous.  Errors as lbm_step. */
#define LBM_TUNE_CANDIDATES 12
typedef struct {
    int levels;
    int candidate_min_blocks[LBM_TUNE_CANDIDATES];
    int candidate_sched[LBM_TUNE_CANDIDATES];
    int candidate_shape[LBM_TUNE_CANDIDATES];
    double level_us[LBM_TUNE_CANDIDATES][16]; /* mean launch time of level l's kernel per candidate */
    int min_blocks[16];                       /* chosen register budget per level                  */
    int sched[16];                            /* chosen grid schedule per level (LBM_SCHED_*)      */
    int shape[16];                            /* chosen work shape per level                       */
    double step_us_confirm[3 + LBM_TUNE_CANDIDATES]; /* coarse step: per-level pick, pick with
                                                 tile blocks for persistent grids, form before
                                                 tuning, then each candidate on every level    */
    int confirm_choice;                       /* index into step_us_confirm of the form kept    */
    double default_step_us;                   /* coarse step through the graphs before tuning      */
    double step_us[2];                        /* coarse step, chosen kernels, PDL off / on         */
    int pdl;                                  /* chosen: 1 programmatic dependent launch on        */
    long long steps_taken;                    /* coarse steps the tuning advanced the solve by     */
} lbm_tune_report;
lbm_status lbm_autotune(lbm_solver *s, int steps, lbm_tune_report *out);

/* Checkpoint and resume.  Not in the paper.  lbm_get_state copies the solve's state at the
 * current level-0 step into a host buffer: for every level its populations and its rho - 1,
 * u, chi at the current time level (raw device layout), the wall records' Newton start
 * values, the step count and the last C_L.  With buf NULL it only returns the size.  That
 * is enough to continue bit for bit: lbm_set_state into a solver created with the same
 * configuration and geometry (or into the same solver, to rewind) makes its next steps
 * equal to those the saved solve would have taken.  The blob records the grid (a hash of
 * the cell flags), and set_state rejects a blob from another configuration or grid with
 * LBM_ERR_INVALID_ARG.  It also clears the device status word.  Both calls are
 * synchronous.  The wall-function outputs (lbm_get_wall_state) are not part of the state;
 * the next step or lbm_get_loads recomputes them.  Errors: LBM_ERR_INVALID_ARG,
 * LBM_ERR_NO_GEOMETRY, LBM_ERR_CUDA. */
lbm_status lbm_get_state(lbm_solver *s, void *buf, size_t cap, size_t *size);
lbm_status lbm_set_state(lbm_solver *s, const void *buf, size_t size);

/* Set the launch variant directly (for instance one lbm_autotune found on a solve of the
 * same shape): min_blocks[l] in {5, 6}, sched[l] one of LBM_SCHED_* and shape[l] in {0, 1}
 * (NULL: shape 0 on every level; the warp-list schedules require shape 0) for each of the solver's
 * levels, pdl 0 or 1; the step graphs are recaptured.  No device work.  Errors:
 * LBM_ERR_INVALID_ARG for a value outside those sets, LBM_ERR_NO_GEOMETRY. */
lbm_status lbm_set_launch_variant(lbm_solver *s, const int *min_blocks, const int *sched, const int *shape,
                                  int pdl);

/* The level kernel's work lists of a level, in launch order (also on host-only handles):
 * warps 0 gives the work tiles (tiles holding an active or ghost fluid cell), warps 1 the
 * work warps (the 16 x 2-cell warps w of those tiles, cells x in [16 (w & 1), +16), y in
 * {2 (w >> 1), +1} of the tile, that hold one); both ordered by cost class (a boundary node
 * of the finest level 3, a band or coalescing cell 2, another active cell 1, ghosts only 0;
 * non-increasing), tile order within a class.  out holds 3 ints per entry: the global cell
 * indices i, j of the tile's first cell and the warp (-1 for tiles); with cap 0 only the
 * count.  Errors: LBM_ERR_INVALID_ARG, LBM_ERR_NO_GEOMETRY. */
lbm_status lbm_get_work_list(lbm_solver *s, int level, int warps, int *out, int cap, int *n);

/* Load history.  With every > 0, lbm_step and lbm_step_async enqueue, after each coarse step
 * whose count is a multiple of every, what lbm_get_loads computes (the wall state query,
 * eq 29-30 with their FP64 sums, the FP64 mass) into the next slot of a device ring of
 * capacity records, without a host synchronisation; the trajectory is unchanged (the query
 * leaves the next step's Newton start alone).  lbm_get_load_history returns the kept records
 * (the last capacity ones) oldest first, after synchronising the stream; the coefficients
 * equal what lbm_get_loads gives at the same step up to the order of the FP64 sums.  every
 * 0 stops recording; a new call clears the ring.  lbm_batch_step records nothing.  Errors:
 * LBM_ERR_INVALID_ARG (capacity < 1 with every > 0; cap below the record count: call with
 * cap 0 for it), LBM_ERR_NO_GEOMETRY, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_CUDA. */
typedef struct {
    long long step;          /* coarse steps taken since lbm_set_geometry                      */
    double CL, CD, CDp, CDf; /* eq 30                                                           */
    double mass;             /* as lbm_loads.mass                                              */
} lbm_load_record;
lbm_status lbm_set_load_history(lbm_solver *s, int every, int capacity);
lbm_status lbm_get_load_history(lbm_solver *s, lbm_load_record *out, int cap, int *n);

/* Launch timeline.  Not in the paper.  With the timeline on, every block of every launch of
 * the step graphs records the GPU's global timer when it has passed its wait for the
 * preceding kernel and when all its threads are done (one thread's clock reads and stores
 * per block, a block barrier at its end); lbm_get_timeline reduces them per launch for the
 * most recent run of each of the two step graphs (level-0 parities), in launch order, times
 * from the first launch of that graph.  lbm_set_timeline recaptures the step graphs (on 1
 * allocates the records, 24 bytes a block of each launch; off 0 keeps them).  Results are
 * those of the steps without it.  Errors: LBM_ERR_INVALID_ARG (cap below the launch count:
 * call with cap 0 for the count), LBM_ERR_NO_GEOMETRY, LBM_ERR_OOM, LBM_ERR_CUDA. */
typedef struct {
    int graph;          /* step graph: the level-0 parity it starts from                         */
    int level;          /* level of the step, or the first level of a prolongation launch        */
    int kind;           /* 0 even sub-step, 1 odd sub-step, 2 prolongation                        */
    int blocks;         /* blocks that recorded                                                   */
    double t_wait_us;   /* first block past its wait for the preceding kernel                    */
    double t_end_us;    /* last block done                                                        */
} lbm_launch_time;
lbm_status lbm_set_timeline(lbm_solver *s, int on);
lbm_status lbm_get_timeline(lbm_solver *s, lbm_launch_time *out, int cap, int *n);

/* Launch grouping of the prolongations (Sec 2.1): in each descent of the recursive schedule
 * the prolongations of consecutive levels l - 1, l go out as one launch (on by default)
 * where level l's band cells have no ghost cell of level l in their 3 x 3 neighbourhood, so
 * that neither reads what the other writes.  on 0 launches each on its own.  merged_levels
 * (may be NULL) returns the number of levels l whose prolongation can join the one of
 * l - 1.  The step graphs are recaptured.  No device work.  Errors: LBM_ERR_INVALID_ARG,
 * LBM_ERR_NO_GEOMETRY. */
lbm_status lbm_set_prolong_merge(lbm_solver *s, int on, int *merged_levels);

/* Per level l (indep[0 .. levels - 1]), 1 where the prolongation of level l may share a
 * launch with that of level l - 1: 1 <= l <= levels - 2 and no band cell of level l has a
 * ghost cell of level l among its eight neighbours.  Also on host-only handles.  Errors:
 * LBM_ERR_INVALID_ARG (cap below the level count), LBM_ERR_NO_GEOMETRY. */
lbm_status lbm_get_prolong_independence(lbm_solver *s, int *indep, int cap);

/* Largest n_cells that lbm_level_mass_noalloc accepts (its fixed scratch holds 4096
 * per-block partial sums of at most 16384 cells each). */
#define LBM_NOALLOC_MAX_CELLS 67108864LL

/* FP64 mass and finiteness check of one level's fields, allocating nothing.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (code running inside another framework's stream capture, real-time loops
 * with a fixed memory plan, allocators owned by someone else).  It computes the same
 * quantities as the mass of lbm_get_loads and the non-finite check of lbm_step:
 *   *mass_out = sum over cells with (flags & 3) == 1 (active) and flags bit 2 clear
 *               (fluid) of area * (1 + drho), in FP64;
 *   *nonfinite_out = 1 if any such cell has a non-finite drho, ux, uy or nu_tilde_ratio.
 * All array arguments and both outputs are DEVICE pointers of n_cells elements (outputs:
 * one element), owned by the caller and on the current device; stream is a
 * cudaStream_t (NULL = legacy default stream).  The call only enqueues work: read the
 * outputs after synchronising the stream.
 * Scratch: a fixed 48 KB array in device memory (file scope), held by every GPU that
 * loads the library until the process exits.  The first call on a device looks up that
 * array's device address (make it before any stream capture) and keeps it for the process;
 * after a cudaDeviceReset of that device the kept address is stale, so do not call this
 * entry point on a device that has been reset.  Every call on a device shares the array:
 * calls that overlap on the GPU (other streams, other threads) race.
 * Errors: LBM_ERR_INVALID_ARG for n_cells < 0, n_cells > LBM_NOALLOC_MAX_CELLS or a NULL
 * pointer (nothing is launched); LBM_ERR_CUDA if the device or the launch fails. */
lbm_status lbm_level_mass_noalloc(const unsigned int *flags, const float *drho, const float *ux, const float *uy,
                                  const float *nu_tilde_ratio, long long n_cells, double area, double *mass_out,
                                  int *nonfinite_out, void *stream);

/* ---- Batched solves (serving) -------------------------------------------------------
 * A batch steps up to LBM_BATCH_MAX_SOLVES resident solves in lockstep, one launch per node
 * of the recursive level schedule of Sec 2.1 covering the same level of every member that
 * has it (level l takes 2^l sub-steps per coarse step in every solve, so members with
 * different level counts share the schedule of the deepest one).  Each block of a launch
 * carries its solve's views, so one graph node advances one level of all members.  No paper
 * counterpart: the paper steps one solve at a time.
 *
 * lbm_batch_create: the members (distinct handles with geometry, on the current device,
 * all with the same population storage, none left off the schedule by lbm_step_launch)
 * stay owned by the caller and must outlive the batch.  The batch owns a stream and two
 * captured step graphs.  Errors: LBM_ERR_INVALID_ARG, LBM_ERR_OOM, LBM_ERR_CUDA.
 * lbm_batch_step: enqueue n coarse steps of every member on the batch's stream, ordered
 * after the work already on the members' streams and before later work on them (events),
 * so a member's queries (lbm_synchronize, lbm_get_loads, ...) see the stepped state.  A
 * member must not be stepped on its own while in a batch (LBM_ERR_INVALID_ARG: make a new
 * batch).  Each member's results equal its results stepped alone up to FP32 rounding.
 * lbm_batch_info: members, levels of the deepest member, launches per coarse step.
 * lbm_batch_destroy: NULL-safe; waits for the batch's work. */
#define LBM_BATCH_MAX_SOLVES 24
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(lbm_solver *const *solvers, int n, lbm_batch **out);
lbm_status lbm_batch_step(lbm_batch *b, int n_coarse_steps);
lbm_status lbm_batch_info(const lbm_batch *b, int *members, int *levels, long long *kernels_per_step);
const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* Per-handle message of the last error. */
const char *lbm_last_error(const lbm_solver *s);

/* Free everything the handle owns.  NULL-safe. */
void lbm_destroy(lbm_solver *s);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
