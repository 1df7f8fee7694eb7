/*
 * oracle.h -- plain FP64 CPU oracle of the LBM-RANS step of Ponsin & Lozano,
 * "Enhanced Wall Boundary Modeling for Turbulent Flows Using the Lattice
 * Boltzmann Method with Adaptive Cartesian Grids" (arXiv 2601.18443).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA product library.
 *
 * Geometry coordinates returned by the oracle are in finest-level lattice units
 * measured from the box origin (x0, y0): x_lat = (x - x0) / h_finest.
 * Level l cell (i, j) has its centre at ((i + 0.5) * 2^(L-1-l), (j + 0.5) * 2^(L-1-l)).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int levels;            /* L >= 1 levels, 2:1, level 0 coarsest              */
    int nx0, ny0;          /* level-0 cells                                      */
    double x0, y0, h0;     /* box origin and level-0 spacing (chord units)       */
    int layers;            /* cells of level l in each refinement band (Sec 2.1) */
    double chord, Re, Ma;  /* reference chord, Reynolds and Mach numbers         */
    double chi_inf;        /* inlet / initial nu_tilde / nu (Sec 3.1.1: 3)       */
    double d_wr, d_wv;     /* reference / virtual node wall distance, finest cells (Sec 2.3) */
    int turbulence;        /* 0 laminar, 1 SA-neg                                */
    int wall_model;        /* 0 VN slip, 1 Nishimura slip (eq 31), 2 prescribed slip per loop, 3 no-slip */
    int periodic;          /* 1: periodic level-0 box, no domain BCs             */
    int solid_walls;       /* 1: loops are walls; 0: loops only drive refinement */
    int sa_convection;     /* 0 Lax-Wendroff (Sec 2.2), 1 first-order upwind (Sec 3.3) */
    int outlet;            /* level-0 outlet (Sec 3.1.1): 0 Yu's linear extrapolation
                              f_q(N-1) = 2 f_q(N-2) - f_q(N-3); 1 zero gradient f_q(N-1) = f_q(N-2) */
} oracle_config;

typedef struct oracle_solver oracle_solver;

typedef struct {
    double CL, CD, CDp, CDf, mass, dCL;
    long long step;
} oracle_loads;

/* status codes follow the product ABI: 0 ok, <0 error */
int  oracle_create(const oracle_config *cfg, oracle_solver **out);
void oracle_destroy(oracle_solver *s);
const char *oracle_last_error(const oracle_solver *s);
int  oracle_set_geometry(oracle_solver *s, const double *xy, const int *loop_offsets, int n_loops);
int  oracle_set_wall_slip(oracle_solver *s, const double *uw_xy, int n_loops);
int  oracle_step(oracle_solver *s, int n_coarse_steps);
int  oracle_level_box(const oracle_solver *s, int level, int *i0, int *j0, int *nx, int *ny);
int  oracle_get_fields(oracle_solver *s, int level, double *rho, double *ux, double *uy,
                       double *chi, unsigned char *mask, int cap);
int  oracle_set_fields(oracle_solver *s, int level, const double *rho, const double *ux,
                       const double *uy, const double *chi);
int  oracle_get_loads(oracle_solver *s, oracle_loads *out, double *cp_seg, double *cf_seg,
                      int cap, int *n_seg);
int  oracle_get_cut_links(const oracle_solver *s, int *ij_dir, double *q, int cap, int *n);
int  oracle_get_wall_records(const oracle_solver *s, int *ij, double *geo, int *nstencil,
                             int cap, int *n);
int  oracle_get_wall_state(oracle_solver *s, double *state, int cap, int *n);
int  oracle_get_wall_distance(const oracle_solver *s, int level, double *d, int cap);
double oracle_mass(const oracle_solver *s);
/* point probes of the geometry predicates, for sampled checks of large grids */
int  oracle_set_walls(oracle_solver *s, const double *xy, const int *loop_offsets, int n_loops);
int  oracle_probe_cells(const oracle_solver *s, int level, const int *ij, int n, unsigned char *solid,
                        unsigned char *near, double *dist);
int  oracle_probe_links(const oracle_solver *s, const int *ijd, int n, double *q);
int  oracle_threads(void);
void oracle_set_threads(int n);

/* building blocks exported for the closed-form pins */
double oracle_wf_uplus(double yplus);                      /* eq 22 */
double oracle_wf_dudy(double yplus);                       /* eq 21 */
double oracle_wf_utau(double ut, double y, double nu);     /* eq 22 inverted (step 3) */
void   oracle_feq(double rho, double ux, double uy, double *feq9);           /* eq 4 */
void   oracle_collide(const double *f9, double omega_nu, double omega_b, double *out9); /* eqs 5-7 */
void   oracle_sa_source(double chi, double nu, double vort, double d, double *P, double *D); /* eqs 11-17 */
double oracle_sa_update_point(const double *chi9, const double *ux9, const double *uy9,
                              double d, double nu, int convection); /* explicit FD update, eqs 12/16 */
double oracle_sa_convection(const double *nt9, double u, double v, int scheme); /* convective increment */
/* wall state of one boundary node from its stencil (Sec 2.3 steps 1-5, eq 28): out = rho_W,
   u_W (2), u_tau, chi_B, t (2), |u_Rt|; dx, dy: stencil cell centres relative to R */
void   oracle_wall_point(const oracle_config *cfg, double nu, int ns, const double *dx, const double *dy,
                         const double *rho, const double *ux, const double *uy, const double *n, double dwb,
                         const double *slip, double *out);
/* Yu's interpolated slip bounce-back for pulled direction q of a boundary node (eq 27; eq 24
   where the next node along the link is not fluid) */
double oracle_yu_link(int q, double qf, double rhoW, double uWx, double uWy, double f_qo_next, double f_qo_B,
                      double f_q_B, int next_fluid);

#ifdef __cplusplus
}
#endif
#endif
