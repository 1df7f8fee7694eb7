/*
 * oracle.c -- plain, slow FP64 CPU oracle of one LBM-RANS time step on a 2:1
 * multilevel cell-centred D2Q9 grid, following Ponsin & Lozano (arXiv 2601.18443).
 *
 * TEST INFRASTRUCTURE ONLY: it is loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA library: it keeps dense per-level arrays with masks, a
 * two-lattice (A/B) pull scheme, the literal 9x9 central-moment transform, and
 * brute-force exact geometry predicates.
 *
 * Every function cites the passage it follows.  Where the paper is silent or
 * garbled, the reading taken is stated next to the code ("reading: ...").
 *
 * Parity pins: each building block is pinned by closed forms and invariants in
 * tests/test_oracle_*.py.  The assembled full-airfoil run has no worked example
 * in the paper ("parity unpinned" for that case as a whole); it is pinned by the
 * pinned parts, by mass conservation, by the uniform-flow and symmetry tests.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

/* ---------------------------------------------------------------------------
 * D2Q9 lattice, eq 2 (0-based; paper index k+1).  Second row of eq 2 is c_iy.
 * ------------------------------------------------------------------------- */
static const int CX[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
static const int CY[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
static const int OPPD[9] = {0, 2, 1, 4, 3, 6, 5, 8, 7};
static const double WQ[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
#define CS2 (1.0 / 3.0)

/* Spalart-Allmaras constants, Sec 2.2 (after eq 17) */
#define SA_CB1 0.1355
#define SA_CB2 0.622
#define SA_SIGMA (2.0 / 3.0)
#define SA_KAPPA 0.41
#define SA_CW1 (SA_CB1 / (SA_KAPPA * SA_KAPPA) + (1.0 + SA_CB2) / SA_SIGMA)
#define SA_CW2 0.3
#define SA_CW3 2.0
#define SA_CV1 7.1
#define SA_RLIM 10.0
#define SA_CV2 0.7
/* reading: c_v3 = 0.9 (the value of the SA-neg source the paper follows, ref [56]); with the printed
   0.3 the second branch of eq 14 has a pole at S_bar = -1.1 Omega inside its own range S_bar < -0.7 Omega */
#define SA_CV3 0.9
#define SA_CT3 1.2
#define SA_CN1 16.0

/* Analytical SA wall-function constants, eq 22 */
#define WF_B 5.033908790505579
#define WF_A1 8.148221580024245
#define WF_A2 (-6.9287093849022945)
#define WF_B1 7.4600876082527945
#define WF_B2 7.468145790401841
#define WF_C1 2.5496773539754747
#define WF_C2 1.3301651588535228
#define WF_C3 3.599459109332379
#define WF_C4 3.639753186868684494

#define MAXL 16
#define FIX_BITS 12               /* fixed-point unit = finest cell / 2^12 */
#define FIX_ONE (1LL << FIX_BITS)
#define D_CAP 1.0e12              /* wall distance used where there is no wall */
/* Smallest wall distance the SA-neg terms of eqs 11-17 see at a fluid node, in lattice
 * units of the node's level.  The paper does not treat a fluid node (no cut link) lying
 * closer than half a spacing to the wall; that happens only beside a wall sliver thinner
 * than the lattice (a sharp trailing edge passing between nodes), where d -> 0 makes the
 * explicit destruction rate 2 c_w1 nu~ / d^2 exceed one per step. */
#define SA_D_MIN 0.5

enum { K_ABSENT = 0, K_ACTIVE = 1, K_COVERED = 2, K_GHOST = 3 };

/* ===========================================================================
 * Wall function (Sec 2.2, eqs 20-22)
 * ========================================================================= */

/* eq 22.  Reading: the arctangents are taken on the continuous branch
 * atan2(b, y+ + a); the literal arctan(b/(y+ + a)) jumps by pi at y+ = -a2. */
double oracle_wf_uplus(double yp)
{
    double t1 = (yp + WF_A1) * (yp + WF_A1) + WF_B1 * WF_B1;
    double t2 = (yp + WF_A2) * (yp + WF_A2) + WF_B2 * WF_B2;
    return WF_B + WF_C1 * log(t1) - WF_C2 * log(t2) - WF_C3 * atan2(WF_B1, yp + WF_A1) -
           WF_C4 * atan2(WF_B2, yp + WF_A2);
}

/* eq 21: du+/dy+ */
double oracle_wf_dudy(double yp)
{
    double k3 = pow(SA_KAPPA * yp, 3.0);
    double c3 = SA_CV1 * SA_CV1 * SA_CV1;
    return (c3 + k3) / (c3 + k3 * (1.0 + SA_KAPPA * yp));
}

/* Step 3 of Sec 2.3: friction velocity from |u_t| sampled at wall distance y, by
 * Newton-Raphson on g(u) = u * u+(u y / nu) - |u_t| (g' = u+ + y+ du+/dy+),
 * kept inside a sign bracket (reading: the paper gives no iteration details). */
double oracle_wf_utau(double ut, double y, double nu)
{
    if (!(ut > 0.0) || !(y > 0.0)) return 0.0;
    double lo = 0.0, hi = sqrt(ut * nu / y);
    if (hi <= 0.0) hi = 1e-300;
    for (int it = 0; it < 4000; it++) {
        double g = hi * oracle_wf_uplus(hi * y / nu) - ut;
        if (g > 0.0) break;
        lo = hi;
        hi *= 2.0;
    }
    double u = 0.5 * (lo + hi);
    for (int it = 0; it < 400; it++) {
        double yp = u * y / nu;
        double g = u * oracle_wf_uplus(yp) - ut;
        if (g > 0.0) hi = u; else lo = u;
        double gp = oracle_wf_uplus(yp) + yp * oracle_wf_dudy(yp);
        double un = (gp > 0.0) ? u - g / gp : 0.5 * (lo + hi);
        if (!(un > lo && un < hi)) un = 0.5 * (lo + hi);
        if (fabs(un - u) <= 4e-16 * un) { u = un; break; }
        u = un;
        if (hi - lo <= 4e-16 * hi) break;
    }
    return u;
}

/* ===========================================================================
 * Equilibrium and central-moment collision (Sec 2.1, eqs 3-10)
 * ========================================================================= */

/* eq 4: fourth-order Hermite equilibrium.  Reading: the H4 coefficient is
 * 1/(4 cs^8) (= 6/4! from the six xxyy permutations); the printed 1/(2 cs^8)
 * does not give the equilibrium fourth central moment rho cs^4. */
void oracle_feq(double rho, double ux, double uy, double *fe)
{
    const double cs4 = CS2 * CS2, cs6 = cs4 * CS2, cs8 = cs4 * cs4;
    for (int i = 0; i < 9; i++) {
        double cx = CX[i], cy = CY[i];
        double cu = cx * ux + cy * uy;
        double h2 = (cx * cx - CS2) * ux * ux + 2.0 * cx * cy * ux * uy + (cy * cy - CS2) * uy * uy;
        double h3xxy = (cx * cx - CS2) * cy, h3xyy = (cy * cy - CS2) * cx;
        double h4 = (cx * cx - CS2) * (cy * cy - CS2);
        fe[i] = WQ[i] * rho *
                (1.0 + cu / CS2 + h2 / (2.0 * cs4) + (h3xxy * ux * ux * uy + h3xyy * ux * uy * uy) / (2.0 * cs6) +
                 h4 * ux * ux * uy * uy / (4.0 * cs8));
    }
}

/* Solve the n x n system A x = b in place (Gaussian elimination, partial pivoting). */
static int solve_dense(int n, double *A, double *b)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int r = k + 1; r < n; r++)
            if (fabs(A[r * n + k]) > fabs(A[p * n + k])) p = r;
        if (A[p * n + k] == 0.0) return -1;
        if (p != k) {
            for (int c = 0; c < n; c++) { double t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t; }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int r = k + 1; r < n; r++) {
            double m = A[r * n + k] / A[k * n + k];
            if (m == 0.0) continue;
            for (int c = k; c < n; c++) A[r * n + c] -= m * A[k * n + c];
            b[r] -= m * b[k];
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        double s = b[k];
        for (int c = k + 1; c < n; c++) s -= A[k * n + c] * b[c];
        b[k] = s / A[k * n + k];
    }
    return 0;
}

/* Row r of the non-orthogonal central-moment basis T of eq 6 for population i,
 * using the shifted velocities of eq 5. */
static double tbasis(int r, double cbx, double cby)
{
    switch (r) {
    case 0: return 1.0;
    case 1: return cbx;
    case 2: return cby;
    case 3: return cbx * cbx + cby * cby;
    case 4: return cbx * cbx - cby * cby;
    case 5: return cbx * cby;
    case 6: return cbx * cbx * cby;
    case 7: return cbx * cby * cby;
    default: return cbx * cbx * cby * cby;
    }
}

/* eqs 3, 5-7: m = T f, m* = (I - K) m + K m_eq, f* = T^-1 m*, with
 * K = diag[1, 1, 1, omega_b, omega_nu, omega_nu, 1, 1, 1].  T^-1 is applied by
 * solving T f* = m* (the oracle does not use the shift-matrix shortcut). */
void oracle_collide(const double *f, double om_nu, double om_b, double *out)
{
    double rho = 0, jx = 0, jy = 0;
    for (int i = 0; i < 9; i++) { rho += f[i]; jx += CX[i] * f[i]; jy += CY[i] * f[i]; }
    double ux = jx / rho, uy = jy / rho;
    double T[81], fe[9], m[9], me[9];
    for (int r = 0; r < 9; r++)
        for (int i = 0; i < 9; i++) T[r * 9 + i] = tbasis(r, CX[i] - ux, CY[i] - uy);
    oracle_feq(rho, ux, uy, fe);
    const double K[9] = {1, 1, 1, om_b, om_nu, om_nu, 1, 1, 1};
    for (int r = 0; r < 9; r++) {
        m[r] = 0; me[r] = 0;
        for (int i = 0; i < 9; i++) { m[r] += T[r * 9 + i] * f[i]; me[r] += T[r * 9 + i] * fe[i]; }
        out[r] = (1.0 - K[r]) * m[r] + K[r] * me[r];
    }
    solve_dense(9, T, out);
}

/* ===========================================================================
 * SA-neg (Sec 2.2, eqs 11-17)
 * ========================================================================= */

static double sa_fv1(double chi)
{
    double c3 = chi * chi * chi;
    return c3 / (c3 + SA_CV1 * SA_CV1 * SA_CV1);
}

/* Production and destruction of eqs 13-17 for nu_tilde = chi * nu at wall
 * distance d with vorticity magnitude vort.  Readings: S_bar = nu_t~ f_v2 /
 * (kappa^2 d^2) (not printed; it gives the log-layer solution of eq 20 exactly);
 * r = r_lim where S_tilde <= 0. */
void oracle_sa_source(double chi, double nu, double vort, double d, double *P, double *D)
{
    double nt = chi * nu;
    if (nt >= 0.0) {
        double fv1 = sa_fv1(chi);
        double fv2 = 1.0 - chi / (1.0 + chi * fv1);
        double sbar = nt * fv2 / (SA_KAPPA * SA_KAPPA * d * d);
        double st;
        if (sbar >= -SA_CV2 * vort)
            st = vort + sbar;
        else
            st = vort + vort * (SA_CV2 * SA_CV2 * vort + SA_CV3 * sbar) / ((SA_CV3 - 2.0 * SA_CV2) * vort - sbar);
        double r = SA_RLIM;
        if (st > 0.0) {
            r = nt / (st * SA_KAPPA * SA_KAPPA * d * d);
            if (r > SA_RLIM) r = SA_RLIM;
        }
        double g = r + SA_CW2 * (pow(r, 6.0) - r);
        double c6 = pow(SA_CW3, 6.0);
        double fw = g * pow((1.0 + c6) / (pow(g, 6.0) + c6), 1.0 / 6.0);
        *P = SA_CB1 * st * nt;
        *D = SA_CW1 * fw * (nt / d) * (nt / d);
    } else {
        *P = SA_CB1 * (1.0 - SA_CT3) * vort * nt;
        *D = -SA_CW1 * (nt / d) * (nt / d);
    }
}

/* diffusion coefficient nu + nu_t~ f_n of eqs 12/16; f_n = 1 for nu_t~ >= 0 */
static double sa_diffusivity(double chi, double nu)
{
    double fn = 1.0;
    if (chi < 0.0) {
        double c3 = chi * chi * chi;
        fn = (SA_CN1 + c3) / (SA_CN1 - c3);
    }
    return nu + chi * nu * fn;
}

/* Unweighted least-squares gradient from the neighbour offsets (Sec 2.2, ref
 * [58]): minimise sum_k (phi_k - phi_0 - g . dx_k)^2 over the listed neighbours. */
static int lsq_gradient(int n, const double *dx, const double *dy, const double *dphi, double *gx, double *gy)
{
    double a11 = 0, a12 = 0, a22 = 0, b1 = 0, b2 = 0;
    for (int k = 0; k < n; k++) {
        a11 += dx[k] * dx[k]; a12 += dx[k] * dy[k]; a22 += dy[k] * dy[k];
        b1 += dx[k] * dphi[k]; b2 += dy[k] * dphi[k];
    }
    double A[4] = {a11, a12, a12, a22}, b[2] = {b1, b2};
    if (n < 2 || solve_dense(2, A, b) != 0) { *gx = 0; *gy = 0; return -1; }
    *gx = b[0]; *gy = b[1];
    return 0;
}

/* Convective increment -dt u . grad(nu_t~) over one step (dt = 1) at the centre of the
 * D2Q9 neighbourhood nt9 (index k at offset (CX[k], CY[k])).
 * scheme 0: Lax-Wendroff (Sec 2.2): -(u d_x + v d_y) phi + (1/2)(u^2 d_xx + 2 u v d_xy + v^2 d_yy) phi
 *           with centred differences.
 * scheme 1: first-order upwind (Sec 3.3, the alternative of Sec 2.2's footnote): one-sided
 *           differences taken from the upstream side of each velocity component. */
double oracle_sa_convection(const double *nt, double u, double v, int scheme)
{
    double c = nt[0], e = nt[1], w = nt[2], n = nt[3], s = nt[4];
    double ne = nt[5], sw = nt[6], se = nt[7], nw = nt[8];
    if (scheme == 1) {
        double dx = u > 0.0 ? c - w : e - c;
        double dy = v > 0.0 ? c - s : n - c;
        return -(u * dx + v * dy);
    }
    double gx = 0.5 * (e - w), gy = 0.5 * (n - s);
    double gxx = e - 2.0 * c + w, gyy = n - 2.0 * c + s, gxy = 0.25 * (ne - nw - se + sw);
    return -(u * gx + v * gy) + 0.5 * (u * u * gxx + 2.0 * u * v * gxy + v * v * gyy);
}

/* One explicit Euler step (dt = 1 lattice step of the level) of eq 12 / eq 16
 * at a node with its 8 D2Q9 neighbours (index k at offset (CX[k], CY[k])).
 * Convection: Lax-Wendroff (Sec 2.2) or first-order upwind (Sec 3.3).  Diffusion:
 * centred, conservative face averages of nu + nu_t~ f_n.  c_b2 |grad nu_t~|^2 with
 * centred gradients.  Vorticity from the LSQ velocity gradient.  Returns chi at the
 * new time. */
double oracle_sa_update_point(const double *chi9, const double *ux9, const double *uy9, double d, double nu,
                              int convection)
{
    double nt[9], dxk[8], dyk[8], du[8], dv[8];
    for (int k = 0; k < 9; k++) nt[k] = chi9[k] * nu;
    for (int k = 1; k < 9; k++) {
        dxk[k - 1] = CX[k]; dyk[k - 1] = CY[k];
        du[k - 1] = ux9[k] - ux9[0]; dv[k - 1] = uy9[k] - uy9[0];
    }
    double dudx, dudy, dvdx, dvdy;
    lsq_gradient(8, dxk, dyk, du, &dudx, &dudy);
    lsq_gradient(8, dxk, dyk, dv, &dvdx, &dvdy);
    double vort = fabs(dvdx - dudy);                         /* Omega = sqrt(2 W:W) in 2D */
    double c = nt[0], e = nt[1], w = nt[2], n = nt[3], s = nt[4];
    double ne = nt[5], sw = nt[6], se = nt[7], nw = nt[8];
    (void)ne; (void)sw; (void)se; (void)nw;
    double gx = 0.5 * (e - w), gy = 0.5 * (n - s);
    double conv = oracle_sa_convection(nt, ux9[0], uy9[0], convection);
    double Dk[9];
    for (int k = 0; k < 9; k++) Dk[k] = sa_diffusivity(chi9[k], nu);
    double De = 0.5 * (Dk[0] + Dk[1]), Dw = 0.5 * (Dk[0] + Dk[2]);
    double Dn = 0.5 * (Dk[0] + Dk[3]), Ds = 0.5 * (Dk[0] + Dk[4]);
    /* diffusion with its diagonal taken at the new time level (point-implicit): the
     * explicit form diverges once (nu + nu~)/sigma passes 1/4 per step; this one has the
     * same steady states and keeps the diffusion a weighted mean at any nu~ */
    double a = (De + Dw + Dn + Ds) / SA_SIGMA;
    double div = De * (e - c) - Dw * (c - w) + Dn * (n - c) - Ds * (c - s);
    double diff = (div + SA_CB2 * (gx * gx + gy * gy)) / SA_SIGMA;
    double P, D;
    oracle_sa_source(chi9[0], nu, vort, d, &P, &D);
    /* (c + conv + P - D + diff + a c) / (1 + a), written as an increment of c */
    double nnew = c + (conv + P - D + diff) / (1.0 + a);
    return nnew / nu;
}

/* ===========================================================================
 * Solver state
 * ========================================================================= */

typedef struct {
    int i0, j0, nx, ny;        /* array box (level-l global cell indices) */
    long long scale;           /* finest cells per level-l cell edge: 2^(L-1-l) */
    double nu;                 /* lattice viscosity of this level (acoustic scaling) */
    unsigned char *kind, *solid, *band, *bnode;
    unsigned short *coal, *cut;
    int *rec;
    double *f, *fn;
    double *rho, *ux, *uy, *chi, *chin, *d;
} olevel;

typedef struct {
    int i, j, seg, loop;
    double iw[2], n[2], dwb, r[2];
    int ns, si[16], sj[16];
    double q[9];
    /* state, refreshed by the wall function */
    double rhoW, uW[2], utau, chiB, t[2], ut;
} orec;

typedef struct { long long x, y; } ipt;

struct oracle_solver {
    oracle_config cfg;
    int L;
    double U;
    char err[256];
    int geometry;
    int nloops, nv, nseg;
    int *loop_off;
    ipt *v;
    int *sa, *sb, *sloop;
    int *loop_ccw;
    double *loop_slip;
    olevel lv[MAXL];
    int nrec;
    orec *rec;
    int *seg_b1, *seg_b2;
    double *seg_w1, *seg_w2;
    long long step;
    double last_cl;
    int have_cl;
};

static int fail(oracle_solver *s, int code, const char *msg)
{
    if (s) snprintf(s->err, sizeof s->err, "%s", msg);
    return code;
}

static long cidx(const olevel *L, long long i, long long j)
{
    if (i < L->i0 || j < L->j0 || i >= L->i0 + L->nx || j >= L->j0 + L->ny) return -1;
    return (long)(j - L->j0) * L->nx + (long)(i - L->i0);
}

/* ===========================================================================
 * Geometry: exact predicates on fixed-point vertices (reading of Sec 2.1's
 * pre-processor: the octree/ADT generator is replaced by distance bands)
 * ========================================================================= */

/* level-l cell centre in fixed-point units */
static ipt centre_fix(const olevel *L, long long i, long long j)
{
    long long h = L->scale * FIX_ONE;
    ipt p = {(2 * i + 1) * (h / 2), (2 * j + 1) * (h / 2)};
    return p;
}

static i128 cross3(ipt a, ipt b, ipt p)
{ /* (b - a) x (p - a) */
    return (i128)(b.x - a.x) * (p.y - a.y) - (i128)(b.y - a.y) * (p.x - a.x);
}

/* Exact: is point p within distance R (fixed units) of segment ab? */
static int seg_within(ipt a, ipt b, ipt p, long long R)
{
    i128 dx = b.x - a.x, dy = b.y - a.y;
    i128 px = p.x - a.x, py = p.y - a.y;
    i128 len2 = dx * dx + dy * dy;
    i128 t = px * dx + py * dy;
    i128 R2 = (i128)R * R;
    if (len2 == 0 || t <= 0) return px * px + py * py <= R2;
    if (t >= len2) {
        i128 qx = p.x - b.x, qy = p.y - b.y;
        return qx * qx + qy * qy <= R2;
    }
    i128 cr = dx * py - dy * px;
    return cr * cr <= R2 * len2;
}

static int near_wall(const oracle_solver *s, ipt p, long long R)
{
    for (int k = 0; k < s->nseg; k++)
        if (seg_within(s->v[s->sa[k]], s->v[s->sb[k]], p, R)) return 1;
    return 0;
}

/* Exact: point on segment */
static int on_segment(ipt a, ipt b, ipt p)
{
    if (cross3(a, b, p) != 0) return 0;
    i128 t = (i128)(p.x - a.x) * (b.x - a.x) + (i128)(p.y - a.y) * (b.y - a.y);
    i128 len2 = (i128)(b.x - a.x) * (b.x - a.x) + (i128)(b.y - a.y) * (b.y - a.y);
    return t >= 0 && t <= len2;
}

/* Reading (O1): a cell is solid iff its centre lies inside any loop (even-odd
 * ray crossing) or on a loop. */
static int point_solid(const oracle_solver *s, ipt p)
{
    if (!s->cfg.solid_walls) return 0;
    int inside = 0;
    for (int k = 0; k < s->nseg; k++) {
        ipt a = s->v[s->sa[k]], b = s->v[s->sb[k]];
        if (on_segment(a, b, p)) return 1;
        if ((a.y > p.y) != (b.y > p.y)) {
            /* crossing x > p.x ?  sign((p.y-a.y)(b.x-a.x) - (p.x-a.x)(b.y-a.y)) vs sign(b.y-a.y) */
            i128 num = (i128)(p.y - a.y) * (b.x - a.x) - (i128)(p.x - a.x) * (b.y - a.y);
            int right = (b.y > a.y) ? (num > 0) : (num < 0);
            if (right) inside ^= 1;
        }
    }
    return inside;
}

/* closest point on segment (double, finest-lattice units) */
static double seg_closest(const oracle_solver *s, int k, double px, double py, double *cx, double *cy)
{
    double ax = (double)s->v[s->sa[k]].x / FIX_ONE, ay = (double)s->v[s->sa[k]].y / FIX_ONE;
    double bx = (double)s->v[s->sb[k]].x / FIX_ONE, by = (double)s->v[s->sb[k]].y / FIX_ONE;
    double dx = bx - ax, dy = by - ay;
    double len2 = dx * dx + dy * dy;
    double t = len2 > 0 ? ((px - ax) * dx + (py - ay) * dy) / len2 : 0.0;
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    *cx = ax + t * dx; *cy = ay + t * dy;
    return sqrt((px - *cx) * (px - *cx) + (py - *cy) * (py - *cy));
}

static double wall_distance(const oracle_solver *s, double px, double py, int *kbest, double *cx, double *cy)
{
    double best = INFINITY;
    int kb = -1;
    double bx = 0, by = 0;
    for (int k = 0; k < s->nseg; k++) {
        double qx, qy;
        double dd = seg_closest(s, k, px, py, &qx, &qy);
        if (dd < best) { best = dd; kb = k; bx = qx; by = qy; }
    }
    if (kbest) *kbest = kb;
    if (cx) *cx = bx;
    if (cy) *cy = by;
    return best;
}

/* fraction t in (0, 1] of the first wall crossing along the link p -> p + d */
static double link_fraction(const oracle_solver *s, ipt p, ipt d)
{
    double best = 2.0;
    for (int k = 0; k < s->nseg; k++) {
        ipt a = s->v[s->sa[k]], b = s->v[s->sb[k]];
        i128 ex = b.x - a.x, ey = b.y - a.y;
        i128 den = (i128)d.x * ey - (i128)d.y * ex;               /* d x e */
        i128 apx = a.x - p.x, apy = a.y - p.y;
        i128 tn = apx * ey - apy * ex;                            /* (a-p) x e */
        i128 sn = apx * d.y - apy * d.x;                          /* (a-p) x d */
        if (den != 0) {
            int ok;
            if (den > 0) ok = tn >= 0 && tn <= den && sn >= 0 && sn <= den;
            else ok = tn <= 0 && tn >= den && sn <= 0 && sn >= den;
            if (ok) {
                double t = (double)tn / (double)den;
                if (t < best) best = t;
            }
        } else if (tn == 0) {
            /* collinear: parameters of a and b along the link */
            double dd = (double)((i128)d.x * d.x + (i128)d.y * d.y);
            double ta = (double)(apx * d.x + apy * d.y) / dd;
            double tb = (double)((i128)(b.x - p.x) * d.x + (i128)(b.y - p.y) * d.y) / dd;
            double lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
            if (hi >= 0 && lo <= 1) {
                double t = lo < 0 ? 0 : lo;
                if (t < best) best = t;
            }
        }
    }
    return best;
}

/* ===========================================================================
 * API: create / destroy
 * ========================================================================= */

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* OpenMP team size of the oracle's later parallel regions in the calling thread (n >= 1);
 * for timing it on one core and on all of them */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

const char *oracle_last_error(const oracle_solver *s) { return s ? s->err : "null handle"; }

int oracle_create(const oracle_config *cfg, oracle_solver **out)
{
    if (!cfg || !out) return -1;
    *out = NULL;
    if (cfg->levels < 1 || cfg->levels > MAXL || cfg->nx0 < 4 || cfg->ny0 < 4 || !(cfg->h0 > 0) ||
        cfg->layers < 3 || !(cfg->Re > 0) || !(cfg->Ma > 0) || !(cfg->chord > 0) || cfg->outlet < 0 ||
        cfg->outlet > 1 || (!cfg->periodic && cfg->nx0 < 8))
        return -1;
    oracle_solver *s = (oracle_solver *)calloc(1, sizeof *s);
    if (!s) return -2;
    s->cfg = *cfg;
    s->L = cfg->levels;
    s->U = cfg->Ma * sqrt(CS2);
    *out = s;
    return 0;
}

static void free_level(olevel *L)
{
    free(L->kind); free(L->solid); free(L->band); free(L->bnode); free(L->coal); free(L->cut); free(L->rec);
    free(L->f); free(L->fn); free(L->rho); free(L->ux); free(L->uy); free(L->chi); free(L->chin); free(L->d);
    memset(L, 0, sizeof *L);
}

static void free_geometry(oracle_solver *s)
{
    for (int l = 0; l < MAXL; l++) free_level(&s->lv[l]);
    free(s->loop_off); free(s->v); free(s->sa); free(s->sb); free(s->sloop); free(s->loop_ccw);
    free(s->loop_slip); free(s->rec);
    free(s->seg_b1); free(s->seg_b2); free(s->seg_w1); free(s->seg_w2);
    s->loop_off = NULL; s->v = NULL; s->sa = s->sb = s->sloop = s->loop_ccw = NULL; s->loop_slip = NULL;
    s->rec = NULL; s->seg_b1 = s->seg_b2 = NULL; s->seg_w1 = s->seg_w2 = NULL;
    s->nrec = 0; s->geometry = 0;
}

void oracle_destroy(oracle_solver *s)
{
    if (!s) return;
    free_geometry(s);
    free(s);
}

static int alloc_level(olevel *L, int i0, int j0, int nx, int ny)
{
    L->i0 = i0; L->j0 = j0; L->nx = nx; L->ny = ny;
    size_t n = (size_t)nx * ny;
    L->kind = calloc(n, 1); L->solid = calloc(n, 1); L->band = calloc(n, 1); L->bnode = calloc(n, 1);
    L->coal = calloc(n, 2); L->cut = calloc(n, 2); L->rec = malloc(n * sizeof(int));
    L->f = calloc(9 * n, 8); L->fn = calloc(9 * n, 8);
    L->rho = calloc(n, 8); L->ux = calloc(n, 8); L->uy = calloc(n, 8);
    L->chi = calloc(n, 8); L->chin = calloc(n, 8); L->d = calloc(n, 8);
    if (!L->kind || !L->solid || !L->band || !L->bnode || !L->coal || !L->cut || !L->rec || !L->f ||
        !L->fn || !L->rho || !L->ux || !L->uy || !L->chi || !L->chin || !L->d)
        return -1;
    for (size_t k = 0; k < n; k++) L->rec[k] = -1;
    return 0;
}

/* ===========================================================================
 * Grid build (reading O1 of the pre-processor, Sec 2.1 / Sec 2.3)
 * ========================================================================= */

static void init_state(oracle_solver *s);

/* the wall polylines: vertices snapped to the fixed-point grid, segments of non-zero length */
static int setup_walls(oracle_solver *s, const double *xy, const int *loop_off, int nloops)
{
    const oracle_config *c = &s->cfg;
    const int L = s->L;
    double hfin = c->h0 / (double)(1LL << (L - 1));
    /* vertices snapped to the fixed-point grid (unit hfin / 4096) */
    s->nloops = nloops;
    s->loop_off = malloc((nloops + 1) * sizeof(int));
    s->loop_ccw = malloc((nloops > 0 ? nloops : 1) * sizeof(int));
    s->loop_slip = calloc(2 * (nloops > 0 ? nloops : 1), sizeof(double));
    int nv = nloops > 0 ? loop_off[nloops] : 0;
    s->nv = nv;
    s->v = malloc((nv > 0 ? nv : 1) * sizeof(ipt));
    s->sa = malloc((nv > 0 ? nv : 1) * sizeof(int));
    s->sb = malloc((nv > 0 ? nv : 1) * sizeof(int));
    s->sloop = malloc((nv > 0 ? nv : 1) * sizeof(int));
    for (int k = 0; k <= nloops; k++) s->loop_off[k] = loop_off[k];
    for (int k = 0; k < nv; k++) {
        s->v[k].x = llround((xy[2 * k] - c->x0) / hfin * (double)FIX_ONE);
        s->v[k].y = llround((xy[2 * k + 1] - c->y0) / hfin * (double)FIX_ONE);
    }
    s->nseg = 0;
    for (int lp = 0; lp < nloops; lp++) {
        int a = loop_off[lp], b = loop_off[lp + 1];
        if (b - a < 3) return fail(s, -5, "loop with fewer than 3 vertices");
        i128 area2 = 0;
        int nl = 0;
        for (int k = a; k < b; k++) {
            int k2 = (k + 1 < b) ? k + 1 : a;
            /* reading: vertices that coincide on the fixed-point grid are merged; a
               zero-length segment has no normal and adds nothing to eq 30 */
            if (s->v[k].x == s->v[k2].x && s->v[k].y == s->v[k2].y) continue;
            s->sa[s->nseg] = k; s->sb[s->nseg] = k2; s->sloop[s->nseg] = lp; s->nseg++; nl++;
            area2 += (i128)s->v[k].x * s->v[k2].y - (i128)s->v[k2].x * s->v[k].y;
            long long ex = s->v[k2].x - s->v[k].x, ey = s->v[k2].y - s->v[k].y;
            if (llabs(ex) > (1LL << 30) || llabs(ey) > (1LL << 30))
                return fail(s, -5, "wall segment longer than 2^18 finest cells");
        }
        if (area2 == 0 || nl < 3) return fail(s, -5, "degenerate loop");
        s->loop_ccw[lp] = area2 > 0;
    }
    return 0;
}

int oracle_set_geometry(oracle_solver *s, const double *xy, const int *loop_off, int nloops)
{
    if (!s || (nloops > 0 && (!xy || !loop_off)) || nloops < 0) return -1;
    free_geometry(s);
    const oracle_config *c = &s->cfg;
    const int L = s->L;
    int rc = setup_walls(s, xy, loop_off, nloops);
    if (rc) return rc;
    /* level 0: every cell of the box is present and active */
    olevel *lv = s->lv;
    for (int l = 0; l < L; l++) lv[l].scale = 1LL << (L - 1 - l);
    if (alloc_level(&lv[0], 0, 0, c->nx0, c->ny0)) return fail(s, -2, "out of memory");
    memset(lv[0].kind, K_ACTIVE, (size_t)c->nx0 * c->ny0);
    /* refinement radii R_l (fixed units): R_{L-1} = layers h_{L-1}, R_l = R_{l+1} + layers h_l */
    long long R[MAXL];
    R[L - 1] = (long long)c->layers * FIX_ONE;
    for (int l = L - 2; l >= 1; l--) R[l] = R[l + 1] + (long long)c->layers * lv[l].scale * FIX_ONE;
    for (int l = 1; l < L; l++) {
        olevel *P = &lv[l - 1];
        /* parents within R_l of the wall are covered (only active cells refine) */
        for (int j = P->j0; j < P->j0 + P->ny; j++)
            for (int i = P->i0; i < P->i0 + P->nx; i++) {
                long k = cidx(P, i, j);
                if (P->kind[k] == K_ACTIVE && near_wall(s, centre_fix(P, i, j), R[l])) P->kind[k] = K_COVERED;
            }
        /* nesting: every covered cell keeps all 8 neighbours on its own level (active or covered),
           and level-0 refinement stays two cells clear of the box edge */
        int bi0 = 1 << 30, bj0 = 1 << 30, bi1 = -(1 << 30), bj1 = -(1 << 30);
        for (int j = P->j0; j < P->j0 + P->ny; j++)
            for (int i = P->i0; i < P->i0 + P->nx; i++) {
                long k = cidx(P, i, j);
                if (P->kind[k] != K_COVERED) continue;
                if (l == 1 && (i < 2 || j < 2 || i >= c->nx0 - 2 || j >= c->ny0 - 2))
                    return fail(s, -5, "refinement reaches the level-0 box edge");
                for (int q = 1; q < 9; q++) {
                    long kn = cidx(P, i + CX[q], j + CY[q]);
                    if (kn < 0 || (P->kind[kn] != K_ACTIVE && P->kind[kn] != K_COVERED))
                        return fail(s, -5, "refinement band violates 2:1 nesting (increase layers)");
                }
                if (i - 1 < bi0) bi0 = i - 1;
                if (j - 1 < bj0) bj0 = j - 1;
                if (i + 1 > bi1) bi1 = i + 1;
                if (j + 1 > bj1) bj1 = j + 1;
            }
        if (bi1 < bi0) return fail(s, -5, "level has no cells (wall far from the box?)");
        /* band: active cells with a covered D2Q9 neighbour */
        for (int j = P->j0; j < P->j0 + P->ny; j++)
            for (int i = P->i0; i < P->i0 + P->nx; i++) {
                long k = cidx(P, i, j);
                if (P->kind[k] != K_ACTIVE) continue;
                for (int q = 1; q < 9; q++) {
                    long kn = cidx(P, i + CX[q], j + CY[q]);
                    if (kn >= 0 && P->kind[kn] == K_COVERED) { P->band[k] = 1; break; }
                }
            }
        /* level-l array box: children of the parent box [bi0, bi1] x [bj0, bj1], plus a margin of one */
        olevel *F = &lv[l];
        if (alloc_level(F, 2 * bi0 - 1, 2 * bj0 - 1, 2 * (bi1 - bi0 + 1) + 2, 2 * (bj1 - bj0 + 1) + 2))
            return fail(s, -2, "out of memory");
        for (int j = bj0; j <= bj1; j++)
            for (int i = bi0; i <= bi1; i++) {
                long k = cidx(P, i, j);
                int kd = (P->kind[k] == K_COVERED) ? K_ACTIVE : (P->band[k] ? K_GHOST : K_ABSENT);
                if (kd == K_ABSENT) continue;
                for (int b = 0; b < 2; b++)
                    for (int a = 0; a < 2; a++) F->kind[cidx(F, 2 * i + a, 2 * j + b)] = (unsigned char)kd;
            }
    }
    /* coalescence flags (reading O5): coarse (c, j) takes the average of its ghost
       children iff one of c - c_j, c - (c_jx, 0), c - (0, c_jy) is covered */
    for (int l = 0; l < L - 1; l++) {
        olevel *P = &lv[l];
        for (int j = P->j0; j < P->j0 + P->ny; j++)
            for (int i = P->i0; i < P->i0 + P->nx; i++) {
                long k = cidx(P, i, j);
                if (!P->band[k]) continue;
                unsigned short m = 0;
                for (int q = 1; q < 9; q++) {
                    long s0 = cidx(P, i - CX[q], j - CY[q]);
                    long s1 = cidx(P, i - CX[q], j);
                    long s2 = cidx(P, i, j - CY[q]);
                    int cov = (s0 >= 0 && P->kind[s0] == K_COVERED) || (s1 >= 0 && P->kind[s1] == K_COVERED) ||
                              (s2 >= 0 && P->kind[s2] == K_COVERED);
                    if (cov) m |= (unsigned short)(1u << q);
                }
                P->coal[k] = m;
            }
    }
    /* solid flags of every present cell */
    for (int l = 0; l < L; l++) {
        olevel *P = &lv[l];
#pragma omp parallel for schedule(dynamic, 4)
        for (int j = P->j0; j < P->j0 + P->ny; j++)
            for (int i = P->i0; i < P->i0 + P->nx; i++) {
                long k = cidx(P, i, j);
                if (P->kind[k] != K_ABSENT) P->solid[k] = (unsigned char)point_solid(s, centre_fix(P, i, j));
            }
    }
    /* walls only touch the finest level: a fluid cell with a solid neighbour elsewhere is an error */
    for (int l = 0; l < L; l++) {
        olevel *P = &lv[l];
        for (int j = P->j0; j < P->j0 + P->ny; j++)
            for (int i = P->i0; i < P->i0 + P->nx; i++) {
                long k = cidx(P, i, j);
                if (P->kind[k] == K_ABSENT || P->solid[k] || P->kind[k] == K_COVERED) continue;
                unsigned short cm = 0;
                for (int q = 1; q < 9; q++) {
                    long long si = i - CX[q], sj = j - CY[q];
                    if (l == 0 && c->periodic) { si = (si + c->nx0) % c->nx0; sj = (sj + c->ny0) % c->ny0; }
                    long kn = cidx(P, si, sj);
                    if (kn >= 0 && P->kind[kn] != K_ABSENT && P->solid[kn]) cm |= (unsigned short)(1u << q);
                }
                if (!cm) continue;
                if (l != L - 1 || P->kind[k] != K_ACTIVE)
                    return fail(s, -5, "wall reaches a cell that is not on the finest active level");
                P->cut[k] = cm;
                P->bnode[k] = 1;
            }
    }
    /* wall distance (finest lattice units -> level units) for active fluid cells */
    for (int l = 0; l < L; l++) {
        olevel *P = &lv[l];
#pragma omp parallel for schedule(dynamic, 4)
        for (int j = P->j0; j < P->j0 + P->ny; j++)
            for (int i = P->i0; i < P->i0 + P->nx; i++) {
                long k = cidx(P, i, j);
                if (P->kind[k] != K_ACTIVE || P->solid[k]) continue;
                double dd = D_CAP;
                if (c->solid_walls && s->nseg > 0) {
                    double px = (i + 0.5) * P->scale, py = (j + 0.5) * P->scale;
                    dd = wall_distance(s, px, py, NULL, NULL, NULL) / (double)P->scale;
                    if (dd > D_CAP) dd = D_CAP;
                }
                P->d[k] = dd;
            }
    }
    /* wall records (Sec 2.3, Fig 2): one per boundary node B, in (j, i) order */
    olevel *Fn = &lv[L - 1];
    int nb = 0;
    for (long k = 0; k < (long)Fn->nx * Fn->ny; k++) nb += Fn->bnode[k];
    s->nrec = nb;
    s->rec = calloc(nb > 0 ? nb : 1, sizeof(orec));
    int r = 0;
    for (int j = Fn->j0; j < Fn->j0 + Fn->ny; j++)
        for (int i = Fn->i0; i < Fn->i0 + Fn->nx; i++) {
            long k = cidx(Fn, i, j);
            if (!Fn->bnode[k]) continue;
            orec *R0 = &s->rec[r];
            Fn->rec[k] = r;
            R0->i = i; R0->j = j;
            double bx = i + 0.5, by = j + 0.5, qx, qy;
            int kb;
            double dwb = wall_distance(s, bx, by, &kb, &qx, &qy);
            R0->seg = kb; R0->loop = s->sloop[kb];
            R0->iw[0] = qx; R0->iw[1] = qy; R0->dwb = dwb;
            R0->n[0] = (bx - qx) / dwb; R0->n[1] = (by - qy) / dwb;
            R0->r[0] = qx + c->d_wr * R0->n[0];
            R0->r[1] = qy + c->d_wr * R0->n[1];
            /* cut-link fractions q_j along B -> B - c_j (Sec 2.3, eq 27) */
            ipt pb = centre_fix(Fn, i, j);
            for (int q = 1; q < 9; q++) {
                if (!(Fn->cut[k] >> q & 1)) continue;
                ipt dvec = {-CX[q] * FIX_ONE, -CY[q] * FIX_ONE};
                double t = link_fraction(s, pb, dvec);
                if (t > 1.0) return fail(s, -5, "cut link without a wall crossing");
                R0->q[q] = t;
            }
            /* reference-point stencil: the 4x4 finest cells around R, minus solid and B nodes */
            int ic = (int)floor(R0->r[0] - 0.5), jc = (int)floor(R0->r[1] - 0.5);
            R0->ns = 0;
            for (int b = -1; b <= 2; b++)
                for (int a = -1; a <= 2; a++) {
                    long kk = cidx(Fn, ic + a, jc + b);
                    if (c->wall_model <= 1 && (kk < 0 || Fn->kind[kk] != K_ACTIVE))
                        return fail(s, -5, "reference point stencil leaves the finest active level");
                    if (kk < 0 || Fn->kind[kk] != K_ACTIVE || Fn->solid[kk] || Fn->bnode[kk]) continue;
                    R0->si[R0->ns] = ic + a; R0->sj[R0->ns] = jc + b; R0->ns++;
                }
            if (c->wall_model <= 1 && R0->ns == 0) return fail(s, -5, "empty reference stencil");
            r++;
        }
    /* surface elements -> two nearest boundary nodes (Sec 3.1.3) */
    s->seg_b1 = malloc((s->nseg > 0 ? s->nseg : 1) * sizeof(int));
    s->seg_b2 = malloc((s->nseg > 0 ? s->nseg : 1) * sizeof(int));
    s->seg_w1 = malloc((s->nseg > 0 ? s->nseg : 1) * sizeof(double));
    s->seg_w2 = malloc((s->nseg > 0 ? s->nseg : 1) * sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < s->nseg; k++) {
        double mx = 0.5 * (double)(s->v[s->sa[k]].x + s->v[s->sb[k]].x) / FIX_ONE;
        double my = 0.5 * (double)(s->v[s->sa[k]].y + s->v[s->sb[k]].y) / FIX_ONE;
        int b1 = -1, b2 = -1;
        double d1 = INFINITY, d2 = INFINITY;
        for (int q = 0; q < s->nrec; q++) {
            double dx = s->rec[q].i + 0.5 - mx, dy = s->rec[q].j + 0.5 - my;
            double dd = dx * dx + dy * dy;
            if (dd < d1) { d2 = d1; b2 = b1; d1 = dd; b1 = q; }
            else if (dd < d2) { d2 = dd; b2 = q; }
        }
        s->seg_b1[k] = b1; s->seg_b2[k] = b2;
        s->seg_w1[k] = b1 >= 0 ? 1.0 / (d1 > 1e-300 ? d1 : 1e-300) : 0.0;
        s->seg_w2[k] = b2 >= 0 ? 1.0 / (d2 > 1e-300 ? d2 : 1e-300) : 0.0;
    }
    /* lattice viscosity per level (acoustic scaling, Sec 2.1): nu_l = U (c / h_l) / Re */
    for (int l = 0; l < L; l++) lv[l].nu = s->U * (c->chord / c->h0) * (double)(1LL << l) / c->Re;
    s->geometry = 1;
    s->step = 0;
    s->have_cl = 0;
    init_state(s);
    return 0;
}

int oracle_set_wall_slip(oracle_solver *s, const double *uw, int n)
{
    if (!s || !s->geometry || n != s->nloops || !uw) return -1;
    for (int k = 0; k < 2 * n; k++) s->loop_slip[k] = uw[k];
    return 0;
}

/* ===========================================================================
 * Interface synchronisation helpers (Sec 2.1, Rohde transfers; reading O5/O6)
 * ========================================================================= */

/* covered cells: rho, chi = mean of fluid children; u mass-weighted */
static void restrict_level(oracle_solver *s, int l)
{
    olevel *P = &s->lv[l], *F = &s->lv[l + 1];
#pragma omp parallel for schedule(static)
    for (int j = P->j0; j < P->j0 + P->ny; j++)
        for (int i = P->i0; i < P->i0 + P->nx; i++) {
            long k = cidx(P, i, j);
            if (P->kind[k] != K_COVERED) continue;
            double sr = 0, sx = 0, sy = 0, sc = 0;
            int n = 0;
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) {
                    long kc = cidx(F, 2 * i + a, 2 * j + b);
                    if (F->solid[kc]) continue;
                    sr += F->rho[kc]; sx += F->rho[kc] * F->ux[kc]; sy += F->rho[kc] * F->uy[kc];
                    sc += F->chi[kc]; n++;
                }
            if (n == 0) continue;
            P->rho[k] = sr / n; P->ux[k] = sx / sr; P->uy[k] = sy / sr; P->chi[k] = sc / n;
        }
}

/* ghost children of band cells: linear LSQ reconstruction about the parent
 * (Sec 2.2 "interpolated using the LSQ method"; reading: gradient-only LSQ
 * anchored at the parent value) */
static void prolong_level(oracle_solver *s, int l)
{
    olevel *P = &s->lv[l], *F = &s->lv[l + 1];
#pragma omp parallel for schedule(static)
    for (int j = P->j0; j < P->j0 + P->ny; j++)
        for (int i = P->i0; i < P->i0 + P->nx; i++) {
            long k = cidx(P, i, j);
            if (!P->band[k] || P->solid[k]) continue;
            double dx[8], dy[8], dc[8], du[8], dv[8];
            int n = 0;
            for (int q = 1; q < 9; q++) {
                long kn = cidx(P, i + CX[q], j + CY[q]);
                if (kn < 0 || P->kind[kn] == K_ABSENT || P->solid[kn]) continue;
                dx[n] = CX[q]; dy[n] = CY[q];
                dc[n] = P->chi[kn] - P->chi[k];
                du[n] = P->ux[kn] - P->ux[k];
                dv[n] = P->uy[kn] - P->uy[k];
                n++;
            }
            double gcx, gcy, gux, guy, gvx, gvy;
            lsq_gradient(n, dx, dy, dc, &gcx, &gcy);
            lsq_gradient(n, dx, dy, du, &gux, &guy);
            lsq_gradient(n, dx, dy, dv, &gvx, &gvy);
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) {
                    long kc = cidx(F, 2 * i + a, 2 * j + b);
                    double ox = 0.5 * (a - 0.5), oy = 0.5 * (b - 0.5);
                    F->chi[kc] = P->chi[k] + gcx * ox + gcy * oy;
                    F->ux[kc] = P->ux[k] + gux * ox + guy * oy;
                    F->uy[kc] = P->uy[k] + gvx * ox + gvy * oy;
                    F->rho[kc] = P->rho[k];
                }
        }
}

/* explosion: post-collision populations of band cells copied to their 4 ghost
 * children in the fine level's current lattice (Rohde, Sec 2.1) */
static void explode_level(oracle_solver *s, int l, const double *fsrc)
{
    olevel *P = &s->lv[l], *F = &s->lv[l + 1];
#pragma omp parallel for schedule(static)
    for (int j = P->j0; j < P->j0 + P->ny; j++)
        for (int i = P->i0; i < P->i0 + P->nx; i++) {
            long k = cidx(P, i, j);
            if (!P->band[k] || P->solid[k]) continue;
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) {
                    long kc = cidx(F, 2 * i + a, 2 * j + b);
                    for (int q = 0; q < 9; q++) F->f[9 * kc + q] = fsrc[9 * k + q];
                }
        }
}

static void init_state(oracle_solver *s)
{
    double fe[9];
    oracle_feq(1.0, s->U, 0.0, fe);
    for (int l = 0; l < s->L; l++) {
        olevel *P = &s->lv[l];
        long n = (long)P->nx * P->ny;
        for (long k = 0; k < n; k++) {
            if (P->kind[k] == K_ABSENT) continue;
            for (int q = 0; q < 9; q++) P->f[9 * k + q] = P->fn[9 * k + q] = fe[q];
            P->rho[k] = 1.0; P->ux[k] = s->U; P->uy[k] = 0.0;
            P->chi[k] = P->chin[k] = s->cfg.chi_inf;
        }
    }
}

/* ===========================================================================
 * Wall function per boundary node (Sec 2.3 steps 1-5, eq 28)
 * ========================================================================= */

/* Wall state of one boundary node (Sec 2.3 steps 1-5, eq 28; reading O7-O9): from the
 * fields rho, u at the ns stencil cells whose centres lie at (dx, dy) from the reference
 * point R, the unit normal n (wall to fluid), the wall distance dwb of B and the level's
 * viscosity nu.  out = rho_W, u_W (2), u_tau, chi_B, t (2), |u_Rt|.  slip: the prescribed
 * wall velocity (wall model 2). */
void oracle_wall_point(const oracle_config *c, double nu, int ns, const double *dx, const double *dy,
                       const double *rho, const double *ux, const double *uy, const double *n, double dwb,
                       const double *slip, double *out)
{
    /* step 1: rho_R by inverse-distance weighting, u_R by unweighted linear LSQ */
    double sw = 0, swr = 0, swu = 0, swv = 0;
    double A[9] = {0}, bu[3] = {0}, bv[3] = {0};
    for (int m = 0; m < ns; m++) {
        double d2 = dx[m] * dx[m] + dy[m] * dy[m];
        double w = 1.0 / (d2 > 1e-20 ? d2 : 1e-20);
        sw += w; swr += w * rho[m]; swu += w * ux[m]; swv += w * uy[m];
        double phi[3] = {1.0, dx[m], dy[m]};
        for (int a = 0; a < 3; a++) {
            for (int b = 0; b < 3; b++) A[3 * a + b] += phi[a] * phi[b];
            bu[a] += phi[a] * ux[m];
            bv[a] += phi[a] * uy[m];
        }
    }
    double rhoR = ns > 0 ? swr / sw : 1.0;
    double uR = ns > 0 ? swu / sw : 0.0, vR = ns > 0 ? swv / sw : 0.0;
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (ns >= 3 && det > 1e-9 * A[0] * A[4] * A[8]) {
        double A2[9];
        memcpy(A2, A, sizeof A2);
        solve_dense(3, A, bu);
        solve_dense(3, A2, bv);
        uR = bu[0]; vR = bv[0];
    }
    /* step 2: tangential component */
    double un = uR * n[0] + vR * n[1];
    double utx = uR - un * n[0], uty = vR - un * n[1];
    double ut = sqrt(utx * utx + uty * uty);
    double t[2];
    if (ut > 0) { t[0] = utx / ut; t[1] = uty / ut; }
    else { t[0] = -n[1]; t[1] = n[0]; }
    double utau = 0, uW[2] = {0, 0}, chiB = 0;
    if (c->wall_model == 0) {
        /* step 3: friction velocity from eq 22 at R */
        utau = oracle_wf_utau(ut, c->d_wr, nu);
        /* step 4: u_V = u_tau f_SA(y+_V) */
        double ypv = utau * c->d_wv / nu;
        double uV = utau * oracle_wf_uplus(ypv);
        /* step 5 / eq 28 with (nu_t)_V = nu kappa y+_V; direction: reading t = u_Rt/|u_Rt| */
        double uWm = uV - utau * utau * c->d_wv / (nu * (1.0 + SA_KAPPA * ypv));
        uW[0] = uWm * t[0];
        uW[1] = uWm * t[1];
        /* SA Dirichlet at B: nu_t~_B = nu kappa d+_WB (Sec 2.2) */
        chiB = SA_KAPPA * utau * dwb / nu;
    } else if (c->wall_model == 1) {
        /* Nishimura's slip adapted to RANS (Sec 3.1.5, eq 31).  Readings: u_tau from eq 22 at
           R (step 3 kept: eq 31 needs it; Sec 2.3 names the VN steps 4-5 as the ones
           Nishimura's approach lacks, so Sec 3.1.5's 'steps 3 and 4' are read as those);
           (nu_t)_R is the eddy viscosity of the SA log layer at R, nu kappa y+_R (eq 20; the
           mixing-length value Nishimura et al. use at R, and the value the VN method takes at
           V); slip along t = u_Rt/|u_Rt|; the SA Dirichlet value as in the VN method. */
        utau = oracle_wf_utau(ut, c->d_wr, nu);
        double ypr = utau * c->d_wr / nu;
        double uWm = ut - utau * utau * c->d_wr / (nu * (1.0 + SA_KAPPA * ypr));
        uW[0] = uWm * t[0];
        uW[1] = uWm * t[1];
        chiB = SA_KAPPA * utau * dwb / nu;
    } else if (c->wall_model == 2) {
        uW[0] = slip[0];
        uW[1] = slip[1];
    }
    out[0] = rhoR;                                          /* step 6: rho_W ~ rho_R */
    out[1] = uW[0]; out[2] = uW[1]; out[3] = utau; out[4] = chiB;
    out[5] = t[0]; out[6] = t[1]; out[7] = ut;
}

static void wall_function(oracle_solver *s)
{
    const oracle_config *c = &s->cfg;
    olevel *F = &s->lv[s->L - 1];
    double nu = F->nu;
#pragma omp parallel for schedule(dynamic, 16)
    for (int r = 0; r < s->nrec; r++) {
        orec *R0 = &s->rec[r];
        double dx[16], dy[16], rho[16], ux[16], uy[16], out[8];
        for (int m = 0; m < R0->ns; m++) {
            long k = cidx(F, R0->si[m], R0->sj[m]);
            dx[m] = R0->si[m] + 0.5 - R0->r[0];
            dy[m] = R0->sj[m] + 0.5 - R0->r[1];
            rho[m] = F->rho[k]; ux[m] = F->ux[k]; uy[m] = F->uy[k];
        }
        oracle_wall_point(c, nu, R0->ns, dx, dy, rho, ux, uy, R0->n, R0->dwb, &s->loop_slip[2 * R0->loop], out);
        R0->rhoW = out[0];
        R0->uW[0] = out[1]; R0->uW[1] = out[2];
        R0->utau = out[3];
        R0->chiB = out[4];
        R0->t[0] = out[5]; R0->t[1] = out[6];
        R0->ut = out[7];
    }
}

/* ===========================================================================
 * SA-neg update of one level (Sec 2.2) + ghost reconstruction for level l+1
 * ========================================================================= */

static void sa_level(oracle_solver *s, int l)
{
    const oracle_config *c = &s->cfg;
    olevel *P = &s->lv[l];
    const int L = s->L;
    if (l < L - 1) prolong_level(s, l);       /* ghosts of l+1 from the level-l fields at t */
    int edge = (l == 0 && !c->periodic);
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = P->j0; j < P->j0 + P->ny; j++)
        for (int i = P->i0; i < P->i0 + P->nx; i++) {
            long k = cidx(P, i, j);
            if (P->kind[k] != K_ACTIVE || P->solid[k]) continue;
            if (P->bnode[k]) { P->chin[k] = s->rec[P->rec[k]].chiB; continue; }
            if (edge && (i == 0 || i == c->nx0 - 1)) continue;
            double ch[9], u[9], v[9];
            for (int q = 0; q < 9; q++) {
                long long ii = i + CX[q], jj = j + CY[q];
                double sgn = 1.0;
                if (l == 0 && c->periodic) { ii = (ii + c->nx0) % c->nx0; jj = (jj + c->ny0) % c->ny0; }
                if (edge && (jj < 0 || jj >= c->ny0)) { jj = jj < 0 ? 0 : c->ny0 - 1; sgn = -1.0; } /* symmetry plane */
                long kn = cidx(P, ii, jj);
                if (kn < 0 || P->kind[kn] == K_ABSENT) { kn = k; sgn = 1.0; }   /* never taken on a valid grid */
                ch[q] = P->chi[kn]; u[q] = P->ux[kn]; v[q] = sgn * P->uy[kn];
            }
            P->chin[k] = oracle_sa_update_point(ch, u, v, fmax(P->d[k], SA_D_MIN), P->nu, c->sa_convection);
        }
    if (edge) {
        for (int j = 0; j < c->ny0; j++) {
            P->chin[cidx(P, 0, j)] = c->chi_inf;                               /* inlet chi = 3 */
            P->chin[cidx(P, c->nx0 - 1, j)] = P->chin[cidx(P, c->nx0 - 2, j)]; /* outlet: first-order extrapolation */
        }
    }
    long n = (long)P->nx * P->ny;
    for (long k = 0; k < n; k++)
        if (P->kind[k] == K_ACTIVE && !P->solid[k]) P->chi[k] = P->chin[k];
}

/* ===========================================================================
 * Stream + collide of one level (eq 1), with the Rohde transfers, Yu's
 * interpolated slip bounce-back and the domain boundary conditions.
 * State convention: the lattice holds post-collision populations f*.
 * ========================================================================= */

/* post-stream population of level-0 cell (i, j) from the current lattice, for a
 * direction whose source lies inside the box in x: in-box pull, or the
 * half-way specular reflection of a symmetry plane (Sec 3.1.1, reading O4) */
static int pull0(const oracle_solver *s, const olevel *P, int i, int j, int q, double *out)
{
    const oracle_config *c = &s->cfg;
    int si = i - CX[q], sj = j - CY[q];
    if (si < 0 || si >= c->nx0) return 0;
    if (sj >= 0 && sj < c->ny0) { *out = P->f[9 * cidx(P, si, sj) + q]; return 1; }
    /* population q left cell (si, j) towards the plane with c_y flipped and came back */
    int qm = -1;
    for (int m = 1; m < 9; m++) if (CX[m] == CX[q] && CY[m] == -CY[q]) qm = m;
    *out = P->f[9 * cidx(P, si, j) + qm];
    return 1;
}

/* Yu's interpolated bounce-back with the wall velocity (eq 27, reading O10) for the pulled
 * direction q of a boundary node B whose upstream B - c_q is solid: from the post-collision
 * f*_qo of the next fluid node B + c_q, f*_qo(B) and f*_q(B) (qo = opposite of q), the wall
 * fraction qf of the cut link and rho_W, u_W of B's wall state; the half-way form (eq 24)
 * where B + c_q is not an active fluid cell. */
double oracle_yu_link(int q, double qf, double rhoW, double uWx, double uWy, double f_qo_next, double f_qo_B,
                      double f_q_B, int next_fluid)
{
    double cu = CX[q] * uWx + CY[q] * uWy;
    double mom = 2.0 * WQ[q] * rhoW * cu / CS2;
    if (next_fluid) {
        double fw = (1.0 - qf) * f_qo_next + qf * f_qo_B + mom;
        return fw / (1.0 + qf) + qf / (1.0 + qf) * f_q_B;
    }
    return f_qo_B + mom;                                   /* half-way fallback, eq 24 */
}

static void stream_collide_level(oracle_solver *s, int l)
{
    const oracle_config *c = &s->cfg;
    olevel *P = &s->lv[l];
    olevel *F = (l < s->L - 1) ? &s->lv[l + 1] : NULL;
    const int edge = (l == 0 && !c->periodic);
    /* 1: pull (stream) for active fluid cells and relay for ghosts */
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = P->j0; j < P->j0 + P->ny; j++)
        for (int i = P->i0; i < P->i0 + P->nx; i++) {
            long k = cidx(P, i, j);
            int kd = P->kind[k];
            if (kd == K_ABSENT || kd == K_COVERED || P->solid[k]) continue;
            double *out = &P->fn[9 * k];
            const double *own = &P->f[9 * k];
            if (kd == K_GHOST) {
                /* ghosts are streamed, never collided */
                for (int q = 0; q < 9; q++) {
                    long ks = cidx(P, i - CX[q], j - CY[q]);
                    out[q] = (ks >= 0 && (P->kind[ks] == K_ACTIVE || P->kind[ks] == K_GHOST) && !P->solid[ks])
                                 ? P->f[9 * ks + q] : own[q];
                }
                continue;
            }
            out[0] = own[0];
            for (int q = 1; q < 9; q++) {
                if (P->coal[k] >> q & 1) {
                    /* coalescence: mean of the 4 ghost children after the two fine sub-steps */
                    double sum = 0;
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++) sum += F->f[9 * cidx(F, 2 * i + a, 2 * j + b) + q];
                    out[q] = 0.25 * sum;
                    continue;
                }
                if (P->cut[k] >> q & 1) {
                    /* Yu interpolated bounce-back with slip velocity (eqs 24, 27; reading O10) */
                    const orec *R0 = &s->rec[P->rec[k]];
                    int qo = OPPD[q];
                    long long fi = i + CX[q], fj = j + CY[q];
                    if (l == 0 && c->periodic) { fi = (fi + c->nx0) % c->nx0; fj = (fj + c->ny0) % c->ny0; }
                    long kf = cidx(P, fi, fj);
                    const int next_fluid = kf >= 0 && P->kind[kf] == K_ACTIVE && !P->solid[kf];
                    out[q] = oracle_yu_link(q, R0->q[q], R0->rhoW, R0->uW[0], R0->uW[1], next_fluid ? P->f[9 * kf + qo] : 0.0,
                                            own[qo], own[q], next_fluid);
                    continue;
                }
                long long si = i - CX[q], sj = j - CY[q];
                if (l == 0 && c->periodic) { si = (si + c->nx0) % c->nx0; sj = (sj + c->ny0) % c->ny0; }
                if (edge && (si < 0 || sj < 0 || si >= c->nx0 || sj >= c->ny0)) {
                    out[q] = NAN;                                      /* filled by the domain BCs below */
                    continue;
                }
                long ks = cidx(P, si, sj);
                out[q] = (ks >= 0 && P->kind[ks] != K_ABSENT) ? P->f[9 * ks + q] : own[q];   /* guard: never taken on a valid grid */
            }
        }
    /* 2: domain boundary conditions on level 0 (Sec 3.1.1; reading O4) */
    if (edge) {
        for (int j = 0; j < c->ny0; j++)
            for (int i = 0; i < c->nx0; i++) {
                if (i > 0 && i < c->nx0 - 1 && j > 0 && j < c->ny0 - 1) continue;
                long k = cidx(P, i, j);
                if (P->solid[k]) continue;
                double *out = &P->fn[9 * k];
                /* symmetry planes top/bottom for sources inside the box in x */
                for (int q = 1; q < 9; q++) {
                    int si = i - CX[q], sj = j - CY[q];
                    if ((sj < 0 || sj >= c->ny0) && si >= 0 && si < c->nx0) pull0(s, P, i, j, q, &out[q]);
                }
                if (i == 0) {
                    /* Zou-He velocity inlet u = (U, 0): unknowns 1, 5, 7 */
                    double U = s->U;
                    double rho = (out[0] + out[3] + out[4] + 2.0 * (out[2] + out[6] + out[8])) / (1.0 - U);
                    out[1] = out[2] + (2.0 / 3.0) * rho * U;
                    out[5] = out[6] - 0.5 * (out[3] - out[4]) + rho * U / 6.0;
                    out[7] = out[8] + 0.5 * (out[3] - out[4]) + rho * U / 6.0;
                }
            }
        /* outlet, on the post-stream values of the three populations entering from outside
         * (q = 2, 6, 8): Yu's linear extrapolation f_q(N-1) = 2 f_q(N-2) - f_q(N-3) (outlet 0,
         * the form Sec 3.1.1 names), or the zero-gradient copy f_q(N-1) = f_q(N-2) (outlet 1).
         * The linear form amplifies the wake's vortices as they cross the last columns. */
        const int qs[3] = {2, 6, 8};
        for (int j = 0; j < c->ny0; j++) {
            long k = cidx(P, c->nx0 - 1, j);
            if (P->solid[k]) continue;
            const long k2 = cidx(P, c->nx0 - 2, j), k3 = cidx(P, c->nx0 - 3, j);
            for (int m = 0; m < 3; m++) {
                int q = qs[m];
                P->fn[9 * k + q] = c->outlet == 0 ? 2.0 * P->fn[9 * k2 + q] - P->fn[9 * k3 + q] : P->fn[9 * k2 + q];
            }
        }
    }
    /* 3: macroscopic fields and central-moment collision with nu + nu_t (eqs 3, 7, 9, 11) */
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = P->j0; j < P->j0 + P->ny; j++)
        for (int i = P->i0; i < P->i0 + P->nx; i++) {
            long k = cidx(P, i, j);
            if (P->kind[k] != K_ACTIVE || P->solid[k]) continue;
            double *fk = &P->fn[9 * k];
            double rho = 0, jx = 0, jy = 0;
            for (int q = 0; q < 9; q++) { rho += fk[q]; jx += CX[q] * fk[q]; jy += CY[q] * fk[q]; }
            P->rho[k] = rho; P->ux[k] = jx / rho; P->uy[k] = jy / rho;
            double nut = 0.0;
            if (c->turbulence) {
                double chi = P->chi[k];
                nut = (chi > 0 ? chi : 0.0) * P->nu * sa_fv1(chi);
            }
            double om = 1.0 / ((P->nu + nut) / CS2 + 0.5);
            double post[9];
            oracle_collide(fk, om, 1.0, post);
            for (int q = 0; q < 9; q++) fk[q] = post[q];
        }
    /* 4: explosion into the fine ghosts; 5: restriction of covered cells */
    if (F) {
        explode_level(s, l, P->fn);
        restrict_level(s, l);
    }
    double *t = P->f; P->f = P->fn; P->fn = t;
}

/* level recursion (Sec 2.1: fine levels take two sub-steps per parent step) */
static void advance(oracle_solver *s, int l)
{
    if (l == s->L - 1 && s->nrec > 0) wall_function(s);
    if (s->cfg.turbulence) sa_level(s, l);
    if (l < s->L - 1) { advance(s, l + 1); advance(s, l + 1); }
    stream_collide_level(s, l);
}

int oracle_step(oracle_solver *s, int n)
{
    if (!s) return -1;
    if (!s->geometry) return fail(s, -4, "no geometry");
    if (n < 0) return fail(s, -1, "negative step count");
    for (int it = 0; it < n; it++) {
        advance(s, 0);
        s->step++;
    }
    for (int l = 0; l < s->L; l++) {
        olevel *P = &s->lv[l];
        long m = (long)P->nx * P->ny;
        for (long k = 0; k < m; k++)
            if (P->kind[k] == K_ACTIVE && !P->solid[k] && !(isfinite(P->rho[k]) && isfinite(P->ux[k])))
                return fail(s, -6, "diverged (non-finite field)");
    }
    return 0;
}

/* ===========================================================================
 * Point probes of the geometry predicates (for sampled checks of grids too large
 * to build here): the walls only, no levels
 * ========================================================================= */

int oracle_set_walls(oracle_solver *s, const double *xy, const int *loop_off, int nloops)
{
    if (!s || (nloops > 0 && (!xy || !loop_off)) || nloops < 0) return -1;
    free_geometry(s);
    return setup_walls(s, xy, loop_off, nloops);
}

/* For level-l cells (ij[2k], ij[2k+1]): solid (centre inside or on a loop), near (centre
 * within R_{l+1} of a wall, the refinement test of level l+1; 0 on the finest level) and
 * the exact distance to the nearest segment in level-l lattice units. */
int oracle_probe_cells(const oracle_solver *s, int level, const int *ij, int n, unsigned char *solid,
                       unsigned char *near, double *dist)
{
    if (!s || level < 0 || level >= s->L || n < 0) return -1;
    const oracle_config *c = &s->cfg;
    const int L = s->L;
    olevel P;
    memset(&P, 0, sizeof P);
    P.scale = 1LL << (L - 1 - level);
    long long R = 0;
    if (level < L - 1) {
        R = (long long)c->layers * FIX_ONE;
        for (int m = L - 2; m >= level + 1; m--) R += (long long)c->layers * (1LL << (L - 1 - m)) * FIX_ONE;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < n; k++) {
        ipt p = centre_fix(&P, ij[2 * k], ij[2 * k + 1]);
        if (solid) solid[k] = (unsigned char)point_solid(s, p);
        if (near) near[k] = (unsigned char)(level < L - 1 ? near_wall(s, p, R) : 0);
        if (dist) {
            double px = (ij[2 * k] + 0.5) * P.scale, py = (ij[2 * k + 1] + 0.5) * P.scale;
            dist[k] = wall_distance(s, px, py, NULL, NULL, NULL) / (double)P.scale;
        }
    }
    return 0;
}

/* wall fraction q of eq 27 for finest-level links (ijd[3k], ijd[3k+1]) -> pulled direction ijd[3k+2] */
int oracle_probe_links(const oracle_solver *s, const int *ijd, int n, double *q)
{
    if (!s || n < 0) return -1;
    olevel F;
    memset(&F, 0, sizeof F);
    F.scale = 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < n; k++) {
        int d = ijd[3 * k + 2];
        ipt pb = centre_fix(&F, ijd[3 * k], ijd[3 * k + 1]);
        ipt dv = {-CX[d] * FIX_ONE, -CY[d] * FIX_ONE};
        q[k] = link_fraction(s, pb, dv);
    }
    return 0;
}

/* ===========================================================================
 * Fields
 * ========================================================================= */

static void present_box(const olevel *P, int *i0, int *j0, int *nx, int *ny)
{
    int a0 = 1 << 30, b0 = 1 << 30, a1 = -(1 << 30), b1 = -(1 << 30);
    for (int j = P->j0; j < P->j0 + P->ny; j++)
        for (int i = P->i0; i < P->i0 + P->nx; i++)
            if (P->kind[cidx(P, i, j)] != K_ABSENT) {
                if (i < a0) a0 = i;
                if (j < b0) b0 = j;
                if (i > a1) a1 = i;
                if (j > b1) b1 = j;
            }
    *i0 = a0; *j0 = b0; *nx = a1 - a0 + 1; *ny = b1 - b0 + 1;
}

int oracle_level_box(const oracle_solver *s, int level, int *i0, int *j0, int *nx, int *ny)
{
    if (!s || !s->geometry || level < 0 || level >= s->L) return -1;
    present_box(&s->lv[level], i0, j0, nx, ny);
    return 0;
}

/* mask: 0 absent, 1 active fluid, 2 boundary node, 3 covered, 4 ghost, 5 solid */
static unsigned char mask_of(const olevel *P, long k)
{
    if (P->kind[k] == K_ABSENT) return 0;
    if (P->solid[k]) return 5;
    if (P->kind[k] == K_COVERED) return 3;
    if (P->kind[k] == K_GHOST) return 4;
    return P->bnode[k] ? 2 : 1;
}

int oracle_get_fields(oracle_solver *s, int level, double *rho, double *ux, double *uy, double *chi,
                      unsigned char *mask, int cap)
{
    int i0, j0, nx, ny;
    if (oracle_level_box(s, level, &i0, &j0, &nx, &ny)) return -1;
    if ((long)nx * ny > cap) return fail(s, -1, "capacity too small");
    const olevel *P = &s->lv[level];
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = cidx(P, i0 + i, j0 + j);
            long o = (long)j * nx + i;
            unsigned char m = mask_of(P, k);
            if (mask) mask[o] = m;
            int has = (m == 1 || m == 2 || m == 3 || m == 4);
            if (rho) rho[o] = has ? P->rho[k] : NAN;
            if (ux) ux[o] = has ? P->ux[k] : NAN;
            if (uy) uy[o] = has ? P->uy[k] : NAN;
            if (chi) chi[o] = has ? P->chi[k] : NAN;
        }
    return 0;
}

int oracle_get_wall_distance(const oracle_solver *s, int level, double *d, int cap)
{
    int i0, j0, nx, ny;
    if (oracle_level_box(s, level, &i0, &j0, &nx, &ny)) return -1;
    if ((long)nx * ny > cap) return -1;
    const olevel *P = &s->lv[level];
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = cidx(P, i0 + i, j0 + j);
            d[(long)j * nx + i] = (P->kind[k] == K_ACTIVE && !P->solid[k]) ? P->d[k] : NAN;
        }
    return 0;
}

/* set macroscopic fields on the active fluid cells of a level; populations are
 * set to the equilibrium of eq 4 and the interfaces re-synchronised */
int oracle_set_fields(oracle_solver *s, int level, const double *rho, const double *ux, const double *uy,
                      const double *chi)
{
    int i0, j0, nx, ny;
    if (oracle_level_box(s, level, &i0, &j0, &nx, &ny)) return -1;
    olevel *P = &s->lv[level];
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = cidx(P, i0 + i, j0 + j);
            long o = (long)j * nx + i;
            if (P->kind[k] != K_ACTIVE || P->solid[k]) continue;
            if (rho) P->rho[k] = rho[o];
            if (ux) P->ux[k] = ux[o];
            if (uy) P->uy[k] = uy[o];
            if (chi) P->chi[k] = P->chin[k] = chi[o];
            oracle_feq(P->rho[k], P->ux[k], P->uy[k], &P->f[9 * k]);
        }
    for (int l = s->L - 2; l >= 0; l--) restrict_level(s, l);
    for (int l = 0; l < s->L - 1; l++) {
        explode_level(s, l, s->lv[l].f);
        prolong_level(s, l);
    }
    return 0;
}

double oracle_mass(const oracle_solver *s)
{
    if (!s || !s->geometry) return NAN;
    double m = 0;
    for (int l = 0; l < s->L; l++) {
        const olevel *P = &s->lv[l];
        double area = (double)P->scale * (double)P->scale;
        double ml = 0;
        long n = (long)P->nx * P->ny;
        for (long k = 0; k < n; k++) {
            if (P->kind[k] != K_ACTIVE || P->solid[k]) continue;
            for (int q = 0; q < 9; q++) ml += P->f[9 * k + q];
        }
        m += area * ml;
    }
    return m;
}

/* ===========================================================================
 * Loads (Sec 3.1.2-3.1.3, eqs 29-30)
 * ========================================================================= */

int oracle_get_loads(oracle_solver *s, oracle_loads *out, double *cp_seg, double *cf_seg, int cap, int *n_seg)
{
    if (!s || !out) return -1;
    if (!s->geometry) return fail(s, -4, "no geometry");
    if (s->nrec > 0) wall_function(s);
    const oracle_config *c = &s->cfg;
    double U = s->U;
    double chord = c->chord / (c->h0 / (double)(1LL << (s->L - 1)));   /* chord in finest cells */
    double CFx = 0, CFy = 0, CPx = 0, CPy = 0;
    if (n_seg) *n_seg = s->nseg;
    for (int k = 0; k < s->nseg; k++) {
        double ax = (double)s->v[s->sa[k]].x / FIX_ONE, ay = (double)s->v[s->sa[k]].y / FIX_ONE;
        double bx = (double)s->v[s->sb[k]].x / FIX_ONE, by = (double)s->v[s->sb[k]].y / FIX_ONE;
        double ds = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
        double tx = (bx - ax) / ds, ty = (by - ay) / ds;
        double nx = s->loop_ccw[s->sloop[k]] ? ty : -ty, ny = s->loop_ccw[s->sloop[k]] ? -tx : tx;
        double cp = 0, cf = 0;
        int b1 = s->seg_b1[k], b2 = s->seg_b2[k];
        if (b1 >= 0) {
            /* eq 29 per boundary node: p = cs^2 rho_R, p_ref = cs^2, rho_ref = 1; rho_w = rho_R */
            const orec *r1 = &s->rec[b1];
            double cp1 = 2.0 * CS2 * (r1->rhoW - 1.0) / (U * U);
            double cf1 = 2.0 * r1->rhoW * (r1->utau / U) * (r1->utau / U);
            double w1 = s->seg_w1[k], w2 = 0, cp2 = 0, cf2 = 0;
            if (b2 >= 0) {
                const orec *r2 = &s->rec[b2];
                w2 = s->seg_w2[k];
                cp2 = 2.0 * CS2 * (r2->rhoW - 1.0) / (U * U);
                cf2 = 2.0 * r2->rhoW * (r2->utau / U) * (r2->utau / U);
            }
            cp = (w1 * cp1 + w2 * cp2) / (w1 + w2);
            cf = (w1 * cf1 + w2 * cf2) / (w1 + w2);
            double sg = (r1->t[0] * tx + r1->t[1] * ty) >= 0 ? 1.0 : -1.0;   /* C_f,sign */
            cf *= sg;
        }
        if (cp_seg && k < cap) cp_seg[k] = cp;
        if (cf_seg && k < cap) cf_seg[k] = cf;
        CFx += cf * tx * ds; CFy += cf * ty * ds;
        CPx -= cp * nx * ds; CPy -= cp * ny * ds;
    }
    CFx /= chord; CFy /= chord; CPx /= chord; CPy /= chord;
    out->CDf = CFx;
    out->CDp = CPx;
    out->CD = CFx + CPx;
    out->CL = CPy;
    out->mass = oracle_mass(s);
    out->dCL = s->have_cl ? out->CL - s->last_cl : 0.0;
    s->last_cl = out->CL;
    s->have_cl = 1;
    out->step = s->step;
    return 0;
}

/* ===========================================================================
 * Geometry tables for bit-exact comparison
 * ========================================================================= */

int oracle_get_cut_links(const oracle_solver *s, int *ijd, double *q, int cap, int *n)
{
    if (!s || !s->geometry) return -1;
    int cnt = 0;
    for (int r = 0; r < s->nrec; r++) {
        const orec *R0 = &s->rec[r];
        const olevel *F = &s->lv[s->L - 1];
        unsigned short m = F->cut[cidx(F, R0->i, R0->j)];
        for (int d = 1; d < 9; d++) {
            if (!(m >> d & 1)) continue;
            if (cnt < cap) {
                ijd[3 * cnt] = R0->i; ijd[3 * cnt + 1] = R0->j; ijd[3 * cnt + 2] = d;
                q[cnt] = R0->q[d];
            }
            cnt++;
        }
    }
    *n = cnt;
    return cnt > cap ? -1 : 0;
}

int oracle_get_wall_records(const oracle_solver *s, int *ij, double *geo, int *ns, int cap, int *n)
{
    if (!s || !s->geometry) return -1;
    *n = s->nrec;
    if (s->nrec > cap) return -1;
    for (int r = 0; r < s->nrec; r++) {
        const orec *R0 = &s->rec[r];
        ij[2 * r] = R0->i; ij[2 * r + 1] = R0->j;
        double *g = &geo[9 * r];
        g[0] = R0->iw[0]; g[1] = R0->iw[1]; g[2] = R0->n[0]; g[3] = R0->n[1];
        g[4] = R0->dwb; g[5] = R0->r[0]; g[6] = R0->r[1]; g[7] = R0->loop; g[8] = R0->seg;
        ns[r] = R0->ns;
    }
    return 0;
}

int oracle_get_wall_state(oracle_solver *s, double *st, int cap, int *n)
{
    if (!s || !s->geometry) return -1;
    *n = s->nrec;
    if (s->nrec > cap) return -1;
    if (s->nrec > 0) wall_function(s);
    for (int r = 0; r < s->nrec; r++) {
        const orec *R0 = &s->rec[r];
        double *g = &st[8 * r];
        g[0] = R0->rhoW; g[1] = R0->uW[0]; g[2] = R0->uW[1]; g[3] = R0->utau;
        g[4] = R0->chiB; g[5] = R0->t[0]; g[6] = R0->t[1]; g[7] = R0->ut;
    }
    return 0;
}
