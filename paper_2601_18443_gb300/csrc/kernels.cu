// kernels.cu -- sm_103a kernels of one LBM-RANS level step.
//
// Populations are stored shifted, g_q = f_q - w_q, in FP32 structure-of-arrays per
// level tile set; every kernel works on one 32 x 8 tile per block, one cell per
// thread.  The collision is the central-moment operator of eqs 5-7 evaluated in
// closed form on the shifted raw moments (rest-state moments subtracted
// analytically), so that FP32 keeps the small departures from rest exact to
// ~1e-7 relative.  No step is a dense contraction; the kernels are HBM/L2 bound.
#include <math.h>

#include "device.cuh"

namespace lbmdev {

// ------------------------------------------------------------------ lattice
__host__ __device__ constexpr int cxq(int q) { return q == 1 || q == 5 || q == 7 ? 1 : (q == 2 || q == 6 || q == 8 ? -1 : 0); }
__host__ __device__ constexpr int cyq(int q) { return q == 3 || q == 5 || q == 8 ? 1 : (q == 4 || q == 6 || q == 7 ? -1 : 0); }
__host__ __device__ constexpr int oppq(int q) { return q == 0 ? 0 : (q & 1 ? q + 1 : q - 1); }
__host__ __device__ constexpr float wq(int q) { return q == 0 ? 4.f / 9.f : (q < 5 ? 1.f / 9.f : 1.f / 36.f); }
// direction with the same c_x and the opposite c_y (specular reflection on a horizontal plane)
__host__ __device__ constexpr int mirror_y(int q)
{
    return q == 3 ? 4 : q == 4 ? 3 : q == 5 ? 7 : q == 7 ? 5 : q == 6 ? 8 : q == 8 ? 6 : q;
}

__device__ __forceinline__ int dir_of(int sx, int sy)
{
    // D2Q9 index of the unit offset (sx, sy)
    return sy == 0 ? (sx == 0 ? 0 : (sx > 0 ? 1 : 2)) : (sy > 0 ? (sx == 0 ? 3 : (sx > 0 ? 5 : 8)) : (sx == 0 ? 4 : (sx > 0 ? 7 : 6)));
}

// slot of the cell at offset (dx, dy) from (lx, ly) in tile t, or -1
__device__ __forceinline__ long long nb_slot(const LevelView &P, int t, int lx, int ly, int dx, int dy)
{
    int nx = lx + dx, ny = ly + dy;
    int sx = nx < 0 ? -1 : (nx >= LBM_TX ? 1 : 0);
    int sy = ny < 0 ? -1 : (ny >= LBM_TY ? 1 : 0);
    int tt = t;
    if (sx | sy) {
        tt = P.nbr[t * 9 + dir_of(sx, sy)];
        if (tt < 0) return -1;
    }
    return (long long)tt * LBM_TILE + ((ny + LBM_TY) & (LBM_TY - 1)) * LBM_TX + ((nx + LBM_TX) & (LBM_TX - 1));
}

// level 0 covers its whole box with tiles in row-major order
__device__ __forceinline__ long long slot0(const StepConsts &k, int i, int j)
{
    return ((long long)(j >> 3) * k.ntx0 + (i >> 5)) * LBM_TILE + (j & 7) * LBM_TX + (i & 31);
}

// the tile of level l+1 holding the four children of (lx, ly) and their first slot
__device__ __forceinline__ long long child_base(const LevelView &P, int t, int lx, int ly)
{
    int ct = P.child[t * 4 + ((2 * ly) >> 3) * 2 + ((2 * lx) >> 5)];
    if (ct < 0) return -1;
    return (long long)ct * LBM_TILE + ((2 * ly) & 7) * LBM_TX + ((2 * lx) & 31);
}

// ------------------------------------------------------------------ SA-neg constants (Sec 2.2)
#define SA_CB1 0.1355f
#define SA_CB2 0.622f
#define SA_SIGMA (2.0f / 3.0f)
#define SA_KAPPA 0.41f
#define SA_CW1 3.2390678f             /* cb1 / kappa^2 + (1 + cb2) / sigma */
#define SA_CW2 0.3f
#define SA_CW3_6 64.0f                /* cw3^6, cw3 = 2 */
#define SA_CV1_3 357.911f             /* cv1^3, cv1 = 7.1 */
#define SA_RLIM 10.0f
#define SA_CV2 0.7f
#define SA_CV3 0.9f                   /* reading: value of the SA-neg source the paper follows */
#define SA_CT3 1.2f
#define SA_CN1 16.0f

// ------------------------------------------------------------------ collision (eqs 5-10)
// Input: post-stream shifted populations g (f - w).  Output: post-collision shifted
// populations.  drho, ux, uy: the macroscopic fields of eq 3.  delta = 2 - omega_nu
// (omega_b = 1: the trace relaxes fully, Sec 2.1).
__device__ __forceinline__ void collide_cm(const float g[9], float drho, float ux, float uy, float delta, float o[9])
{
    const float rho = 1.0f + drho;
    const float m20 = g[1] + g[2] + g[5] + g[6] + g[7] + g[8];   // sum cx^2 g  (= m20 - 1/3)
    const float m02 = g[3] + g[4] + g[5] + g[6] + g[7] + g[8];   // sum cy^2 g
    const float m11 = g[5] + g[6] - g[7] - g[8];
    const float uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const float D = (m20 - m02) - rho * (uxx - uyy);              // k20 - k02
    const float K = m11 - rho * uxy;                              // k11
    const float Ds = delta * D - D;                               // (1 - omega) (k20 - k02)
    const float Ks = delta * K - K;                               // (1 - omega) k11
    const float k20 = rho * (1.0f / 3.0f) + 0.5f * Ds;            // post-collision central moments
    const float k02 = rho * (1.0f / 3.0f) - 0.5f * Ds;
    // raw post-collision moments minus their rest-state values (binomial shift back)
    const float M00 = drho;
    const float M10 = rho * ux, M01 = rho * uy;
    const float M20 = drho * (1.0f / 3.0f) + 0.5f * Ds + rho * uxx;
    const float M02 = drho * (1.0f / 3.0f) - 0.5f * Ds + rho * uyy;
    const float M11 = Ks + rho * uxy;
    const float M21 = uy * k20 + 2.0f * ux * Ks + rho * uxx * uy;
    const float M12 = ux * k02 + 2.0f * uy * Ks + rho * ux * uyy;
    const float M22 = drho * (1.0f / 9.0f) + uyy * k20 + uxx * k02 + 4.0f * uxy * Ks + rho * uxx * uyy;
    // populations from the nine raw moments of D2Q9
    o[0] = M00 - M20 - M02 + M22;
    o[1] = 0.5f * (M10 + M20 - M12 - M22);
    o[2] = 0.5f * (-M10 + M20 + M12 - M22);
    o[3] = 0.5f * (M01 + M02 - M21 - M22);
    o[4] = 0.5f * (-M01 + M02 + M21 - M22);
    o[5] = 0.25f * (M11 + M21 + M12 + M22);
    o[6] = 0.25f * (M11 - M21 - M12 + M22);
    o[7] = 0.25f * (-M11 - M21 + M12 + M22);
    o[8] = 0.25f * (-M11 + M21 - M12 + M22);
}

__device__ __forceinline__ float sa_fv1(float chi)
{
    float c3 = chi * chi * chi;
    return c3 / (c3 + SA_CV1_3);
}

// 2 - omega for the effective viscosity nu + nu_t (eq 9 with the RANS substitution)
__device__ __forceinline__ float delta_of(float nu, float chi, int turbulence)
{
    float nue = nu;
    if (turbulence) nue += fmaxf(chi, 0.0f) * nu * sa_fv1(chi);
    return 12.0f * nue / (1.0f + 6.0f * nue);
}

// ------------------------------------------------------------------ stream + collide
__device__ __forceinline__ float pull0(const StepConsts &k, const float *fc, long long ns, int i, int j, int q)
{
    // post-stream value at level-0 cell (i, j), direction q, source inside the box in x
    int si = i - cxq(q), sj = j - cyq(q);
    if (sj >= 0 && sj < k.ny0) return fc[q * ns + slot0(k, si, sj)];
    return fc[mirror_y(q) * ns + slot0(k, si, j)];
}

__global__ void __launch_bounds__(256) k_stream_collide(LevelView P, LevelView F, int has_child, int cur, int fcur,
                                                         int fchicur, RecView R, StepConsts k, int is_level0)
{
    const int t = blockIdx.x, c = threadIdx.x;
    const int lx = c & (LBM_TX - 1), ly = c >> 5;
    const long long slot = (long long)t * LBM_TILE + c;
    const uint32_t fl = P.flags[slot];
    const uint32_t kind = fl & FL_KIND_MASK;
    if (kind == KIND_ABSENT || (fl & FL_SOLID)) return;
    const long long ns = P.ns;
    const float *fc = P.f[cur];
    float *fn = P.f[cur ^ 1];

    if (kind == KIND_COVERED) {
        // restriction of the macroscopic fields from the four children (time t+1)
        long long cb = child_base(P, t, lx, ly);
        if (cb < 0) return;
        float sdr = 0.f, sr = 0.f, sx = 0.f, sy = 0.f, sc = 0.f;
        int n = 0;
        const long long off[4] = {0, 1, LBM_TX, LBM_TX + 1};
#pragma unroll
        for (int m = 0; m < 4; m++) {
            long long cs = cb + off[m];
            if (F.flags[cs] & FL_SOLID) continue;
            float dr = F.drho[cs], r = 1.0f + dr;
            sdr += dr; sr += r; sx += r * F.ux[cs]; sy += r * F.uy[cs]; sc += F.chi[fchicur][cs];
            n++;
        }
        if (n == 0) return;
        P.drho[slot] = sdr / n; P.ux[slot] = sx / sr; P.uy[slot] = sy / sr;
        P.chi[cur ^ 1][slot] = sc / n;
        return;
    }
    if (kind == KIND_GHOST) {
        // ghosts are streamed (relayed), never collided
#pragma unroll
        for (int q = 0; q < 9; q++) {
            long long s = nb_slot(P, t, lx, ly, -cxq(q), -cyq(q));
            bool ok = false;
            if (s >= 0) {
                uint32_t fs = P.flags[s];
                uint32_t ks = fs & FL_KIND_MASK;
                ok = (ks == KIND_ACTIVE || ks == KIND_GHOST) && !(fs & FL_SOLID);
            }
            fn[q * ns + slot] = ok ? fc[q * ns + s] : fc[q * ns + slot];
        }
        return;
    }

    float g[9];
    g[0] = fc[slot];
    const bool edge = is_level0 && k.level0_edges && (fl & (FL_INLET | FL_OUTLET | FL_BOTTOM | FL_TOP));
    if (!edge) {
#pragma unroll
        for (int q = 1; q < 9; q++) {
            if (fl & (1u << (FL_COAL_SHIFT + q - 1))) {
                // coalescence: mean of the four ghost children after the two fine sub-steps
                long long cb = child_base(P, t, lx, ly);
                const float *ff = F.f[fcur] + q * F.ns;
                g[q] = cb >= 0 ? 0.25f * (ff[cb] + ff[cb + 1] + ff[cb + LBM_TX] + ff[cb + LBM_TX + 1]) : fc[q * ns + slot];
            } else if (fl & (1u << (FL_CUT_SHIFT + q - 1))) {
                // Yu interpolated bounce-back with the slip velocity of the wall record (eq 27)
                const int r = P.rec[slot];
                const int qo = oppq(q);
                const float qf = R.q[r * 9 + q];
                const float mom = 6.0f * wq(q) * (1.0f + R.drhoW[r]) * (cxq(q) * R.uWx[r] + cyq(q) * R.uWy[r]);
                long long sf = nb_slot(P, t, lx, ly, cxq(q), cyq(q));
                bool ok = false;
                if (sf >= 0) {
                    uint32_t ff = P.flags[sf];
                    ok = (ff & FL_KIND_MASK) == KIND_ACTIVE && !(ff & FL_SOLID);
                }
                if (ok)
                    g[q] = ((1.0f - qf) * fc[qo * ns + sf] + qf * fc[qo * ns + slot] + mom) / (1.0f + qf) +
                           qf / (1.0f + qf) * fc[q * ns + slot];
                else
                    g[q] = fc[qo * ns + slot] + mom;                // half-way form, eq 24
            } else {
                long long s = nb_slot(P, t, lx, ly, -cxq(q), -cyq(q));
                g[q] = fc[q * ns + (s >= 0 ? s : slot)];
            }
        }
    } else {
        // level-0 box edge: in-box pulls, symmetry planes, Zou-He inlet, extrapolated outlet
        const int i = P.tile_x[t] * LBM_TX + lx, j = P.tile_y[t] * LBM_TY + ly;
#pragma unroll
        for (int q = 1; q < 9; q++) {
            int si = i - cxq(q), sj = j - cyq(q);
            bool xin = si >= 0 && si < k.nx0, yin = sj >= 0 && sj < k.ny0;
            if (xin && yin) g[q] = fc[q * ns + slot0(k, si, sj)];
            else if (xin) g[q] = fc[mirror_y(q) * ns + slot0(k, si, j)];
            else g[q] = 0.0f;
        }
        if (i == 0) {
            const float U = k.U;
            float S = g[0] + g[3] + g[4] + 2.0f * (g[2] + g[6] + g[8]);       // sum of w over these is 1
            float rho = (1.0f + S) / (1.0f - U);
            g[1] = g[2] + (2.0f / 3.0f) * rho * U;
            g[5] = g[6] - 0.5f * (g[3] - g[4]) + rho * U * (1.0f / 6.0f);
            g[7] = g[8] + 0.5f * (g[3] - g[4]) + rho * U * (1.0f / 6.0f);
        }
        if (i == k.nx0 - 1) {
            const int qs[3] = {2, 6, 8};
#pragma unroll
            for (int m = 0; m < 3; m++) {
                int q = qs[m];
                g[q] = 2.0f * pull0(k, fc, ns, k.nx0 - 2, j, q) - pull0(k, fc, ns, k.nx0 - 3, j, q);
            }
        }
    }
    // macroscopic fields (eq 3)
    const float drho = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
    const float rho = 1.0f + drho;
    const float ux = (g[1] - g[2] + g[5] - g[6] + g[7] - g[8]) / rho;
    const float uy = (g[3] - g[4] + g[5] - g[6] - g[7] + g[8]) / rho;
    P.drho[slot] = drho; P.ux[slot] = ux; P.uy[slot] = uy;
    const float chi = k.turbulence ? P.chi[cur ^ 1][slot] : 0.0f;
    float o[9];
    collide_cm(g, drho, ux, uy, delta_of(P.nu, chi, k.turbulence), o);
#pragma unroll
    for (int q = 0; q < 9; q++) fn[q * ns + slot] = o[q];
    if (has_child && (fl & FL_BAND)) {
        // explosion: post-collision populations copied to the four ghost children
        long long cb = child_base(P, t, lx, ly);
        if (cb >= 0) {
#pragma unroll
            for (int q = 0; q < 9; q++) {
                float *ff = F.f[fcur] + q * F.ns;
                ff[cb] = o[q]; ff[cb + 1] = o[q]; ff[cb + LBM_TX] = o[q]; ff[cb + LBM_TX + 1] = o[q];
            }
        }
    }
}

// ------------------------------------------------------------------ SA-neg (Sec 2.2)
struct Stencil {
    float chi[9], ux[9], uy[9];
};

__device__ __forceinline__ void gather(const LevelView &P, const float *chi, int t, int lx, int ly, long long slot,
                                       Stencil &S)
{
#pragma unroll
    for (int q = 0; q < 9; q++) {
        long long s = q == 0 ? slot : nb_slot(P, t, lx, ly, cxq(q), cyq(q));
        if (s < 0) s = slot;
        S.chi[q] = chi[s]; S.ux[q] = P.ux[s]; S.uy[q] = P.uy[s];
    }
}

// level-0 box edge: neighbours across the top/bottom symmetry planes are mirror images
__device__ __forceinline__ void gather0(const LevelView &P, const float *chi, const StepConsts &k, int i, int j,
                                        Stencil &S)
{
#pragma unroll
    for (int q = 0; q < 9; q++) {
        int ii = i + cxq(q), jj = j + cyq(q);
        float sg = 1.0f;
        if (jj < 0) { jj = 0; sg = -1.0f; }
        if (jj >= k.ny0) { jj = k.ny0 - 1; sg = -1.0f; }
        if (ii < 0) ii = 0;
        if (ii >= k.nx0) ii = k.nx0 - 1;
        long long s = slot0(k, ii, jj);
        S.chi[q] = chi[s]; S.ux[q] = P.ux[s]; S.uy[q] = sg * P.uy[s];
    }
}

// LSQ gradient over the full D2Q9 neighbourhood: sum_k c_k (phi_k - phi_0) / 6
__device__ __forceinline__ void lsq_grad(const float *v, float &gx, float &gy)
{
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int q = 1; q < 9; q++) { sx += cxq(q) * (v[q] - v[0]); sy += cyq(q) * (v[q] - v[0]); }
    gx = sx * (1.0f / 6.0f); gy = sy * (1.0f / 6.0f);
}

__device__ __forceinline__ float sa_diff_coef(float chi)
{   // (nu + nu_t~ f_n) / nu
    float fn = 1.0f;
    if (chi < 0.0f) { float c3 = chi * chi * chi; fn = (SA_CN1 + c3) / (SA_CN1 - c3); }
    return 1.0f + chi * fn;
}

// explicit Euler + Lax-Wendroff step of eqs 12 / 16 written for chi = nu_t~ / nu
__device__ float sa_update(const Stencil &S, float d, float nu)
{
    float dudx, dudy, dvdx, dvdy;
    lsq_grad(S.ux, dudx, dudy);
    lsq_grad(S.uy, dvdx, dvdy);
    const float vort = fabsf(dvdx - dudy);
    const float *x = S.chi;      // 0 C, 1 E, 2 W, 3 N, 4 S, 5 NE, 6 SW, 7 SE, 8 NW
    const float gx = 0.5f * (x[1] - x[2]), gy = 0.5f * (x[3] - x[4]);
    const float gxx = x[1] - 2.0f * x[0] + x[2], gyy = x[3] - 2.0f * x[0] + x[4];
    const float gxy = 0.25f * (x[5] - x[8] - x[7] + x[6]);
    const float u = S.ux[0], v = S.uy[0];
    const float conv = -(u * gx + v * gy) + 0.5f * (u * u * gxx + 2.0f * u * v * gxy + v * v * gyy);
    const float Dc = sa_diff_coef(x[0]);
    const float De = 0.5f * (Dc + sa_diff_coef(x[1])), Dw = 0.5f * (Dc + sa_diff_coef(x[2]));
    const float Dn = 0.5f * (Dc + sa_diff_coef(x[3])), Ds = 0.5f * (Dc + sa_diff_coef(x[4]));
    const float div = De * (x[1] - x[0]) - Dw * (x[0] - x[2]) + Dn * (x[3] - x[0]) - Ds * (x[0] - x[4]);
    const float diff = nu * (div + SA_CB2 * (gx * gx + gy * gy)) * (1.0f / SA_SIGMA);
    const float chi = x[0];
    const float kd2 = SA_KAPPA * SA_KAPPA * d * d;
    float src;
    if (chi >= 0.0f) {
        const float fv1 = sa_fv1(chi);
        const float fv2 = 1.0f - chi / (1.0f + chi * fv1);
        const float sbar = nu * chi * fv2 / kd2;
        float st;
        if (sbar >= -SA_CV2 * vort) st = vort + sbar;
        else st = vort + vort * (SA_CV2 * SA_CV2 * vort + SA_CV3 * sbar) / ((SA_CV3 - 2.0f * SA_CV2) * vort - sbar);
        float r = SA_RLIM;
        if (st > 0.0f) r = fminf(nu * chi / (st * kd2), SA_RLIM);
        const float r2 = r * r, r6 = r2 * r2 * r2;
        const float gg = r + SA_CW2 * (r6 - r);
        const float g2 = gg * gg, g6 = g2 * g2 * g2;
        const float fw = gg * powf((1.0f + SA_CW3_6) / (g6 + SA_CW3_6), 1.0f / 6.0f);
        src = SA_CB1 * st * chi - SA_CW1 * fw * nu * chi * chi / (d * d);
    } else {
        src = SA_CB1 * (1.0f - SA_CT3) * vort * chi + SA_CW1 * nu * chi * chi / (d * d);
    }
    return chi + conv + src + diff;
}

__global__ void __launch_bounds__(256) k_sa(LevelView P, LevelView F, int has_child, int cur, RecView R,
                                             StepConsts k, int is_level0)
{
    const int t = blockIdx.x, c = threadIdx.x;
    const int lx = c & (LBM_TX - 1), ly = c >> 5;
    const long long slot = (long long)t * LBM_TILE + c;
    const uint32_t fl = P.flags[slot];
    if ((fl & FL_KIND_MASK) != KIND_ACTIVE || (fl & FL_SOLID)) return;
    const float *chi = P.chi[cur];
    float *chin = P.chi[cur ^ 1];
    const bool edge = is_level0 && k.level0_edges && (fl & (FL_INLET | FL_OUTLET | FL_BOTTOM | FL_TOP));
    Stencil S;
    if (has_child && (fl & FL_BAND)) {
        // ghost children of the next level: LSQ linear reconstruction about this cell (time t)
        gather(P, chi, t, lx, ly, slot, S);
        float gcx, gcy, gux, guy, gvx, gvy;
        lsq_grad(S.chi, gcx, gcy); lsq_grad(S.ux, gux, guy); lsq_grad(S.uy, gvx, gvy);
        long long cb = child_base(P, t, lx, ly);
        if (cb >= 0) {
            const float dr = P.drho[slot];
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const int a = m & 1, b = m >> 1;
                const float ox = 0.5f * (a - 0.5f), oy = 0.5f * (b - 0.5f);
                const long long cs = cb + b * LBM_TX + a;
                const float vc = S.chi[0] + gcx * ox + gcy * oy;
                F.chi[0][cs] = vc; F.chi[1][cs] = vc;
                F.ux[cs] = S.ux[0] + gux * ox + guy * oy;
                F.uy[cs] = S.uy[0] + gvx * ox + gvy * oy;
                F.drho[cs] = dr;
            }
        }
    }
    if (fl & FL_BNODE) { chin[slot] = R.chiB[P.rec[slot]]; return; }   // Dirichlet nu_t~_B (Sec 2.2)
    if (edge) {
        const int i = P.tile_x[t] * LBM_TX + lx, j = P.tile_y[t] * LBM_TY + ly;
        if (fl & FL_INLET) { chin[slot] = k.chi_inf; return; }
        const int ic = (fl & FL_OUTLET) ? k.nx0 - 2 : i;                   // outlet: copy of its neighbour
        gather0(P, chi, k, ic, j, S);
        chin[slot] = sa_update(S, P.dist[slot0(k, ic, j)], P.nu);
        return;
    }
    if (!(has_child && (fl & FL_BAND))) gather(P, chi, t, lx, ly, slot, S);
    chin[slot] = sa_update(S, P.dist[slot], P.nu);
}

// ------------------------------------------------------------------ wall function (Sec 2.3 steps 1-5)
#define WF_B 5.033908790505579f
#define WF_A1 8.148221580024245f
#define WF_A2 (-6.9287093849022945f)
#define WF_B1 7.4600876082527945f
#define WF_B2 7.468145790401841f
#define WF_C1 2.5496773539754747f
#define WF_C2 1.3301651588535228f
#define WF_C3 3.599459109332379f
#define WF_C4 3.639753186868684494f

__device__ __forceinline__ float wf_uplus(float y)
{   // eq 22, continuous arctangent branch
    float t1 = (y + WF_A1) * (y + WF_A1) + WF_B1 * WF_B1;
    float t2 = (y + WF_A2) * (y + WF_A2) + WF_B2 * WF_B2;
    return WF_B + WF_C1 * logf(t1) - WF_C2 * logf(t2) - WF_C3 * atan2f(WF_B1, y + WF_A1) - WF_C4 * atan2f(WF_B2, y + WF_A2);
}

__device__ __forceinline__ float wf_dudy(float y)
{   // eq 21
    float k3 = SA_KAPPA * y;
    k3 = k3 * k3 * k3;
    return (SA_CV1_3 + k3) / (SA_CV1_3 + k3 * (1.0f + SA_KAPPA * y));
}

// friction velocity from u_t at distance y (Newton inside a sign bracket, bounded iterations)
__device__ float wf_utau(float ut, float y, float nu)
{
    if (!(ut > 0.0f)) return 0.0f;
    float lo = 0.0f, hi = sqrtf(ut * nu / y);
    for (int it = 0; it < 128; it++) {
        if (hi * wf_uplus(hi * y / nu) - ut > 0.0f) break;
        lo = hi;
        hi *= 2.0f;
    }
    float u = 0.5f * (lo + hi);
    for (int it = 0; it < 40; it++) {
        const float yp = u * y / nu;
        const float up = wf_uplus(yp);
        const float gv = u * up - ut;
        if (gv > 0.0f) hi = u; else lo = u;
        const float gp = up + yp * wf_dudy(yp);
        float un = gp > 0.0f ? u - gv / gp : 0.5f * (lo + hi);
        if (!(un > lo && un < hi)) un = 0.5f * (lo + hi);
        const bool done = fabsf(un - u) <= 2e-7f * un;
        u = un;
        if (done || hi - lo <= 2e-7f * hi) break;
    }
    return u;
}

// one half-warp per wall record: the 16 lanes hold the 4 x 4 reference stencil
__global__ void __launch_bounds__(256) k_wallfn(LevelView P, RecView R, StepConsts k)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = gt >> 4, m = gt & 15;
    const bool valid = r < R.n;
    float v[13];
#pragma unroll
    for (int a = 0; a < 13; a++) v[a] = 0.0f;
    if (valid && m < R.ns[r]) {
        const long long s = R.st_slot[r * 16 + m];
        const float dx = R.st_dx[r * 16 + m], dy = R.st_dy[r * 16 + m];
        const float dr = P.drho[s], u = P.ux[s], w = P.uy[s];
        const float wt = 1.0f / fmaxf(dx * dx + dy * dy, 1e-20f);
        v[0] = wt; v[1] = wt * dr; v[2] = wt * u; v[3] = wt * w;                  // IDW sums
        v[4] = 1.0f; v[5] = dx; v[6] = dy; v[7] = dx * dx; v[8] = dx * dy; v[9] = dy * dy;   // LSQ normal matrix
        v[10] = u; v[11] = u * dx; v[12] = u * dy;
    }
    // the v-component LSQ right-hand side uses a second pass of the same lanes
    float wv0 = 0.f, wv1 = 0.f, wv2 = 0.f;
    if (valid && m < R.ns[r]) {
        const long long s = R.st_slot[r * 16 + m];
        const float dx = R.st_dx[r * 16 + m], dy = R.st_dy[r * 16 + m], w = P.uy[s];
        wv0 = w; wv1 = w * dx; wv2 = w * dy;
    }
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
#pragma unroll
        for (int a = 0; a < 13; a++) v[a] += __shfl_xor_sync(0xffffffffu, v[a], off);
        wv0 += __shfl_xor_sync(0xffffffffu, wv0, off);
        wv1 += __shfl_xor_sync(0xffffffffu, wv1, off);
        wv2 += __shfl_xor_sync(0xffffffffu, wv2, off);
    }
    if (!valid || m != 0) return;
    const int ns = R.ns[r];
    float drR = 0.f, uR = 0.f, vR = 0.f;
    if (ns > 0) { drR = v[1] / v[0]; uR = v[2] / v[0]; vR = v[3] / v[0]; }
    // unweighted linear LSQ u = a + b dx + c dy: intercept a by Cramer's rule
    const float A0 = v[4], A1 = v[5], A2 = v[6], A4 = v[7], A5 = v[8], A8 = v[9];
    const float det = A0 * (A4 * A8 - A5 * A5) - A1 * (A1 * A8 - A5 * A2) + A2 * (A1 * A5 - A4 * A2);
    if (ns >= 3 && det > 1e-9f * A0 * A4 * A8) {
        const float c0 = A4 * A8 - A5 * A5, c1 = A2 * A5 - A1 * A8, c2 = A1 * A5 - A2 * A4;
        uR = (c0 * v[10] + c1 * v[11] + c2 * v[12]) / det;
        vR = (c0 * wv0 + c1 * wv1 + c2 * wv2) / det;
    }
    const float nx = R.nx[r], ny = R.ny[r];
    const float un = uR * nx + vR * ny;
    const float utx = uR - un * nx, uty = vR - un * ny;
    const float ut = sqrtf(utx * utx + uty * uty);
    float tx = -ny, ty = nx;
    if (ut > 0.0f) { tx = utx / ut; ty = uty / ut; }
    float utau = 0.f, uWx = 0.f, uWy = 0.f, chiB = 0.f;
    if (k.wall_model == 0) {
        const float nu = P.nu;
        utau = wf_utau(ut, k.d_wr, nu);                                     // step 3
        const float ypv = utau * k.d_wv / nu;
        const float uV = utau * wf_uplus(ypv);                              // step 4
        const float uW = uV - utau * utau * k.d_wv / (nu * (1.0f + SA_KAPPA * ypv));   // eq 28
        uWx = uW * tx; uWy = uW * ty;                                       // step 5
        chiB = SA_KAPPA * utau * R.dwb[r] / nu;
    } else if (k.wall_model == 2) {
        uWx = R.slip[2 * R.loop[r]]; uWy = R.slip[2 * R.loop[r] + 1];
    }
    R.drhoW[r] = drR; R.uWx[r] = uWx; R.uWy[r] = uWy; R.utau[r] = utau; R.chiB[r] = chiB;
    R.tx[r] = tx; R.ty[r] = ty; R.ut[r] = ut;
}

// ------------------------------------------------------------------ interface sync (set_fields)
__global__ void k_restrict(LevelView P, LevelView F, int pchi, int fchi)
{
    const int t = blockIdx.x, c = threadIdx.x;
    const long long slot = (long long)t * LBM_TILE + c;
    const uint32_t fl = P.flags[slot];
    if ((fl & FL_KIND_MASK) != KIND_COVERED) return;
    long long cb = child_base(P, t, c & 31, c >> 5);
    if (cb < 0) return;
    float sdr = 0.f, sr = 0.f, sx = 0.f, sy = 0.f, sc = 0.f;
    int n = 0;
    const long long off[4] = {0, 1, LBM_TX, LBM_TX + 1};
    for (int m = 0; m < 4; m++) {
        long long cs = cb + off[m];
        if (F.flags[cs] & FL_SOLID) continue;
        float dr = F.drho[cs], r = 1.0f + dr;
        sdr += dr; sr += r; sx += r * F.ux[cs]; sy += r * F.uy[cs]; sc += F.chi[fchi][cs];
        n++;
    }
    if (n == 0) return;
    P.drho[slot] = sdr / n; P.ux[slot] = sx / sr; P.uy[slot] = sy / sr;
    P.chi[pchi][slot] = sc / n;
}

__global__ void k_explode_prolong(LevelView P, LevelView F, int cur, int fcur, StepConsts k)
{
    const int t = blockIdx.x, c = threadIdx.x;
    const int lx = c & 31, ly = c >> 5;
    const long long slot = (long long)t * LBM_TILE + c;
    const uint32_t fl = P.flags[slot];
    if ((fl & FL_KIND_MASK) != KIND_ACTIVE || (fl & FL_SOLID) || !(fl & FL_BAND)) return;
    long long cb = child_base(P, t, lx, ly);
    if (cb < 0) return;
    Stencil S;
    gather(P, P.chi[cur], t, lx, ly, slot, S);
    float gcx, gcy, gux, guy, gvx, gvy;
    lsq_grad(S.chi, gcx, gcy); lsq_grad(S.ux, gux, guy); lsq_grad(S.uy, gvx, gvy);
    for (int m = 0; m < 4; m++) {
        const int a = m & 1, b = m >> 1;
        const float ox = 0.5f * (a - 0.5f), oy = 0.5f * (b - 0.5f);
        const long long cs = cb + b * LBM_TX + a;
        const float vc = S.chi[0] + gcx * ox + gcy * oy;
        F.chi[0][cs] = vc; F.chi[1][cs] = vc;
        F.ux[cs] = S.ux[0] + gux * ox + guy * oy;
        F.uy[cs] = S.uy[0] + gvx * ox + gvy * oy;
        F.drho[cs] = P.drho[slot];
        for (int q = 0; q < 9; q++) F.f[fcur][q * F.ns + cs] = P.f[cur][q * P.ns + slot];
    }
}

struct Feq9 { float g[9]; };

__global__ void k_init(LevelView P, Feq9 e, float U, float chi_inf)
{
    const long long slot = (long long)blockIdx.x * LBM_TILE + threadIdx.x;
    const uint32_t fl = P.flags[slot];
    const bool present = (fl & FL_KIND_MASK) != KIND_ABSENT;
    for (int q = 0; q < 9; q++) {
        float v = present ? e.g[q] : 0.0f;
        P.f[0][q * P.ns + slot] = v;
        P.f[1][q * P.ns + slot] = v;
    }
    P.drho[slot] = 0.0f;
    P.ux[slot] = present ? U : 0.0f;
    P.uy[slot] = 0.0f;
    P.chi[0][slot] = chi_inf;
    P.chi[1][slot] = chi_inf;
}

// ------------------------------------------------------------------ FP64 reductions
__device__ __forceinline__ double warp_sum(double v)
{
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// surface loads, eqs 29-30: per segment IDW of C_p and signed C_f from two boundary nodes
__global__ void __launch_bounds__(256) k_loads(LoadsView S, RecView R, float U, double *acc)
{
    __shared__ double red[4][8];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double cfx = 0, cfy = 0, cpx = 0, cpy = 0;
    if (k < S.nseg) {
        const int b1 = S.b1[k], b2 = S.b2[k];
        double cp = 0, cf = 0;
        if (b1 >= 0) {
            const double U2 = (double)U * (double)U;
            const double rho1 = 1.0 + (double)R.drhoW[b1];
            const double cp1 = 2.0 / 3.0 * (double)R.drhoW[b1] / U2;
            const double cf1 = 2.0 * rho1 * (double)R.utau[b1] * (double)R.utau[b1] / U2;
            double w1 = S.w1[k], w2 = 0, cp2 = 0, cf2 = 0;
            if (b2 >= 0) {
                const double rho2 = 1.0 + (double)R.drhoW[b2];
                w2 = S.w2[k];
                cp2 = 2.0 / 3.0 * (double)R.drhoW[b2] / U2;
                cf2 = 2.0 * rho2 * (double)R.utau[b2] * (double)R.utau[b2] / U2;
            }
            cp = (w1 * cp1 + w2 * cp2) / (w1 + w2);
            cf = (w1 * cf1 + w2 * cf2) / (w1 + w2);
            const double sg = ((double)R.tx[b1] * S.tx[k] + (double)R.ty[b1] * S.ty[k]) >= 0.0 ? 1.0 : -1.0;
            cf *= sg;
        }
        S.cp[k] = cp;
        S.cf[k] = cf;
        cfx = cf * S.tx[k] * S.ds[k]; cfy = cf * S.ty[k] * S.ds[k];
        cpx = -cp * S.nx[k] * S.ds[k]; cpy = -cp * S.ny[k] * S.ds[k];
    }
    cfx = warp_sum(cfx); cfy = warp_sum(cfy); cpx = warp_sum(cpx); cpy = warp_sum(cpy);
    const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (ln == 0) { red[0][w] = cfx; red[1][w] = cfy; red[2][w] = cpx; red[3][w] = cpy; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0;
        for (int i = 0; i < 8; i++) s += red[threadIdx.x][i];
        atomicAdd(&acc[threadIdx.x], s);
    }
}

__global__ void __launch_bounds__(256) k_mass(LevelView P, double area, double *acc, int *status)
{
    __shared__ double red[8];
    const long long slot = (long long)blockIdx.x * LBM_TILE + threadIdx.x;
    const uint32_t fl = P.flags[slot];
    double v = 0;
    if ((fl & FL_KIND_MASK) == KIND_ACTIVE && !(fl & FL_SOLID)) {
        const float dr = P.drho[slot], u = P.ux[slot], w = P.uy[slot];
        if (!(isfinite(dr) && isfinite(u) && isfinite(w))) atomicOr(status, 1);
        v = area * (1.0 + (double)dr);
    }
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int i = 0; i < 8; i++) s += red[i];
        atomicAdd(acc, s);
    }
}

// ------------------------------------------------------------------ launchers
void launch_stream_collide(cudaStream_t st, const LevelView &P, const LevelView *F, int cur, int fcur, int fchicur,
                           const RecView &R, const StepConsts &k, int is_level0)
{
    LevelView Fv = F ? *F : P;
    k_stream_collide<<<P.ntiles, LBM_TILE, 0, st>>>(P, Fv, F != nullptr, cur, fcur, fchicur, R, k, is_level0);
}

void launch_sa(cudaStream_t st, const LevelView &P, const LevelView *F, int cur, const RecView &R,
               const StepConsts &k, int is_level0)
{
    LevelView Fv = F ? *F : P;
    k_sa<<<P.ntiles, LBM_TILE, 0, st>>>(P, Fv, F != nullptr, cur, R, k, is_level0);
}

void launch_wallfn(cudaStream_t st, const LevelView &P, const RecView &R, const StepConsts &k)
{
    if (R.n <= 0) return;
    const long long threads = (long long)R.n * 16;
    k_wallfn<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P, R, k);
}

void launch_restrict(cudaStream_t st, const LevelView &P, const LevelView &F, int pchi, int fchi)
{
    k_restrict<<<P.ntiles, LBM_TILE, 0, st>>>(P, F, pchi, fchi);
}

void launch_explode_prolong(cudaStream_t st, const LevelView &P, const LevelView &F, int cur, int fcur,
                            const StepConsts &k)
{
    k_explode_prolong<<<P.ntiles, LBM_TILE, 0, st>>>(P, F, cur, fcur, k);
}

void launch_init_feq(cudaStream_t st, const LevelView &P, const float *feq9, float U, float chi_inf)
{
    Feq9 e;
    for (int q = 0; q < 9; q++) e.g[q] = feq9[q];
    k_init<<<P.ntiles, LBM_TILE, 0, st>>>(P, e, U, chi_inf);
}

void launch_loads(cudaStream_t st, const LoadsView &S, const RecView &R, float U, double *acc4)
{
    if (S.nseg <= 0) return;
    k_loads<<<(S.nseg + 255) / 256, 256, 0, st>>>(S, R, U, acc4);
}

void launch_mass(cudaStream_t st, const LevelView &P, double area, double *acc, int *status)
{
    k_mass<<<P.ntiles, LBM_TILE, 0, st>>>(P, area, acc, status);
}

}  // namespace lbmdev
