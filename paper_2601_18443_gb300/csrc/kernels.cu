// kernels.cu -- sm_103a kernels of one LBM-RANS level step.
//
// Populations are stored shifted, g_q = f_q - w_q, in FP32 structure-of-arrays per
// level tile set; every kernel works on one 32 x 8 tile per block, one cell per
// thread.  The collision is the central-moment operator of eqs 5-7 evaluated in
// closed form on the shifted raw moments (rest-state moments subtracted
// analytically), so that FP32 keeps the small departures from rest exact to
// ~1e-7 relative.  No step is a dense contraction; the kernels are bound by
// memory bandwidth (HBM, or L2 where a level stays resident across sub-steps).
//
// One launch of k_level advances every active cell of a level by one level step:
// wall function of its boundary node (finest level, Sec 2.3 steps 1-5), SA-neg
// update of chi (Sec 2.2), pull streaming with coalescence from the finer level and
// Yu's slip bounce-back on cut links (eq 27), central-moment collision relaxing with
// nu + nu_t, explosion into the finer level's ghosts, and -- on the second sub-step
// of a level -- the restriction of the new fields into the covered parents.  Fields
// of time t are read from buffer [p] and those of t + 1 written to [p ^ 1], so that
// no cell reads a value another block of the same launch writes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "device.cuh"

namespace lbmdev {

// ------------------------------------------------------------------ lattice (eq 2)
__host__ __device__ constexpr int cxq(int q) { return q == 1 || q == 5 || q == 7 ? 1 : (q == 2 || q == 6 || q == 8 ? -1 : 0); }
__host__ __device__ constexpr int cyq(int q) { return q == 3 || q == 5 || q == 8 ? 1 : (q == 4 || q == 6 || q == 7 ? -1 : 0); }
__host__ __device__ constexpr int oppq(int q) { return q == 0 ? 0 : (q & 1 ? q + 1 : q - 1); }
__host__ __device__ constexpr float wq(int q) { return q == 0 ? 4.f / 9.f : (q < 5 ? 1.f / 9.f : 1.f / 36.f); }
// direction with the same c_x and the opposite c_y (specular reflection on a horizontal plane)
__host__ __device__ constexpr int mirror_y(int q)
{
    return q == 3 ? 4 : q == 4 ? 3 : q == 5 ? 7 : q == 7 ? 5 : q == 6 ? 8 : q == 8 ? 6 : q;
}
// D2Q9 index of the offset (sx, sy) stored at position (sy + 1) * 3 + (sx + 1)
__host__ __device__ constexpr int dir_of3(int m)
{
    return m == 4 ? 0 : m == 5 ? 1 : m == 3 ? 2 : m == 7 ? 3 : m == 1 ? 4 : m == 8 ? 5 : m == 0 ? 6 : m == 2 ? 7 : 8;
}

// The 3 x 3 block of tiles around the block's tile, staged in shared memory.
__device__ __forceinline__ void load_nb3(const LevelView &P, int t, int *nb3)
{
    if (threadIdx.x < 9) nb3[threadIdx.x] = P.nbr[t * 9 + dir_of3(threadIdx.x)];
}

// Thread -> cell map of the level kernel (the work shape of a warp).  Shape 0: warp w
// covers the 16 x 2 cells x in [16 (w & 1), +16), y in {2 (w >> 1), +1}, so that every 2 x 2
// group of children lies inside one warp (the restriction is a warp shuffle) and a warp
// reads two 64-byte row segments per plane.  Shape 1: warp w covers row w, one 128-byte
// segment per plane, so that an access shifted by one cell touches 5 sectors instead of 6;
// its 2 x 2 groups span two warps and the restriction goes through shared memory.
__device__ __forceinline__ void cell_of_thread(int c, int &lx, int &ly, int shape)
{
    const int w = c >> 5, lane = c & 31;
    if (shape) {
        lx = lane;
        ly = w;
    } else {
        lx = (w & 1) * 16 + (lane & 15);
        ly = (w >> 1) * 2 + (lane >> 4);
    }
}

// slot of the cell at offset (dx, dy) from (lx, ly), or -1 if its tile is absent
__device__ __forceinline__ int nb_slot(const int *nb3, int lx, int ly, int dx, int dy)
{
    const int nx = lx + dx, ny = ly + dy;
    const int sx = nx < 0 ? 0 : (nx >= LBM_TX ? 2 : 1);
    const int sy = ny < 0 ? 0 : (ny >= LBM_TY ? 2 : 1);
    const int tt = nb3[sy * 3 + sx];
    return tt < 0 ? -1 : tt * LBM_TILE + (ny & (LBM_TY - 1)) * LBM_TX + (nx & (LBM_TX - 1));
}

// The slots of the eight D2Q9 neighbours at offsets +c_q (q = 1..8) and the own slot
// (q = 0); a neighbour in an absent tile maps to the own slot and clears bit q of the
// returned presence mask.  The SA stencil reads offset +c_q, the pull of direction q
// reads offset -c_q = +c_opp(q).
__device__ __forceinline__ unsigned neighbours(const int *nb3, int lx, int ly, int slot, int nbs[9])
{
    const int xm = lx - 1, xp = lx + 1, ym = ly - 1, yp = ly + 1;
    const int cm = xm < 0 ? 0 : 1, cp = xp >= LBM_TX ? 2 : 1;              // tile column of x -/+ 1
    const int rm = ym < 0 ? 0 : 3, rp = yp >= LBM_TY ? 6 : 3;              // tile row (x 3) of y -/+ 1
    const int colm = xm & (LBM_TX - 1), colp = xp & (LBM_TX - 1);
    const int rowm = (ym & (LBM_TY - 1)) * LBM_TX, rowp = (yp & (LBM_TY - 1)) * LBM_TX, row0 = ly * LBM_TX;
    const int tl[9] = {0, nb3[3 + cp], nb3[3 + cm], nb3[rp + 1], nb3[rm + 1], nb3[rp + cp], nb3[rm + cm],
                       nb3[rm + cp], nb3[rp + cm]};
    const int off[9] = {0, row0 + colp, row0 + colm, rowp + lx, rowm + lx, rowp + colp, rowm + colm, rowm + colp,
                        rowp + colm};
    unsigned present = 1u;
    nbs[0] = slot;
#pragma unroll
    for (int q = 1; q < 9; q++) {
        const bool ok = tl[q] >= 0;
        nbs[q] = ok ? tl[q] * LBM_TILE + off[q] : slot;
        present |= ok ? (1u << q) : 0u;
    }
    return present;
}

// level 0 covers its whole box with tiles in row-major order
__device__ __forceinline__ int slot0(const StepConsts &k, int i, int j)
{
    return ((j >> 3) * k.ntx0 + (i >> 5)) * LBM_TILE + (j & 7) * LBM_TX + (i & 31);
}

// the tile of level l+1 holding the four children of (lx, ly) and their first slot
__device__ __forceinline__ int child_base(const LevelView &P, int t, int lx, int ly)
{
    const int ct = P.child[t * 4 + ((2 * ly) >> 3) * 2 + ((2 * lx) >> 5)];
    return ct < 0 ? -1 : ct * LBM_TILE + ((2 * ly) & 7) * LBM_TX + ((2 * lx) & 31);
}

// ------------------------------------------------------------------ population storage
// Populations are stored shifted (f - w) in FP32, FP16 or BF16; every load converts to
// FP32 and every store rounds to nearest, so the arithmetic is FP32 in all three forms.
template <typename T> struct PopIO;
template <> struct PopIO<float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float ldp(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct PopIO<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float ldp(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct PopIO<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float ldp(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// ------------------------------------------------------------------ programmatic dependent launch
// The level-step kernels are launched with programmatic stream serialization: the next
// kernel's blocks may be scheduled while this one drains.  Each kernel reads only the
// static tile tables before griddep_wait(), which returns once the preceding kernel has
// completed and its writes are visible; griddep_launch() lets the next kernel start
// being scheduled as soon as every block of this one has begun.
__device__ __forceinline__ void griddep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void griddep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------ launch timeline
// With a timeline buffer (lbm_set_timeline), thread 0 of each block records the global
// timer (ns) at the block's entry, once its wait for the preceding kernel has returned, and
// once all its threads are done, at tl[3 (base + block) + 0, 1, 2].  Without one (tl null,
// a kernel parameter, so every branch here is uniform) nothing is read or written.
__device__ __forceinline__ void tl_mark(unsigned long long *tl, int base, int m)
{
    if (tl != nullptr && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        tl[3ull * (unsigned)(base + (int)blockIdx.x) + (unsigned)m] = t;
    }
}

__device__ __forceinline__ void tl_end(unsigned long long *tl, int base)
{
    if (tl == nullptr) return;
    __syncthreads();
    tl_mark(tl, base, 2);
}

// ------------------------------------------------------------------ bounds-checked builds
// With LBM_BOUNDS_CHECK every index the level step follows from a table (the work lists,
// tile neighbours, children and parents, the aux word, the wall stencils) is checked
// against its buffer: one outside it sets LBM_STATUS_BOUNDS in the status word (when the
// caller has one) and is replaced by 0, so that the access stays inside the buffer and no
// lane leaves its warp early; the host then fails the next synchronising call.  The default
// build compiles none of it.
__device__ __forceinline__ int checked_index(int i, int n, int *status)
{
#ifdef LBM_BOUNDS_CHECK
    if (i < 0 || i >= n) {
        if (status) atomicOr(status, LBM_STATUS_BOUNDS);
        return 0;
    }
#else
    (void)n;
    (void)status;
#endif
    return i;
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
// populations.  drho, jx, jy: the conserved moments of eq 3 summed from g; ux, uy the
// velocity j / rho.  The conserved raw moments are taken from the sums themselves, so
// mass and momentum are conserved to the rounding of those sums whatever the rounding
// of u.  delta = 2 - omega_nu (omega_b = 1: the trace relaxes fully, Sec 2.1).
__device__ __forceinline__ void collide_cm(const float g[9], float drho, float jx, float jy, float ux, float uy,
                                           float delta, float o[9])
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
    const float M10 = jx, M01 = jy;
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

// 2 - omega for the effective viscosity nu + nu_t (eq 9 with the RANS substitution);
// the divisions use the fast reciprocal path (about 2 ulp)
__device__ __forceinline__ float delta_of(float nu, float chi, int turbulence)
{
    float nue = nu;
    if (turbulence) {
        const float c3 = chi * chi * chi;
        nue += fmaxf(chi, 0.0f) * nu * __fdividef(c3, c3 + SA_CV1_3);
    }
    return __fdividef(12.0f * nue, 1.0f + 6.0f * nue);
}

// ------------------------------------------------------------------ SA-neg (Sec 2.2)
struct Stencil {
    float chi[9], ux[9], uy[9];
};

__device__ __forceinline__ void gather(const int *nb3, const float *chi, const float *ux, const float *uy, int lx,
                                       int ly, int slot, Stencil &S)
{
#pragma unroll
    for (int q = 0; q < 9; q++) {
        int s = q == 0 ? slot : nb_slot(nb3, lx, ly, cxq(q), cyq(q));
        if (s < 0) s = slot;
        S.chi[q] = __ldg(chi + s); S.ux[q] = __ldg(ux + s); S.uy[q] = __ldg(uy + s);
    }
}

// level-0 box edge: neighbours across the top/bottom symmetry planes are mirror images
__device__ __forceinline__ void gather0(const float *chi, const float *ux, const float *uy, const StepConsts &k, int i,
                                        int j, Stencil &S)
{
#pragma unroll
    for (int q = 0; q < 9; q++) {
        int ii = i + cxq(q), jj = j + cyq(q);
        float sg = 1.0f;
        if (jj < 0) { jj = 0; sg = -1.0f; }
        if (jj >= k.ny0) { jj = k.ny0 - 1; sg = -1.0f; }
        if (ii < 0) ii = 0;
        if (ii >= k.nx0) ii = k.nx0 - 1;
        const int s = slot0(k, ii, jj);
        S.chi[q] = chi[s]; S.ux[q] = ux[s]; S.uy[q] = sg * uy[s];
    }
}

// LSQ gradient over the full D2Q9 neighbourhood: the normal matrix is 6 I, so the
// gradient is sum_k c_k (phi_k - phi_0) / 6 = sum_k c_k phi_k / 6 (sum_k c_k = 0)
__device__ __forceinline__ void lsq_grad(const float *v, float &gx, float &gy)
{
    gx = ((v[1] - v[2]) + (v[5] - v[6]) + (v[7] - v[8])) * (1.0f / 6.0f);
    gy = ((v[3] - v[4]) + (v[5] - v[6]) + (v[8] - v[7])) * (1.0f / 6.0f);
}

__device__ __forceinline__ float sa_diff_coef(float chi)
{   // (nu + nu_t~ f_n) / nu
    const float c3 = chi * chi * chi;
    const float fn = chi < 0.0f ? __fdividef(SA_CN1 + c3, SA_CN1 - c3) : 1.0f;
    return 1.0f + chi * fn;
}

// Euler step of eqs 12 / 16 written for chi = nu_t~ / nu (explicit, with the diagonal of the
// diffusion at the new time level), with Lax-Wendroff (conv = 0, Sec 2.2) or first-order
// upwind (conv = 1, Sec 3.3) convection;
// id2 = 1 / d^2 (wall distance d in level lattice units)
__device__ float sa_update(const Stencil &S, float id2, float nu, int conv)
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
    const float cv = conv == 1
                         ? -(u * (u > 0.0f ? x[0] - x[2] : x[1] - x[0]) + v * (v > 0.0f ? x[0] - x[4] : x[3] - x[0]))
                         : -(u * gx + v * gy) + 0.5f * (u * u * gxx + 2.0f * u * v * gxy + v * v * gyy);
    float Dc, De, Dw, Dn, Ds;
    if (fminf(fminf(x[0], x[1]), fminf(fminf(x[2], x[3]), x[4])) >= 0.0f) {
        // nu_t~ >= 0 on the whole stencil: f_n = 1
        Dc = 1.0f + x[0];
        De = 0.5f * (Dc + 1.0f + x[1]); Dw = 0.5f * (Dc + 1.0f + x[2]);
        Dn = 0.5f * (Dc + 1.0f + x[3]); Ds = 0.5f * (Dc + 1.0f + x[4]);
    } else {
        Dc = sa_diff_coef(x[0]);
        De = 0.5f * (Dc + sa_diff_coef(x[1])); Dw = 0.5f * (Dc + sa_diff_coef(x[2]));
        Dn = 0.5f * (Dc + sa_diff_coef(x[3])); Ds = 0.5f * (Dc + sa_diff_coef(x[4]));
    }
    const float div = De * (x[1] - x[0]) - Dw * (x[0] - x[2]) + Dn * (x[3] - x[0]) - Ds * (x[0] - x[4]);
    const float diff = nu * (div + SA_CB2 * (gx * gx + gy * gy)) * (1.0f / SA_SIGMA);
    const float chi = x[0];
    const float ikd2 = id2 * (1.0f / (SA_KAPPA * SA_KAPPA));      // 1 / (kappa d)^2
    float src;
    if (chi >= 0.0f) {
        const float c3 = chi * chi * chi;
        const float fv1 = __fdividef(c3, c3 + SA_CV1_3);
        const float fv2 = 1.0f - __fdividef(chi, 1.0f + chi * fv1);
        const float sbar = nu * chi * fv2 * ikd2;
        float st;
        if (sbar >= -SA_CV2 * vort) st = vort + sbar;
        else st = vort + __fdividef(vort * (SA_CV2 * SA_CV2 * vort + SA_CV3 * sbar), (SA_CV3 - 2.0f * SA_CV2) * vort - sbar);
        float r = SA_RLIM;
        if (st > 0.0f) r = fminf(__fdividef(nu * chi * ikd2, st), SA_RLIM);
        const float r2 = r * r, r6 = r2 * r2 * r2;
        const float gg = r + SA_CW2 * (r6 - r);
        const float g2 = gg * gg, g6 = g2 * g2 * g2;
        const float fw = gg * __powf(__fdividef(1.0f + SA_CW3_6, g6 + SA_CW3_6), 1.0f / 6.0f);
        src = SA_CB1 * st * chi - SA_CW1 * fw * nu * chi * chi * id2;
    } else {
        src = SA_CB1 * (1.0f - SA_CT3) * vort * chi + SA_CW1 * nu * chi * chi * id2;
    }
    // the diffusion's diagonal at the new time level (point-implicit): the explicit increment
    // divided by 1 + sum_f D_f / sigma; unconditionally stable diffusion, same steady states
    const float a = nu * (De + Dw + Dn + Ds) * (1.0f / SA_SIGMA);
    return chi + __fdividef(cv + src + diff, 1.0f + a);
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
{   // eq 22 on the continuous arctangent branch: with b > 0, atan2(b, x) = pi/2 - atan(x / b)
    const float z1 = (y + WF_A1) * (1.0f / WF_B1), z2 = (y + WF_A2) * (1.0f / WF_B2);
    const float t1 = (y + WF_A1) * (y + WF_A1) + WF_B1 * WF_B1;
    const float t2 = (y + WF_A2) * (y + WF_A2) + WF_B2 * WF_B2;
    return (WF_B - (WF_C3 + WF_C4) * 1.5707963267948966f) + WF_C1 * __logf(t1) - WF_C2 * __logf(t2) +
           WF_C3 * atanf(z1) + WF_C4 * atanf(z2);
}

__device__ __forceinline__ float wf_dudy(float y)
{   // eq 21
    float k3 = SA_KAPPA * y;
    k3 = k3 * k3 * k3;
    return __fdividef(SA_CV1_3 + k3, SA_CV1_3 + k3 * (1.0f + SA_KAPPA * y));
}

// Friction velocity from u_t at distance y (step 3): Newton on g(u) = u u+(u y / nu) - u_t,
// g' = u+ + y+ du+/dy+ > 0, started from the previous sub-step's value when there is one,
// else from the viscous-sublayer value (which lies left of the root, since u+ <= y+).
// y_nu = y / nu.  Every evaluation narrows a sign bracket; steps leaving it are replaced by
// bisection (or doubling while no right end is known).  The iteration stops after a Newton
// step (not a bisection) shorter than 3e-4 u: Newton's error after a step of relative size
// e is about (g'' u / 2 g') e^2, at most e^2 / 2 (the viscous sublayer; about 0.05 e^2 in
// the log layer), so the result is within 4.5e-8 relative of the root, below FP32
// resolution.  At most 24 evaluations.
__device__ float wf_utau(float ut, float y_nu, float guess)
{
    if (!(ut > 0.0f)) return 0.0f;
    float lo = 0.0f, hi = INFINITY;
    float u = guess > 0.0f ? guess : sqrtf(ut / y_nu);
    for (int it = 0; it < 24; it++) {
        const float yp = u * y_nu;
        const float up = wf_uplus(yp);
        const float gv = u * up - ut;
        if (gv > 0.0f) hi = u; else lo = u;
        const float gp = up + yp * wf_dudy(yp);
        float un = gp > 0.0f ? u - __fdividef(gv, gp) : -1.0f;
        const bool newton = un > lo && un < hi;
        if (!newton) un = isinf(hi) ? 2.0f * fmaxf(u, lo) : 0.5f * (lo + hi);
        const bool done = newton && fabsf(un - u) <= 3e-4f * un;
        u = un;
        if (done) break;
    }
    return u;
}

// Wall state of one boundary node from the macroscopic fields at time level p:
// steps 1-5 of Sec 2.3 (IDW density and LSQ velocity at R, tangential part, u_tau from
// eq 22, u_V, slip velocity of eq 28 along t) and the SA Dirichlet value (Sec 2.2).
// Returns rho_W - 1, u_W and chi_B.  The Newton iteration starts from the u_tau of the
// previous step; only the step (keep_start) stores its result as the next start, so that
// queries leave the trajectory unchanged, and only queries (!keep_start) write the
// record's state arrays.
__device__ void wall_record(const LevelView &P, int p, const RecView &R, const StepConsts &k, int r, bool keep_start,
                            float &drW, float &uWx, float &uWy, float &chiB, int *status = nullptr)
{
    const float *dr = P.drho[p], *ux = P.ux[p], *uy = P.uy[p];
    // step 1: rho_R and u_R as fixed weighted sums over the 16-entry stencil (unused
    // entries carry zero weight); all 48 loads are independent
    float drR = 0.f, uR = 0.f, vR = 0.f;
    const int4 *sl4 = reinterpret_cast<const int4 *>(R.st_slot + r * 16);      // 64-byte records
    const float4 *wr4 = reinterpret_cast<const float4 *>(R.st_wr + r * 16);
    const float4 *wu4 = reinterpret_cast<const float4 *>(R.st_wu + r * 16);
#pragma unroll
    for (int m4 = 0; m4 < 4; m4++) {
        const int4 sv = __ldg(sl4 + m4);
        const float4 wrv = __ldg(wr4 + m4), wuv = __ldg(wu4 + m4);
        const int sa[4] = {sv.x, sv.y, sv.z, sv.w};
        const float ra[4] = {wrv.x, wrv.y, wrv.z, wrv.w}, ua[4] = {wuv.x, wuv.y, wuv.z, wuv.w};
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const int s = checked_index(sa[m], P.ns, status);
            drR += ra[m] * dr[s]; uR += ua[m] * ux[s]; vR += ua[m] * uy[s];
        }
    }
    const float nx = R.nx[r], ny = R.ny[r];
    const float un = uR * nx + vR * ny;
    const float utx = uR - un * nx, uty = vR - un * ny;
    const float ut = sqrtf(utx * utx + uty * uty);
    float tx = -ny, ty = nx;
    if (ut > 0.0f) { const float iut = 1.0f / ut; tx = utx * iut; ty = uty * iut; }
    float utau = 0.f;
    uWx = 0.f; uWy = 0.f; chiB = 0.f;
    if (k.wall_model == 0) {
        const float inu = 1.0f / P.nu;
        utau = wf_utau(ut, k.d_wr * inu, R.utau_start[r]);                  // step 3
        if (keep_start) R.utau_start[r] = utau;
        const float ypv = utau * k.d_wv * inu;
        const float uV = utau * wf_uplus(ypv);                              // step 4
        const float uW = uV - __fdividef(utau * utau * k.d_wv * inu, 1.0f + SA_KAPPA * ypv);   // eq 28
        uWx = uW * tx; uWy = uW * ty;                                       // step 5
        chiB = SA_KAPPA * utau * R.dwb[r] * inu;
    } else if (k.wall_model == 1) {
        // Nishimura's slip adapted to RANS (Sec 3.1.5, eq 31): u_tau from eq 22 at R and the
        // slip extrapolated linearly from R with the SA log-layer eddy viscosity
        // (nu_t)_R = nu kappa y+_R (eq 20)
        const float inu = 1.0f / P.nu;
        utau = wf_utau(ut, k.d_wr * inu, R.utau_start[r]);
        if (keep_start) R.utau_start[r] = utau;
        const float ypr = utau * k.d_wr * inu;
        const float uW = ut - __fdividef(utau * utau * k.d_wr * inu, 1.0f + SA_KAPPA * ypr);
        uWx = uW * tx; uWy = uW * ty;
        chiB = SA_KAPPA * utau * R.dwb[r] * inu;
    } else if (k.wall_model == 2) {
        uWx = R.slip[2 * R.loop[r]]; uWy = R.slip[2 * R.loop[r] + 1];
    }
    drW = drR;
    if (!keep_start) {
        // the query form fills the record's state arrays (lbm_get_loads, lbm_get_wall_state
        // run it first); the step only needs the returned values
        R.drhoW[r] = drR; R.uWx[r] = uWx; R.uWy[r] = uWy; R.utau[r] = utau; R.chiB[r] = chiB;
        R.tx[r] = tx; R.ty[r] = ty; R.ut[r] = ut;
    }
}

// ------------------------------------------------------------------ the fused level step
// Population layout (one lattice per level, updated in place; the "AA pattern").  With
// d the storage direction of a slot and q the population it holds:
//   before an even step (p = 0) slot (x, q) holds the population f_q arriving at x,
//   before an odd step  (p = 1) slot (x, opp q) holds the post-collision f*_q of x.
// An even step reads its cell's own nine slots and writes f*_q to (x, opp q).  An odd
// step reads f*_q of the upstream cell from (x - c_q, opp q) and writes its own f*_q to
// (x + c_q, q), the slot the downstream cell reads in the next even step.  In either
// step each slot is read and then written by one thread only (its own cell in an even
// step, the cell x - c_q of slot (x, q) in an odd step), so one lattice suffices.
// Levels l >= 1 take their two sub-steps of a parent step as an even and an odd step;
// level 0 alternates from coarse step to coarse step.
//
// Values that a step needs but that another thread's slot holds are kept in small side
// buffers written by the cell that owns them:
//   - a boundary node's last post-collision populations (R.fpost), for eq 27;
//   - the outlet columns' post-collision populations entering from x = N (k.obuf);
//   - a band cell's last post-collision populations (ebuf: the explosion), which its ghost
//     children keep where their upstream cell is not fluid;
//   - the populations each ghost child pulled in the fine level's odd sub-step (gbuf), which
//     the band cell averages (the coalescence).
// 16-bit storage keeps populations relative to the free-stream equilibrium, so that in
// most of the domain the stored values are small and their relative rounding is small in
// absolute terms; FP32 storage keeps g = f - w itself.  The shift belongs to the population
// (q), not to the slot direction (d).
// Slot (d, s) is element d * ns + s: a 32-bit index, since the host keeps 9 ns below 2^31.
template <typename T> struct Lat {
    T *f;
    int ns;
    const float *sh;
    __device__ __forceinline__ float ld(int d, int s, int q) const
    {
        if constexpr (std::is_same<T, float>::value) return PopIO<T>::ld(f + (d * ns + s));
        else return PopIO<T>::ld(f + (d * ns + s)) + sh[q];
    }
    __device__ __forceinline__ void st(int d, int s, int q, float v) const
    {
        if constexpr (std::is_same<T, float>::value) PopIO<T>::st(f + (d * ns + s), v);
        else PopIO<T>::st(f + (d * ns + s), v - sh[q]);
    }
};

// outlet buffer index of direction 2, 6 or 8
__device__ __forceinline__ int obuf_m(int q) { return q == 2 ? 0 : (q == 6 ? 1 : 2); }

// Post-collision populations o of an active fluid cell into the layout the next step of
// the level reads: an even step (ODD false) keeps them in the cell's own slots, an odd
// step sends each to the downstream cell, with the level-0 box edges (specular reflection
// at the symmetry planes, nothing across the inlet and the outlet).  nbs / present: slots
// at offsets +c_q and the mask of the present ones.  Boundary nodes, outlet columns and
// band cells also fill their side buffers (the explosion is done by the caller).
template <typename T, bool ODD>
__device__ __forceinline__ void put_post(const Lat<T> &F, const StepConsts &k, int slot, const int nbs[9],
                                         unsigned present, bool edge, int gi, int gj, const float o[9])
{
    if (!ODD) {
#pragma unroll
        for (int q = 0; q < 9; q++) F.st(oppq(q), slot, q, o[q]);
    } else if (!edge) {
        F.st(0, slot, 0, o[0]);
#pragma unroll
        for (int q = 1; q < 9; q++)
            if (present >> q & 1) F.st(q, nbs[q], q, o[q]);
    } else {
        F.st(0, slot, 0, o[0]);
#pragma unroll
        for (int q = 1; q < 9; q++) {
            const int di = gi + cxq(q), dj = gj + cyq(q);
            if (di < 0 || di >= k.nx0) continue;                       // across the inlet or the outlet
            if (dj >= 0 && dj < k.ny0) F.st(q, slot0(k, di, dj), q, o[q]);
            else F.st(mirror_y(q), slot0(k, di, gj), mirror_y(q), o[q]);  // reflected at the plane
        }
    }
}

// Outlet side buffer (parity par): the populations 2, 6, 8 of the outlet columns N-1 and N-2
// (flags FL_OUTLET, FL_OUTLET2) at row gj.
__device__ __forceinline__ void put_obuf(const StepConsts &k, int par, uint32_t fl, int gj, const float o[9])
{
    float *ob = k.obuf + par * (6 * k.ny0) + ((fl & FL_OUTLET) ? 0 : 3 * k.ny0);
    ob[gj] = o[2]; ob[k.ny0 + gj] = o[6]; ob[2 * k.ny0 + gj] = o[8];
}

// Explosion (Rohde, Sec 2.1) of band cell (t, lx, ly) with post-collision populations o: they
// become those of its four ghost children, written where the fine level's next even sub-step
// reads them (slot (g + c_q, q) for child g).  Children that are solid or have no tile relay
// nothing, so their share of the next coalescence is this value too.
template <typename T>
__device__ __forceinline__ void explode_band(const LevelView &P, const LevelView &F, const StepConsts &k, int t, int lx,
                                             int ly, uint32_t fl, int b, const float o[9], int *ls_status = nullptr)
{
    b = checked_index(b, P.n_band, ls_status);
    float *eb = P.ebuf + b * 9;
#pragma unroll
    for (int q = 0; q < 9; q++) eb[q] = o[q];
    const uint32_t sch = fl >> FL_SCH_SHIFT;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        if (sch >> m & 1) {
            float *gb = P.gbuf + (4 * b + m) * 9;
#pragma unroll
            for (int q = 0; q < 9; q++) gb[q] = o[q];
        }
    }
    int ct = P.child[t * 4 + ((2 * ly) >> 3) * 2 + ((2 * lx) >> 5)];
    if (ct < 0) return;
    ct = checked_index(ct, F.ntiles, ls_status);
    const Lat<T> LF{static_cast<T *>(F.f), F.ns, k.pshift};
    const int cx0 = (2 * lx) & (LBM_TX - 1), cy0 = (2 * ly) & (LBM_TY - 1);
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int ax = cx0 + (m & 1), ay = cy0 + (m >> 1);
#pragma unroll
        for (int q = 0; q < 9; q++) {
            const int nx = ax + cxq(q), ny = ay + cyq(q);
            const int sx = nx < 0 ? 0 : (nx >= LBM_TX ? 2 : 1), sy = ny < 0 ? 0 : (ny >= LBM_TY ? 2 : 1);
            const int tt = (sx == 1 && sy == 1) ? ct : __ldg(F.nbr + ct * 9 + dir_of3(sy * 3 + sx));
            if (tt >= 0)
                LF.st(q, checked_index(tt, F.ntiles, ls_status) * LBM_TILE + (ny & (LBM_TY - 1)) * LBM_TX + (nx & (LBM_TX - 1)),
                      q, o[q]);
        }
    }
}

// Whether a cell's aux word is used by the level step: ghosts, boundary nodes, band cells
// and coalescing cells.
__device__ __forceinline__ bool uses_aux(uint32_t fl)
{
    return (fl & FL_KIND_MASK) == KIND_GHOST || (fl & (FL_BNODE | FL_BAND | (0xFFu << FL_COAL_SHIFT)));
}

// One tile of the fused level step (the body of k_level): every thread updates its cell
// of tile t.  nb3 holds the 3 x 3 neighbour tiles of t for this warp.  The cell's flag
// word and aux word are read here, or passed in (FL_GIVEN) when the caller has fetched
// them ahead (the aux word only where uses_aux holds).
template <bool WALL, bool CHILD, typename T, bool ODD, bool FL_GIVEN>
__device__ __forceinline__ void level_tile(const LevelView &P, const LevelView &F, const LevelView &C, const RecView &R,
                                           const StepConsts &k, const LevelStep &ls, const Lat<T> &L, int t, int lane,
                                           int lx, int ly, const int *nb3, uint32_t fl_given, int ax_given, float *red)
{
    const int slot = t * LBM_TILE + ly * LBM_TX + lx;
    const uint32_t fl = FL_GIVEN ? fl_given : __ldg(P.flags + slot);
    auto aux_of = [&]() { return FL_GIVEN ? ax_given : __ldg(P.aux + slot); };
    const uint32_t kind = fl & FL_KIND_MASK;
    const bool fluid = !(fl & FL_SOLID);
    const int p = ls.p;
    bool valid = false;
    float n_dr = 0.f, n_ux = 0.f, n_uy = 0.f, n_chi = 0.f;

    if (kind == KIND_GHOST && fluid) {
        // ghosts are streamed (relayed), never collided.  Even sub-step: the arriving
        // populations stay in the cell, moved to the slots an odd step reads; odd sub-step:
        // the pulled populations go to the parent's coalescence buffer.  Where the upstream
        // cell is not fluid the ghost keeps its own value, the parent's exploded one.
        const int ax = checked_index(aux_of(), 4 * C.n_band, ls.status);
        const float *eb = C.ebuf + (ax >> 2) * 9;
        const uint32_t keep = fl >> FL_KEEP_SHIFT;
        if (!ODD) {
            float v[9];
            v[0] = L.ld(0, slot, 0);
#pragma unroll
            for (int q = 1; q < 9; q++) v[q] = (keep >> (q - 1) & 1) ? eb[q] : L.ld(q, slot, q);
#pragma unroll
            for (int q = 0; q < 9; q++) L.st(oppq(q), slot, q, v[q]);
        } else {
            float *gb = C.gbuf + ax * 9;
            gb[0] = L.ld(0, slot, 0);
#pragma unroll
            for (int q = 1; q < 9; q++) {
                int s = nb_slot(nb3, lx, ly, -cxq(q), -cyq(q));          // -1: no upstream tile
                if (s >= 0) s = checked_index(s, P.ns, ls.status);
                gb[q] = (keep >> (q - 1) & 1) || s < 0 ? eb[q] : L.ld(oppq(q), s, q);
            }
        }
    } else if (kind == KIND_ACTIVE && fluid) {
        const bool edge = ls.is_level0 && k.level0_edges && (fl & (FL_INLET | FL_OUTLET | FL_BOTTOM | FL_TOP));
        const bool bnode = WALL && (fl & FL_BNODE);
        int nbs[9];
        const unsigned present = neighbours(nb3, lx, ly, slot, nbs);
#ifdef LBM_BOUNDS_CHECK
#pragma unroll
        for (int q = 1; q < 9; q++) nbs[q] = checked_index(nbs[q], P.ns, ls.status);
#endif
        int gi = 0, gj = 0;
        if (edge) { gi = P.tile_x[t] * LBM_TX + lx; gj = P.tile_y[t] * LBM_TY + ly; }
        // ---- wall function of the boundary node (Sec 2.3), fields at time t
        float drW = 0.f, uWx = 0.f, uWy = 0.f, chiB = 0.f;
        int r = -1;
        if (bnode) {
            r = checked_index(aux_of(), R.n, ls.status);
            wall_record(P, p, R, k, r, true, drW, uWx, uWy, chiB, ls.status);
        }
        // ---- SA-neg update of chi (Sec 2.2), fields at time t
        float chin;
        if (k.turbulence) {
            if (bnode) {
                chin = chiB;                                        // Dirichlet nu_t~_B (Sec 2.2)
            } else if (edge) {
                if (fl & FL_INLET) {
                    chin = k.chi_inf;
                } else {
                    const int ic = (fl & FL_OUTLET) ? k.nx0 - 2 : gi;     // outlet: copy of its neighbour
                    Stencil S;
                    gather0(P.chi[p], P.ux[p], P.uy[p], k, ic, gj, S);
                    chin = sa_update(S, P.inv_d2[slot0(k, ic, gj)], P.nu, k.sa_convection);
                }
            } else {
                Stencil S;
                const float *xc = P.chi[p], *xu = P.ux[p], *xv = P.uy[p];
#pragma unroll
                for (int q = 0; q < 9; q++) {
                    S.chi[q] = __ldg(xc + nbs[q]); S.ux[q] = __ldg(xu + nbs[q]); S.uy[q] = __ldg(xv + nbs[q]);
                }
                chin = sa_update(S, __ldg(P.inv_d2 + slot), P.nu, k.sa_convection);
            }
            P.chi[p ^ 1][slot] = chin;
        } else {
            chin = __ldg(P.chi[p] + slot);
        }
        // ---- streaming (eq 1): the populations arriving at the cell
        float g[9];
        g[0] = L.ld(0, slot, 0);
        if (!ODD) {
#pragma unroll
            for (int q = 1; q < 9; q++) g[q] = L.ld(q, slot, q);
        } else if (!edge) {
#pragma unroll
            for (int q = 1; q < 9; q++) g[q] = L.ld(oppq(q), nbs[oppq(q)], q);
        } else {
            // level-0 box edge: in-box pulls and the symmetry planes' reflections
#pragma unroll
            for (int q = 1; q < 9; q++) {
                const int si = gi - cxq(q), sj = gj - cyq(q);
                const bool xin = si >= 0 && si < k.nx0, yin = sj >= 0 && sj < k.ny0;
                if (xin && yin) g[q] = L.ld(oppq(q), slot0(k, si, sj), q);
                else if (xin) g[q] = L.ld(oppq(mirror_y(q)), slot0(k, si, gj), mirror_y(q));
                else g[q] = 0.0f;
            }
        }
        const uint32_t special = fl & (0xFFu << FL_COAL_SHIFT | 0xFFu << FL_CUT_SHIFT);
        if (CHILD && (fl & (0xFFu << FL_COAL_SHIFT))) {
            // coalescence: mean of what the four ghost children pulled in the fine level's odd sub-step
            const float *gb = P.gbuf + checked_index(aux_of(), P.n_band, ls.status) * 36;
#pragma unroll
            for (int q = 1; q < 9; q++)
                if (fl & (1u << (FL_COAL_SHIFT + q - 1)))
                    g[q] = 0.25f * (gb[q] + gb[9 + q] + gb[18 + q] + gb[27 + q]);
        }
        if (WALL && bnode && special) {
            // Yu's interpolated bounce-back with the slip velocity of the wall record (eq 27): the
            // next fluid node's f*_qo arrives at B as its own f_qo; f*_q(B) and f*_qo(B) of the last
            // step come from the record's buffer
            const float *fp = R.fpost + r * 9;
            const uint32_t nf = __ldg(R.nfluid + r);      // bit q: the node B + c_q is active fluid
            float gin[9];
#pragma unroll
            for (int q = 0; q < 9; q++) gin[q] = g[q];
#pragma unroll
            for (int q = 1; q < 9; q++) {
                if (!(fl & (1u << (FL_CUT_SHIFT + q - 1)))) continue;
                const int qo = oppq(q);
                const float qf = R.q[r * 9 + q];
                const float mom = 6.0f * wq(q) * (1.0f + drW) * (cxq(q) * uWx + cyq(q) * uWy);
                if (nf >> q & 1) {
                    const float2 c = __ldg(reinterpret_cast<const float2 *>(R.yc) + r * 9 + q);   // 1/(1+q), q/(1+q)
                    g[q] = ((1.0f - qf) * gin[qo] + qf * fp[qo] + mom) * c.x + c.y * fp[q];
                }
                else g[q] = fp[qo] + mom;                               // half-way form, eq 24
            }
        }
        if (edge) {
            if (gi == 0) {
                // Zou-He velocity inlet (Sec 3.1.1)
                const float U = k.U;
                const float S = g[0] + g[3] + g[4] + 2.0f * (g[2] + g[6] + g[8]);   // sum of w over these is 1
                const float rho = (1.0f + S) / (1.0f - U);
                g[1] = g[2] + (2.0f / 3.0f) * rho * U;
                g[5] = g[6] - 0.5f * (g[3] - g[4]) + rho * U * (1.0f / 6.0f);
                g[7] = g[8] + 0.5f * (g[3] - g[4]) + rho * U * (1.0f / 6.0f);
            }
            if (gi == k.nx0 - 1) {
                // outlet, for the directions 2, 6, 8 entering from outside, on the post-stream
                // values of the columns N-2 and N-3 (the post-collision values of the columns
                // N-1 and N-2 one row up or down, or reflected at a symmetry plane):
                // Yu's linear extrapolation 2 g_q(N-2) - g_q(N-3), or the zero-gradient copy g_q(N-2)
                const float *ob = k.obuf + p * (6 * k.ny0);
#pragma unroll
                for (int m = 0; m < 3; m++) {
                    const int q = m == 0 ? 2 : (m == 1 ? 6 : 8);
                    const int sj = gj - cyq(q);
                    const bool yin = sj >= 0 && sj < k.ny0;
                    const int ms = obuf_m(yin ? q : mirror_y(q)), js = yin ? sj : gj;
                    const float g2 = ob[ms * k.ny0 + js];
                    g[q] = k.outlet == 0 ? 2.0f * g2 - ob[(3 + ms) * k.ny0 + js] : g2;
                }
            }
        }
        // ---- macroscopic fields (eq 3) and central-moment collision (eqs 5-11)
        const float drho = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
        const float jx = g[1] - g[2] + g[5] - g[6] + g[7] - g[8];
        const float jy = g[3] - g[4] + g[5] - g[6] - g[7] + g[8];
        const float irho = __fdividef(1.0f, 1.0f + drho);
        const float ux = jx * irho, uy = jy * irho;
        P.drho[p ^ 1][slot] = drho; P.ux[p ^ 1][slot] = ux; P.uy[p ^ 1][slot] = uy;
        float o[9];
        collide_cm(g, drho, jx, jy, ux, uy, delta_of(P.nu, chin, k.turbulence), o);
        put_post<T, ODD>(L, k, slot, nbs, present, edge, gi, gj, o);
        if (bnode) {
            float *fp = R.fpost + r * 9;
#pragma unroll
            for (int q = 0; q < 9; q++) fp[q] = o[q];
        }
        if (ls.is_level0 && k.level0_edges && (fl & (FL_OUTLET | FL_OUTLET2)))
            put_obuf(k, p ^ 1, fl, P.tile_y[t] * LBM_TY + ly, o);
        if (CHILD && (fl & FL_BAND)) explode_band<T>(P, F, k, t, lx, ly, fl, aux_of(), o, ls.status);
        valid = true;
        n_dr = drho; n_ux = ux; n_uy = uy; n_chi = chin;
    }

    if (ls.restrict_up) {
        // restriction into the covered parents (their children are this level's active
        // cells): rho and chi are the means over the fluid children, u is mass-weighted
        // (Rohde transfers, Sec 2.1).  Sums in the order ((x, y) + (x+1, y)) + ((x, y+1) +
        // (x+1, y+1)) in both work shapes.
        const float rr = valid ? 1.0f + n_dr : 0.0f;
        float a0 = valid ? n_dr : 0.0f, a1 = rr, a2 = rr * n_ux, a3 = rr * n_uy, a4 = valid ? n_chi : 0.0f;
        float a5 = valid ? 1.0f : 0.0f;
        bool head;
        if (ls.shape == 0) {
            // a 2 x 2 group lies inside the warp, lanes l, l+1, l+16, l+17: sum over (l, l+1)
            // then over (l, l+16)
#pragma unroll
            for (int d = 1; d <= 16; d <<= 4) {
                a0 += __shfl_down_sync(0xffffffffu, a0, d); a1 += __shfl_down_sync(0xffffffffu, a1, d);
                a2 += __shfl_down_sync(0xffffffffu, a2, d); a3 += __shfl_down_sync(0xffffffffu, a3, d);
                a4 += __shfl_down_sync(0xffffffffu, a4, d); a5 += __shfl_down_sync(0xffffffffu, a5, d);
            }
            head = !(lane & 1) && lane < 16;
        } else {
            // rows ly and ly + 1 are two warps: pairs along x by shuffle, then the two rows
            // through shared memory behind a block barrier (this branch is block-uniform)
            a0 += __shfl_down_sync(0xffffffffu, a0, 1); a1 += __shfl_down_sync(0xffffffffu, a1, 1);
            a2 += __shfl_down_sync(0xffffffffu, a2, 1); a3 += __shfl_down_sync(0xffffffffu, a3, 1);
            a4 += __shfl_down_sync(0xffffffffu, a4, 1); a5 += __shfl_down_sync(0xffffffffu, a5, 1);
            float *rs = red + 6 * (ly * LBM_TX + lx);
            rs[0] = a0; rs[1] = a1; rs[2] = a2; rs[3] = a3; rs[4] = a4; rs[5] = a5;
            __syncthreads();
            const float *rn = red + 6 * (((ly + 1) & (LBM_TY - 1)) * LBM_TX + lx);
            a0 += rn[0]; a1 += rn[1]; a2 += rn[2]; a3 += rn[3]; a4 += rn[4]; a5 += rn[5];
            __syncthreads();
            head = !(lx & 1) && !(ly & 1);
        }
        if (head && kind == KIND_ACTIVE) {
#ifdef LBM_BOUNDS_CHECK
            const int pt = P.parent[t] < 0 ? -1 : checked_index(P.parent[t], C.ntiles, ls.status);
#else
            const int pt = P.parent[t];
#endif
            const int n = (int)a5;
            if (pt >= 0 && n > 0) {
                const int px = (P.tile_x[t] & 1) * (LBM_TX / 2) + (lx >> 1);
                const int py = (P.tile_y[t] & 1) * (LBM_TY / 2) + (ly >> 1);
                const int ps = pt * LBM_TILE + py * LBM_TX + px;
                const int q1 = ls.pp ^ 1;
                C.drho[q1][ps] = a0 / n; C.ux[q1][ps] = a2 / a1; C.uy[q1][ps] = a3 / a1;
                C.chi[q1][ps] = a4 / n;
            }
        }
    }
}

// MINB: minimum resident blocks per SM the register allocation must allow (5 or 6, that
// is at most 48 or 40 registers a thread).  PERSIST: the grid (2 x SMs x MINB blocks)
// strides over the level's work tiles instead of one block per tile.  Both are picked
// per level by the autotuner.  Every variant computes bit-identical results (larger
// budgets, 3 or 4 blocks, were measured to round differently and to run no faster, and
// are not offered).  ODD: the parity of the in-place population update.
template <bool WALL, bool CHILD, typename T, int MINB, bool PERSIST, bool ODD>
__global__ void __launch_bounds__(256, MINB) k_level(LevelView P, LevelView F, LevelView C, RecView R, StepConsts k,
                                                      LevelStep ls)
{
    const Lat<T> L{static_cast<T *>(P.f), P.ns, k.pshift};
    __shared__ int nb3w[LBM_TILE / 32][9];       // one copy per warp: no block-wide barrier
    extern __shared__ float red[];               // restriction sums of work shape 1 (dynamic:
                                                 // 6 floats a thread, launched with shape 1 only)
    const int c = threadIdx.x;
    const int lane = c & 31;
    int lx, ly;
    cell_of_thread(c, lx, ly, ls.shape);
    int *nb3 = nb3w[c >> 5];
    tl_mark(ls.tl, ls.tl_base, 0);
    if constexpr (!PERSIST) {
        const int t = checked_index(P.work_tiles[blockIdx.x], P.ntiles, ls.status);
        if (lane < 9) nb3[lane] = P.nbr[t * 9 + dir_of3(lane)];
        __syncwarp();
        griddep_launch();
        griddep_wait();
        tl_mark(ls.tl, ls.tl_base, 1);
        level_tile<WALL, CHILD, T, ODD, false>(P, F, C, R, k, ls, L, t, lane, lx, ly, nb3, 0u, 0, red);
    } else {
        // the grid tables are static: the first tile's neighbour table and flag word are
        // read before the wait, and each tile's flag word one tile ahead
        const int cell = ly * LBM_TX + lx;
        int wt = blockIdx.x;
        uint32_t fl_next = 0;
        if (wt < P.n_work_tiles) {
            const int t0 = checked_index(P.work_tiles[wt], P.ntiles, ls.status);
            if (lane < 9) nb3[lane] = P.nbr[t0 * 9 + dir_of3(lane)];
            fl_next = __ldg(P.flags + t0 * LBM_TILE + cell);
        }
        __syncwarp();
        griddep_launch();
        griddep_wait();
        tl_mark(ls.tl, ls.tl_base, 1);
        for (; wt < P.n_work_tiles; wt += gridDim.x) {
            const int t = checked_index(P.work_tiles[wt], P.ntiles, ls.status);
            const uint32_t fl = fl_next;
            if (wt + (int)gridDim.x < P.n_work_tiles)
                fl_next = __ldg(P.flags + checked_index(P.work_tiles[wt + gridDim.x], P.ntiles, ls.status) * LBM_TILE + cell);
            if (wt != (int)blockIdx.x) {
                __syncwarp();
                if (lane < 9) nb3[lane] = P.nbr[t * 9 + dir_of3(lane)];
                __syncwarp();
            }
            const int ax = uses_aux(fl) ? __ldg(P.aux + t * LBM_TILE + cell) : -1;
            level_tile<WALL, CHILD, T, ODD, true>(P, F, C, R, k, ls, L, t, lane, lx, ly, nb3, fl, ax, red);
        }
    }
    tl_end(ls.tl, ls.tl_base);

}

// Warp-list schedules of k_level: blocks of WPB warps (2 or 4), each warp taking one entry
// of the level's work-warp list (tile * 8 + its warp in work shape 0), so that the warps of
// a work tile holding no active or ghost fluid cell are not launched, and a block is retired
// (and replaced) as soon as its WPB warps are done rather than its tile's eight.  Smaller
// blocks balance better; larger ones ask less of the block dispatcher, which refills an SM
// at a bounded rate.  MINB keeps the register budget of k_level<.., MINB, ..>: 40 warps a
// SM fit 48 registers a thread, 48 fit 40 (a sub-partition's 16384 registers hold 10 warps
// of 48 or 12 of 40, whatever the block size).  Per cell it runs the same code as k_level
// with work shape 0.  (A persistent form, the resident blocks walking the list, measured
// 30 % slower on the finest level of the c/4096 workload: with every resident warp busy all
// the time each entry takes longer, so the throughput falls; it is not offered.)
template <bool WALL, bool CHILD, typename T, int MINB, int WPB, bool ODD>
__global__ void __launch_bounds__(WPB * 32, (MINB == 6 ? 48 : 40) / WPB)
    k_level_wl(LevelView P, LevelView F, LevelView C, RecView R, StepConsts k, LevelStep ls)
{
    const Lat<T> L{static_cast<T *>(P.f), P.ns, k.pshift};
    __shared__ int nb3w[WPB][9];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int w = blockIdx.x * WPB + wb;
    const bool have = w < P.n_work_warps;
    int *nb3 = nb3w[wb];
    int t = 0, lx = 0, ly = 0;
    tl_mark(ls.tl, ls.tl_base, 0);
    if (have) {
        const int e = __ldg(P.work_warps + w);
        t = checked_index(e >> 3, P.ntiles, ls.status);
        cell_of_thread((e & 7) * 32 + lane, lx, ly, 0);
        if (lane < 9) nb3[lane] = P.nbr[t * 9 + dir_of3(lane)];
    }
    __syncwarp();
    griddep_launch();
    griddep_wait();
    tl_mark(ls.tl, ls.tl_base, 1);
    LevelStep l0 = ls;
    l0.shape = 0;
    if (have) level_tile<WALL, CHILD, T, ODD, false>(P, F, C, R, k, l0, L, t, lane, lx, ly, nb3, 0u, 0, nullptr);
    tl_end(ls.tl, ls.tl_base);
}

// The batched form of k_level (one block per work tile, register budget of 5 blocks per SM):
// block b belongs to the last solve whose first block is at most b; its kind and the
// parity of its level select the body.  Per cell it runs the same code as k_level.
template <typename T>
__global__ void __launch_bounds__(256, 5) k_level_batch(const __grid_constant__ BatchArgs a)
{
    int i = 0;
    for (int m = 1; m < a.n; m++)
        if (a.d[m].first_block <= (int)blockIdx.x) i = m;
    const SolveDesc &d = a.d[i];
    __shared__ int nb3w[LBM_TILE / 32][9];
    float *red = nullptr;                        // batched launches use work shape 0
    const int c = threadIdx.x;
    const int lane = c & 31;
    int lx, ly;
    cell_of_thread(c, lx, ly, 0);
    int *nb3 = nb3w[c >> 5];
    const int t = checked_index(d.P.work_tiles[blockIdx.x - d.first_block], d.P.ntiles, d.ls.status);
    if (lane < 9) nb3[lane] = d.P.nbr[t * 9 + dir_of3(lane)];
    __syncwarp();
    griddep_launch();
    griddep_wait();
    const Lat<T> L{static_cast<T *>(d.P.f), d.P.ns, d.k.pshift};
    const bool odd = d.ls.p != 0;
    if (d.kind == 2) {
        if (odd) level_tile<true, false, T, true, false>(d.P, d.F, d.C, d.R, d.k, d.ls, L, t, lane, lx, ly, nb3, 0u, 0, red);
        else level_tile<true, false, T, false, false>(d.P, d.F, d.C, d.R, d.k, d.ls, L, t, lane, lx, ly, nb3, 0u, 0, red);
    } else if (d.kind == 1) {
        if (odd) level_tile<false, true, T, true, false>(d.P, d.F, d.C, d.R, d.k, d.ls, L, t, lane, lx, ly, nb3, 0u, 0, red);
        else level_tile<false, true, T, false, false>(d.P, d.F, d.C, d.R, d.k, d.ls, L, t, lane, lx, ly, nb3, 0u, 0, red);
    } else {
        if (odd) level_tile<false, false, T, true, false>(d.P, d.F, d.C, d.R, d.k, d.ls, L, t, lane, lx, ly, nb3, 0u, 0, red);
        else level_tile<false, false, T, false, false>(d.P, d.F, d.C, d.R, d.k, d.ls, L, t, lane, lx, ly, nb3, 0u, 0, red);
    }
}

// ------------------------------------------------------------------ prolongation (Sec 2.2)
// ghost children of the band cells of level l: linear LSQ reconstruction of chi and u
// about the parent (fields at time t), rho copied; written to both time levels of l+1
__device__ __forceinline__ void prolong_tile(const LevelView &P, const LevelView &F, int p, int t, int *nb3)
{
    const int c = threadIdx.x;
    const int lx = c & 31, ly = c >> 5;
    const int slot = t * LBM_TILE + c;
    const uint32_t fl = P.flags[slot];
    if ((fl & FL_KIND_MASK) != KIND_ACTIVE || (fl & FL_SOLID) || !(fl & FL_BAND)) return;
    const int cb = child_base(P, t, lx, ly);
    if (cb < 0) return;
    Stencil S;
    gather(nb3, P.chi[p], P.ux[p], P.uy[p], lx, ly, slot, S);
    float gcx, gcy, gux, guy, gvx, gvy;
    lsq_grad(S.chi, gcx, gcy); lsq_grad(S.ux, gux, guy); lsq_grad(S.uy, gvx, gvy);
    const float dr = P.drho[p][slot];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int a = m & 1, b = m >> 1;
        const float ox = 0.5f * (a - 0.5f), oy = 0.5f * (b - 0.5f);
        const int cs = cb + b * LBM_TX + a;
        const float vc = S.chi[0] + gcx * ox + gcy * oy;
        const float vu = S.ux[0] + gux * ox + guy * oy;
        const float vv = S.uy[0] + gvx * ox + gvy * oy;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            F.chi[h][cs] = vc; F.ux[h][cs] = vu; F.uy[h][cs] = vv; F.drho[h][cs] = dr;
        }
    }
}

__global__ void __launch_bounds__(256) k_prolong(LevelView P, LevelView F, int p, unsigned long long *tl, int tl_base)
{
    tl_mark(tl, tl_base, 0);
    __shared__ int nb3[9];
    const int t = P.band_tiles[blockIdx.x];
    load_nb3(P, t, nb3);
    __syncthreads();
    griddep_launch();
    griddep_wait();
    tl_mark(tl, tl_base, 1);
    prolong_tile(P, F, p, t, nb3);
    tl_end(tl, tl_base);
}

// batched form of k_prolong (same solve lookup as k_level_batch, over band tiles)
__global__ void __launch_bounds__(256) k_prolong_batch(const __grid_constant__ ProlongBatchArgs a)
{
    int i = 0;
    for (int m = 1; m < a.n; m++)
        if (a.d[m].first_block <= (int)blockIdx.x) i = m;
    const ProlongDesc &d = a.d[i];
    tl_mark(a.tl, a.tl_base, 0);
    __shared__ int nb3[9];
    const int t = d.P.band_tiles[blockIdx.x - d.first_block];
    load_nb3(d.P, t, nb3);
    __syncthreads();
    griddep_launch();
    griddep_wait();
    tl_mark(a.tl, a.tl_base, 1);
    prolong_tile(d.P, d.F, d.p, t, nb3);
    tl_end(a.tl, a.tl_base);
}

// ------------------------------------------------------------------ wall-state query
__global__ void __launch_bounds__(128) k_wallfn(LevelView P, int p, RecView R, StepConsts k)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R.n) return;
    float drW, uWx, uWy, chiB;
    wall_record(P, p, R, k, r, false, drW, uWx, uWy, chiB);
}

// ------------------------------------------------------------------ interface sync (set_fields)
__global__ void k_restrict(LevelView P, LevelView F, int pp, int pf)
{
    const int t = blockIdx.x, c = threadIdx.x;
    const int slot = t * LBM_TILE + c;
    const uint32_t fl = P.flags[slot];
    if ((fl & FL_KIND_MASK) != KIND_COVERED) return;
    const int cb = child_base(P, t, c & 31, c >> 5);
    if (cb < 0) return;
    float sdr = 0.f, sr = 0.f, sx = 0.f, sy = 0.f, sc = 0.f;
    int n = 0;
    for (int m = 0; m < 4; m++) {
        const int cs = cb + (m & 1) + (m >> 1) * LBM_TX;
        if (F.flags[cs] & FL_SOLID) continue;
        const float dr = F.drho[pf][cs], r = 1.0f + dr;
        sdr += dr; sr += r; sx += r * F.ux[pf][cs]; sy += r * F.uy[pf][cs]; sc += F.chi[pf][cs];
        n++;
    }
    if (n == 0) return;
    P.drho[pp][slot] = sdr / n; P.ux[pp][slot] = sx / sr; P.uy[pp][slot] = sy / sr;
    P.chi[pp][slot] = sc / n;
}

// Logical post-collision populations (f - w, unshifted) of the active fluid cells of a level
// whose next step has parity p, gathered from the in-place layout into out[q * ns + slot]:
// the inverse of put_post.  Values the layout does not keep (populations leaving across the
// inlet or the outlet, or towards a cell without a tile; no step reads them) are NaN.
// Boundary nodes come from their record buffer.  Ghosts report their parent's exploded
// values before an even sub-step and what they relay before an odd one.
template <typename T>
__global__ void k_gather_post(LevelView P, LevelView C, RecView R, StepConsts k, int p, int is_level0, float *out)
{
    __shared__ int nb3[9];
    const int t = blockIdx.x, c = threadIdx.x;
    const int lx = c & 31, ly = c >> 5;
    load_nb3(P, t, nb3);
    __syncthreads();
    const int slot = t * LBM_TILE + c;
    const Lat<T> L{static_cast<T *>(P.f), P.ns, k.pshift};
    const uint32_t fl = P.flags[slot];
    const uint32_t kind = fl & FL_KIND_MASK;
    float o[9];
    for (int q = 0; q < 9; q++) o[q] = NAN;
    if (kind == KIND_GHOST && !(fl & FL_SOLID)) {
        // before an odd sub-step a ghost holds what it relays next (its even sub-step's
        // pulls); before an even one, its parent's exploded values
        const float *eb = C.ebuf + (P.aux[slot] >> 2) * 9;
        for (int q = 0; q < 9; q++) o[q] = p == 1 ? L.ld(oppq(q), slot, q) : eb[q];
    } else if (kind == KIND_ACTIVE && !(fl & FL_SOLID)) {
        if (R.n > 0 && (fl & FL_BNODE) && P.aux) {
            const float *fp = R.fpost + P.aux[slot] * 9;
            for (int q = 0; q < 9; q++) o[q] = fp[q];
        } else if (p == 1) {
            for (int q = 0; q < 9; q++) o[q] = L.ld(oppq(q), slot, q);
        } else {
            int nbs[9];
            const unsigned present = neighbours(nb3, lx, ly, slot, nbs);
            o[0] = L.ld(0, slot, 0);
            const bool edge = is_level0 && k.level0_edges && (fl & (FL_INLET | FL_OUTLET | FL_BOTTOM | FL_TOP));
            const int gi = P.tile_x[t] * LBM_TX + lx, gj = P.tile_y[t] * LBM_TY + ly;
            for (int q = 1; q < 9; q++) {
                if (!edge) {
                    if (present >> q & 1) o[q] = L.ld(q, nbs[q], q);
                } else {
                    const int di = gi + cxq(q), dj = gj + cyq(q);
                    if (di < 0 || di >= k.nx0) continue;
                    if (dj >= 0 && dj < k.ny0) o[q] = L.ld(q, slot0(k, di, dj), q);
                    else o[q] = L.ld(mirror_y(q), slot0(k, di, gj), mirror_y(q));
                }
            }
        }
    }
    for (int q = 0; q < 9; q++) out[(size_t)q * P.ns + slot] = o[q];
}

// Store logical post-collision populations in[q * ns + slot] (f - w) of the active fluid
// cells of a level whose next step has parity p into the in-place layout, the record
// buffers of boundary nodes and the outlet buffer (put_post's writes).  Ghost slots are left
// to the explosion.
template <typename T>
__global__ void k_store_post(LevelView P, RecView R, StepConsts k, int p, int is_level0, const float *in)
{
    __shared__ int nb3[9];
    const int t = blockIdx.x, c = threadIdx.x;
    const int lx = c & 31, ly = c >> 5;
    load_nb3(P, t, nb3);
    __syncthreads();
    const int slot = t * LBM_TILE + c;
    const uint32_t fl = P.flags[slot];
    if ((fl & FL_KIND_MASK) != KIND_ACTIVE || (fl & FL_SOLID)) return;
    const Lat<T> L{static_cast<T *>(P.f), P.ns, k.pshift};
    float o[9];
    for (int q = 0; q < 9; q++) o[q] = in[(size_t)q * P.ns + slot];
    int nbs[9];
    const unsigned present = neighbours(nb3, lx, ly, slot, nbs);
    const bool edge = is_level0 && k.level0_edges && (fl & (FL_INLET | FL_OUTLET | FL_BOTTOM | FL_TOP));
    const int gi = P.tile_x[t] * LBM_TX + lx, gj = P.tile_y[t] * LBM_TY + ly;
    if (p == 0) put_post<T, true>(L, k, slot, nbs, present, edge, gi, gj, o);
    else put_post<T, false>(L, k, slot, nbs, present, edge, gi, gj, o);
    if (R.n > 0 && (fl & FL_BNODE) && P.aux) {
        float *fp = R.fpost + P.aux[slot] * 9;
        for (int q = 0; q < 9; q++) fp[q] = o[q];
    }
    if (is_level0 && k.level0_edges && (fl & (FL_OUTLET | FL_OUTLET2))) put_obuf(k, p, fl, gj, o);
}

// explosion of every band cell of P into the ghosts of F from logical post-collision
// populations post[q * ns + slot] of P
template <typename T>
__global__ void k_explode(LevelView P, LevelView F, StepConsts k, const float *post)
{
    const int t = blockIdx.x, c = threadIdx.x;
    const int lx = c & 31, ly = c >> 5;
    const int slot = t * LBM_TILE + c;
    const uint32_t fl = P.flags[slot];
    if ((fl & FL_KIND_MASK) != KIND_ACTIVE || (fl & FL_SOLID) || !(fl & FL_BAND)) return;
    float o[9];
    for (int q = 0; q < 9; q++) o[q] = post[(size_t)q * P.ns + slot];
    explode_band<T>(P, F, k, t, lx, ly, fl, __ldg(P.aux + slot), o);
}

// rest state: every present cell's populations are e (values to store, relative to the
// storage shift), its fields rho = 1, u = (U, 0), chi = chi_inf
struct Feq9 { float g[9]; };

template <typename T>
__global__ void k_init(LevelView P, Feq9 e, float U, float chi_inf)
{
    const int slot = blockIdx.x * LBM_TILE + threadIdx.x;
    const uint32_t fl = P.flags[slot];
    const bool present = (fl & FL_KIND_MASK) != KIND_ABSENT;
    for (int q = 0; q < 9; q++) PopIO<T>::st(static_cast<T *>(P.f) + (size_t)q * P.ns + slot, present ? e.g[q] : 0.0f);
    for (int h = 0; h < 2; h++) {
        P.drho[h][slot] = 0.0f;
        P.ux[h][slot] = present ? U : 0.0f;
        P.uy[h][slot] = 0.0f;
        P.chi[h][slot] = chi_inf;
    }
}

// n groups of nine values g (side buffers at rest)
__global__ void k_fill9(float *buf, long long n, Feq9 g)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 9 * n) buf[i] = g.g[i % 9];
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

__global__ void __launch_bounds__(256) k_mass(LevelView P, int p, double area, double *acc, int *status)
{
    __shared__ double red[8];
    const int slot = blockIdx.x * LBM_TILE + threadIdx.x;
    const uint32_t fl = P.flags[slot];
    double v = 0;
    if ((fl & FL_KIND_MASK) == KIND_ACTIVE && !(fl & FL_SOLID)) {
        const float dr = P.drho[p][slot], u = P.ux[p][slot], w = P.uy[p][slot], x = P.chi[p][slot];
        if (!(isfinite(dr) && isfinite(u) && isfinite(w) && isfinite(x))) atomicOr(status, 1);
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

// one record of the load history (lbm_set_load_history): the step and eq 30's coefficients
// from the loads' FP64 sums, formed as lbm_get_loads forms them, and the FP64 mass
__global__ void k_hist_push(const double *acc, double *ring, int slot, long long step, double chord)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double *r = ring + 6 * (size_t)slot;
        const double cdf = acc[0] / chord, cdp = acc[2] / chord;
        r[0] = (double)step;
        r[1] = acc[3] / chord;
        r[2] = cdf + cdp;
        r[3] = cdp;
        r[4] = cdf;
        r[5] = acc[4];
    }
}

void launch_hist_push(cudaStream_t st, const double *acc, double *ring, int slot, long long step, double chord)
{
    k_hist_push<<<1, 32, 0, st>>>(acc, ring, slot, step, chord);
}

// ------------------------------------------------------------------ launchers
// launch, with programmatic stream serialization when pdl is set (see griddep_wait)
template <typename... Args>
static void launch_pdl_bs(void (*kern)(Args...), unsigned grid, unsigned block, cudaStream_t st, int pdl, size_t smem,
                          Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename... Args>
static void launch_pdl_smem(void (*kern)(Args...), unsigned grid, cudaStream_t st, int pdl, size_t smem, Args... args)
{
    launch_pdl_bs(kern, grid, LBM_TILE, st, pdl, smem, args...);
}

template <typename... Args>
static void launch_pdl(void (*kern)(Args...), unsigned grid, cudaStream_t st, int pdl, Args... args)
{
    launch_pdl_smem(kern, grid, st, pdl, 0, args...);
}

// the level holding the wall records is the finest one, which has no child level
template <typename T, int MINB, bool PERSIST, bool ODD>
static void launch_level_mb(cudaStream_t st, const LevelView &P, const LevelView &Fv, const LevelView &Cv, bool child,
                            const RecView &R, const StepConsts &k, const LevelStep &ls, int pdl)
{
    // persistent: two rounds of the resident blocks stride over the work tiles
    const unsigned grid = PERSIST ? (unsigned)std::min(P.n_work_tiles, 2 * k.sms * MINB) : (unsigned)P.n_work_tiles;
    const size_t smem = ls.shape ? 6 * LBM_TILE * sizeof(float) : 0;
    if (ls.wall) launch_pdl_smem(k_level<true, false, T, MINB, PERSIST, ODD>, grid, st, pdl, smem, P, Fv, Cv, R, k, ls);
    else if (child) launch_pdl_smem(k_level<false, true, T, MINB, PERSIST, ODD>, grid, st, pdl, smem, P, Fv, Cv, R, k, ls);
    else launch_pdl_smem(k_level<false, false, T, MINB, PERSIST, ODD>, grid, st, pdl, smem, P, Fv, Cv, R, k, ls);
}

template <typename T, int MINB, int WPB, bool ODD>
static void launch_level_wl(cudaStream_t st, const LevelView &P, const LevelView &Fv, const LevelView &Cv, bool child,
                            const RecView &R, const StepConsts &k, const LevelStep &ls, int pdl)
{
    const unsigned grid = (unsigned)((P.n_work_warps + WPB - 1) / WPB);
    if (grid == 0) return;
    const unsigned bs = WPB * 32;
    if (ls.wall) launch_pdl_bs(k_level_wl<true, false, T, MINB, WPB, ODD>, grid, bs, st, pdl, 0, P, Fv, Cv, R, k, ls);
    else if (child) launch_pdl_bs(k_level_wl<false, true, T, MINB, WPB, ODD>, grid, bs, st, pdl, 0, P, Fv, Cv, R, k, ls);
    else launch_pdl_bs(k_level_wl<false, false, T, MINB, WPB, ODD>, grid, bs, st, pdl, 0, P, Fv, Cv, R, k, ls);
}

template <typename T, bool ODD>
static void launch_level_t(cudaStream_t st, const LevelView &P, const LevelView &Fv, const LevelView &Cv, bool child,
                           const RecView &R, const StepConsts &k, const LevelStep &ls, const LevelTune &tu)
{
    if (tu.min_blocks == 6) {
        if (tu.sched == LBM_SCHED_WARPS) launch_level_wl<T, 6, 2, ODD>(st, P, Fv, Cv, child, R, k, ls, tu.pdl);
        else if (tu.sched == LBM_SCHED_WARPS4) launch_level_wl<T, 6, 4, ODD>(st, P, Fv, Cv, child, R, k, ls, tu.pdl);
        else if (tu.sched == LBM_SCHED_PERSIST) launch_level_mb<T, 6, true, ODD>(st, P, Fv, Cv, child, R, k, ls, tu.pdl);
        else launch_level_mb<T, 6, false, ODD>(st, P, Fv, Cv, child, R, k, ls, tu.pdl);
    } else {
        if (tu.sched == LBM_SCHED_WARPS) launch_level_wl<T, 5, 2, ODD>(st, P, Fv, Cv, child, R, k, ls, tu.pdl);
        else if (tu.sched == LBM_SCHED_WARPS4) launch_level_wl<T, 5, 4, ODD>(st, P, Fv, Cv, child, R, k, ls, tu.pdl);
        else if (tu.sched == LBM_SCHED_PERSIST) launch_level_mb<T, 5, true, ODD>(st, P, Fv, Cv, child, R, k, ls, tu.pdl);
        else launch_level_mb<T, 5, false, ODD>(st, P, Fv, Cv, child, R, k, ls, tu.pdl);
    }
}

template <typename T>
static void launch_level_p(cudaStream_t st, const LevelView &P, const LevelView &Fv, const LevelView &Cv, bool child,
                           const RecView &R, const StepConsts &k, const LevelStep &ls, const LevelTune &tu)
{
    if (ls.p) launch_level_t<T, true>(st, P, Fv, Cv, child, R, k, ls, tu);
    else launch_level_t<T, false>(st, P, Fv, Cv, child, R, k, ls, tu);
}

void launch_level(cudaStream_t st, const LevelView &P, const LevelView *F, const LevelView *C, const RecView &R,
                  const StepConsts &k, const LevelStep &ls, const LevelTune &tu)
{
    const LevelView Fv = F ? *F : P, Cv = C ? *C : P;
    if (P.n_work_tiles <= 0) return;
    switch (P.store) {
    case 1: launch_level_p<__half>(st, P, Fv, Cv, F != nullptr, R, k, ls, tu); break;
    case 2: launch_level_p<__nv_bfloat16>(st, P, Fv, Cv, F != nullptr, R, k, ls, tu); break;
    default: launch_level_p<float>(st, P, Fv, Cv, F != nullptr, R, k, ls, tu); break;
    }
}

void launch_level_batch(cudaStream_t st, const BatchArgs &a, int store, unsigned grid, int pdl)
{
    if (grid == 0) return;
    switch (store) {
    case 1: launch_pdl(k_level_batch<__half>, grid, st, pdl, a); break;
    case 2: launch_pdl(k_level_batch<__nv_bfloat16>, grid, st, pdl, a); break;
    default: launch_pdl(k_level_batch<float>, grid, st, pdl, a); break;
    }
}

void launch_prolong_batch(cudaStream_t st, const ProlongBatchArgs &a, unsigned grid, int pdl)
{
    if (grid > 0) launch_pdl(k_prolong_batch, grid, st, pdl, a);
}

void launch_prolong(cudaStream_t st, const LevelView &P, const LevelView &F, int p, int pdl, unsigned long long *tl,
                    int tl_base)
{
    if (P.n_band_tiles > 0) launch_pdl(k_prolong, (unsigned)P.n_band_tiles, st, pdl, P, F, p, tl, tl_base);
}

void launch_wallfn(cudaStream_t st, const LevelView &P, int p, const RecView &R, const StepConsts &k)
{
    if (R.n <= 0) return;
    k_wallfn<<<(R.n + 127) / 128, 128, 0, st>>>(P, p, R, k);
}

void launch_restrict(cudaStream_t st, const LevelView &P, const LevelView &F, int pp, int pf)
{
    k_restrict<<<P.ntiles, LBM_TILE, 0, st>>>(P, F, pp, pf);
}

template <typename T>
static void launch_aa_util(int what, cudaStream_t st, const LevelView &P, const LevelView &Q, const RecView &R,
                           const StepConsts &k, int p, int is_level0, float *buf)
{
    if (what == 0) k_gather_post<T><<<P.ntiles, LBM_TILE, 0, st>>>(P, Q, R, k, p, is_level0, buf);
    else if (what == 1) k_store_post<T><<<P.ntiles, LBM_TILE, 0, st>>>(P, R, k, p, is_level0, buf);
    else k_explode<T><<<P.ntiles, LBM_TILE, 0, st>>>(P, Q, k, buf);
}

static void launch_aa(int what, cudaStream_t st, const LevelView &P, const LevelView &Q, const RecView &R,
                      const StepConsts &k, int p, int is_level0, float *buf)
{
    if (P.ntiles <= 0) return;
    switch (P.store) {
    case 1: launch_aa_util<__half>(what, st, P, Q, R, k, p, is_level0, buf); break;
    case 2: launch_aa_util<__nv_bfloat16>(what, st, P, Q, R, k, p, is_level0, buf); break;
    default: launch_aa_util<float>(what, st, P, Q, R, k, p, is_level0, buf); break;
    }
}

void launch_gather_post(cudaStream_t st, const LevelView &P, const LevelView *C, const RecView &R, const StepConsts &k,
                        int p, int is_level0, float *out)
{
    launch_aa(0, st, P, C ? *C : P, R, k, p, is_level0, out);
}

void launch_store_post(cudaStream_t st, const LevelView &P, const RecView &R, const StepConsts &k, int p, int is_level0,
                       const float *in)
{
    launch_aa(1, st, P, P, R, k, p, is_level0, const_cast<float *>(in));
}

void launch_explode(cudaStream_t st, const LevelView &P, const LevelView &F, const RecView &R, const StepConsts &k,
                    const float *post)
{
    launch_aa(2, st, P, F, R, k, 0, 0, const_cast<float *>(post));
}

void launch_init_feq(cudaStream_t st, const LevelView &P, const float *feq9, float U, float chi_inf)
{
    Feq9 e;
    for (int q = 0; q < 9; q++) e.g[q] = feq9[q];
    switch (P.store) {
    case 1: k_init<__half><<<P.ntiles, LBM_TILE, 0, st>>>(P, e, U, chi_inf); break;
    case 2: k_init<__nv_bfloat16><<<P.ntiles, LBM_TILE, 0, st>>>(P, e, U, chi_inf); break;
    default: k_init<float><<<P.ntiles, LBM_TILE, 0, st>>>(P, e, U, chi_inf); break;
    }
}

void launch_fill9(cudaStream_t st, float *buf, long long n, const float *g9)
{
    if (n <= 0) return;
    Feq9 e;
    for (int q = 0; q < 9; q++) e.g[q] = g9[q];
    k_fill9<<<(unsigned)((9 * n + 255) / 256), 256, 0, st>>>(buf, n, e);
}

void launch_loads(cudaStream_t st, const LoadsView &S, const RecView &R, float U, double *acc4)
{
    if (S.nseg <= 0) return;
    k_loads<<<(S.nseg + 255) / 256, 256, 0, st>>>(S, R, U, acc4);
}

void launch_mass(cudaStream_t st, const LevelView &P, int p, double area, double *acc, int *status)
{
    k_mass<<<P.ntiles, LBM_TILE, 0, st>>>(P, p, area, acc, status);
}

}  // namespace lbmdev
