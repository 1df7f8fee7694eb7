// noalloc.cu -- FP64 mass and non-finite check of one level's fields with no device
// allocation: the per-block partial sums live in a fixed file-scope device array.
//
// Callers that cannot allocate device memory -- code running where cudaMalloc is
// forbidden or unavailable (inside another framework's stream capture, real-time
// loops with a fixed memory plan, memory pools owned by someone else) -- can still
// check a level's mass and finiteness with this entry point.  The scratch array is
// held by every GPU that loads the library until the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "../../include/lbm.h"
#include "layout.hpp"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 4096;            // 4096 partial sums + flags: 48 KB per device
constexpr int NA_CELLS_PER_THREAD = 64;        // so n <= 4096 * 256 * 64 = 67,108,864 cells
constexpr int NA_MAX_DEVICES = 64;

struct NaScratch {
    double partial[NA_MAX_BLOCKS];
    int nonfinite[NA_MAX_BLOCKS];
};

static __device__ __align__(256) NaScratch na_scratch;

// Device address of na_scratch per device ordinal, looked up once per device (under
// na_mu, so that first calls from several host threads look it up once) and read
// without a lock afterwards.  A cudaDeviceReset destroys the module instance the
// address belongs to: the cached address is then stale.
static std::atomic<NaScratch *> na_ptr[NA_MAX_DEVICES];
static std::mutex na_mu;

__device__ __forceinline__ double na_warp_sum(double v)
{
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// pass 1: block b sums area * rho over the active fluid cells of its contiguous chunk
// and records whether any of them holds a non-finite rho, u or chi
__global__ void __launch_bounds__(NA_THREADS) k_mass_partial(const uint32_t *flags, const float *drho, const float *ux,
                                                              const float *uy, const float *chi, long long n,
                                                              long long chunk, double area, NaScratch *sc)
{
    __shared__ double red[NA_THREADS / 32];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    double v = 0.0;
    int nf = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += NA_THREADS) {
        const uint32_t fl = flags[i];
        if ((fl & FL_KIND_MASK) != KIND_ACTIVE || (fl & FL_SOLID)) continue;
        const float d = drho[i];
        if (!(isfinite(d) && isfinite(ux[i]) && isfinite(uy[i]) && isfinite(chi[i]))) nf = 1;
        v += area * (1.0 + (double)d);
    }
    v = na_warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    if (nf) atomicOr(&bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NA_THREADS / 32; w++) s += red[w];
        sc->partial[blockIdx.x] = s;
        sc->nonfinite[blockIdx.x] = bad;
    }
}

// pass 2: one block adds the partial sums in a fixed order
__global__ void __launch_bounds__(NA_THREADS) k_mass_final(const NaScratch *sc, int nblocks, double *mass_out,
                                                            int *nonfinite_out)
{
    __shared__ double red[NA_THREADS / 32];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double v = 0.0;
    int nf = 0;
    for (int b = threadIdx.x; b < nblocks; b += NA_THREADS) {
        v += sc->partial[b];
        nf |= sc->nonfinite[b];
    }
    v = na_warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    if (nf) atomicOr(&bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NA_THREADS / 32; w++) s += red[w];
        *mass_out = s;
        *nonfinite_out = bad;
    }
}

}  // namespace

extern "C" lbm_status lbm_level_mass_noalloc(const unsigned int *flags, const float *drho, const float *ux,
                                             const float *uy, const float *nu_tilde_ratio, long long n_cells,
                                             double area, double *mass_out, int *nonfinite_out, void *stream)
{
    if (n_cells < 0 || n_cells > LBM_NOALLOC_MAX_CELLS || !mass_out || !nonfinite_out ||
        (n_cells > 0 && (!flags || !drho || !ux || !uy || !nu_tilde_ratio)))
        return LBM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return LBM_ERR_CUDA;
    NaScratch *sc = na_ptr[dev].load(std::memory_order_acquire);
    if (!sc) {
        // first call on this device: look up the device address of the scratch array
        std::lock_guard<std::mutex> lock(na_mu);
        sc = na_ptr[dev].load(std::memory_order_relaxed);
        if (!sc) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) return LBM_ERR_CUDA;
            sc = (NaScratch *)p;
            na_ptr[dev].store(sc, std::memory_order_release);
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long per_block = (long long)NA_THREADS * NA_CELLS_PER_THREAD;
    long long nb = (n_cells + per_block - 1) / per_block;
    if (nb < 1) nb = 1;
    const long long chunk = (n_cells + nb - 1) / nb > 0 ? (n_cells + nb - 1) / nb : 1;
    k_mass_partial<<<(unsigned)nb, NA_THREADS, 0, st>>>(flags, (const float *)drho, ux, uy, nu_tilde_ratio, n_cells,
                                                        chunk, area, sc);
    k_mass_final<<<1, NA_THREADS, 0, st>>>(sc, (int)nb, mass_out, nonfinite_out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
