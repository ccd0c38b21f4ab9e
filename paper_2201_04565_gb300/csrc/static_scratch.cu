// static_scratch.cu -- spring energy and virial sum without device allocation.
//
// Same per-spring arithmetic and two-pass fixed-order reduction as the sample
// path of the spring-list kernels, but the per-chunk partial sums live in a
// file-scope device array instead of context memory, so this entry point never
// calls cudaMalloc or cudaFree. It exists for callers that cannot allocate:
// code that works inside a memory pool or budget owned by another framework,
// and code that must not trigger the implicit device-wide synchronisation of
// cudaFree.
//
// The array is shared by every call on a device and keeps the last call's
// contents. Each call overwrites exactly the partials it then reads, so
// nothing needs clearing; calls whose kernels overlap on the GPU (different
// streams, no ordering) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "lsm_internal.h"

namespace lsm {
namespace {

constexpr int ST_THREADS = 256;
constexpr int64_t ST_CHUNK = 4096;        // springs folded into one partial
constexpr int64_t ST_MAX_CHUNKS = 65536;  // partial slots: 2 x 65536 doubles = 1 MiB

static __device__ __align__(256) double g_partials[2 * ST_MAX_CHUNKS];

// Device address of g_partials for each device, looked up once per device
// with that device current (the symbol's name in host code is only a
// host-side stand-in).
std::mutex g_mu;
double *g_addr[64] = {nullptr};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int DIM>
__global__ void __launch_bounds__(ST_THREADS)
k_static_energy(int64_t n, int64_t m, const double *__restrict__ x, const int32_t *__restrict__ si,
                const int32_t *__restrict__ sj, const double *__restrict__ k, const double *__restrict__ r0,
                const uint8_t *__restrict__ broken, double *__restrict__ part, int64_t nchunks)
{
    __shared__ double sw[ST_THREADS / 32], su[ST_THREADS / 32];
    const int64_t c0 = (int64_t)blockIdx.x * ST_CHUNK;
    double w = 0.0, u = 0.0;
    for (int64_t s = c0 + threadIdx.x; s < c0 + ST_CHUNK && s < m; s += ST_THREADS) {
        if (broken && broken[s]) continue;
        const int32_t i = si[s], j = sj[s];
        double d[DIM];
#pragma unroll
        for (int c = 0; c < DIM; c++) d[c] = __dsub_rn(x[c * n + j], x[c * n + i]);
        double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
        if constexpr (DIM == 3) r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
        const double r = __dsqrt_rn(r2);
        const double st = __dsub_rn(r, r0[s]);
        const double cs = __ddiv_rn(__dmul_rn(k[s], st), r);
        u += __dmul_rn(__dmul_rn(__dmul_rn(0.5, k[s]), st), st);
        w += __dmul_rn(d[0], __dmul_rn(cs, d[0]));
    }
    w = warp_sum(w);
    u = warp_sum(u);
    if ((threadIdx.x & 31) == 0) {
        sw[threadIdx.x >> 5] = w;
        su[threadIdx.x >> 5] = u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tw = 0.0, tu = 0.0;
        for (int q = 0; q < ST_THREADS / 32; q++) {
            tw += sw[q];
            tu += su[q];
        }
        part[blockIdx.x] = tu;
        part[ST_MAX_CHUNKS + blockIdx.x] = tw;
    }
    (void)nchunks;
}

__global__ void __launch_bounds__(1024)
k_static_fold(const double *__restrict__ part, int64_t nchunks, double *__restrict__ out)
{
    __shared__ double sh[2][32];
    double u = 0.0, w = 0.0;
    for (int64_t b = threadIdx.x; b < nchunks; b += 1024) {
        u += part[b];
        w += part[ST_MAX_CHUNKS + b];
    }
    u = warp_sum(u);
    w = warp_sum(w);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = u;
        sh[1][threadIdx.x >> 5] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tu = 0.0, tw = 0.0;
        for (int q = 0; q < 32; q++) {
            tu += sh[0][q];
            tw += sh[1][q];
        }
        out[0] = tu;
        out[1] = tw;
    }
}

}  // namespace
}  // namespace lsm

extern "C" lsm_status lsm_spring_energy_static(int32_t dim, int64_t n, int64_t m, const double *x,
                                               const int32_t *si, const int32_t *sj, const double *k,
                                               const double *r0, const uint8_t *broken, double *out,
                                               void *stream)
{
    using namespace lsm;
    if ((dim != 2 && dim != 3) || n < 1 || m < 0 || !x || !out || (m > 0 && (!si || !sj || !k || !r0))) {
        set_thread_error("lsm_spring_energy_static: need dim 2 or 3, n >= 1, m >= 0 and non-null arrays");
        return LSM_EINVAL;
    }
    if (m > ST_CHUNK * ST_MAX_CHUNKS) {  // beyond the static partial buffer
        set_thread_error("lsm_spring_energy_static: more than 268435456 springs (static buffer limit)");
        return LSM_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set_thread_error("lsm_spring_energy_static: no usable current device (device index must be < 64)");
        return LSM_ECUDA;
    }
    double *part;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
                set_thread_error("lsm_spring_energy_static: cudaGetSymbolAddress failed");
                return LSM_ECUDA;
            }
            g_addr[dev] = (double *)p;
        }
        part = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetLastError();  // launch errors below are reported, not earlier ones
    const int64_t nchunks = (m + ST_CHUNK - 1) / ST_CHUNK;
    if (nchunks > 0) {
        if (dim == 3)
            k_static_energy<3><<<(unsigned)nchunks, ST_THREADS, 0, st>>>(n, m, x, si, sj, k, r0, broken, part, nchunks);
        else
            k_static_energy<2><<<(unsigned)nchunks, ST_THREADS, 0, st>>>(n, m, x, si, sj, k, r0, broken, part, nchunks);
    }
    k_static_fold<<<1, 1024, 0, st>>>(part, nchunks, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return LSM_ECUDA;
    }
    return LSM_OK;
}
