// kernels.cu -- sm_103a kernels of the general (CSR) lattice-spring path.
//
// One time step (Section 2.2, Eqs. 3-5, half-step velocity form) is two
// launches:
//   k_springs : one thread per spring. Spring vector, break test on the
//               squared length (Section 2.3 force listing: a spring longer
//               than rc is zeroed for good in the step the test fires), and
//               the spring force of Eq. 2, written once per spring.
//   k_gather  : one thread per particle. Sums the forces of its springs in
//               ascending spring order (no atomics: the sum is the same on
//               every run and equals the sequential canonical-order sum), then
//               the second half-kick with viscous damping (Eqs. 4-5) and, when
//               another step follows in the same call, the next half-kick and
//               drift (Eq. 3), so a step costs one particle pass.
// On the last step of a call both kernels also emit per-block partials of the
// sample observables (virial sum, Eq. 7; PE, Eq. 1; KE; grip reaction;
// residual), which k_reduce folds in a fixed order into one sample.
//
// Partials are per fixed block of TPB elements, so the reduction order does
// not depend on the grid; every launch covers its range with one block per
// chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "dfloat.cuh"
#include "lsm_internal.h"

namespace lsm {

constexpr int TPB = 256;
constexpr int RED_THREADS = 1024;

// ------------------------------------------------------------- arithmetic
// EXACT64 uses only correctly rounded IEEE operations in a fixed order (no
// contraction into fused multiply-add).
__device__ __forceinline__ double ad(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sb(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ml(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dv(double a, double b) { return __ddiv_rn(a, b); }

// Fixed-order block sum of one value per thread (TPB threads): warp xor tree,
// then the warps in order. Deterministic for a given TPB.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += sh[q];
    return t;
}

__device__ __forceinline__ double block_max(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t = fmax(t, sh[q]);
    return t;
}

// ------------------------------------------------------------ spring pass
template <int DIM, int PREC, bool BREAK, bool SAMPLE>
__global__ void __launch_bounds__(TPB)
k_springs(int64_t m, int64_t n, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
          const uint16_t *__restrict__ stype, const SpringType *__restrict__ types,
          uint8_t *__restrict__ state, long long *__restrict__ brk, const double *__restrict__ x,
          double *__restrict__ fs, const long long *__restrict__ d_step,
          unsigned long long *__restrict__ first_break, unsigned long long *__restrict__ nbroken,
          double *__restrict__ part, int64_t nblk)
{
    __shared__ double sh[TPB / 32];
    const int64_t s = (int64_t)blockIdx.x * TPB + threadIdx.x;
    double w = 0.0, u = 0.0;
    if (s < m && !state[s]) {
        const int32_t i = si[s], j = sj[s];
        const SpringType t = types[stype[s]];
        double d[DIM];
#pragma unroll
        for (int c = 0; c < DIM; c++) d[c] = sb(x[c * n + j], x[c * n + i]);
        double r2;
        if constexpr (PREC == LSM_PREC_EXACT64) {
            r2 = ad(ml(d[0], d[0]), ml(d[1], d[1]));
            if constexpr (DIM == 3) r2 = ad(r2, ml(d[2], d[2]));
        } else {
            r2 = d[0] * d[0];
#pragma unroll
            for (int c = 1; c < DIM; c++) r2 = fma(d[c], d[c], r2);
        }
        if (BREAK && r2 > t.rc2) {
            // Heaviside switch: the spring is broken for good and gives no
            // force from this step on.
            state[s] = 1;
            const long long st = *d_step;
            brk[s] = st;
            atomicMin(first_break, (unsigned long long)st);
            atomicAdd(nbroken, 1ull);
#pragma unroll
            for (int c = 0; c < DIM; c++) fs[c * m + s] = 0.0;
        } else {
            double cs;
            if constexpr (PREC == LSM_PREC_EXACT64) {
                const double r = __dsqrt_rn(r2);
                cs = dv(ml(t.k, sb(r, t.r0)), r);
                if (SAMPLE) {
                    const double e = sb(r, t.r0);
                    u = ml(ml(ml(0.5, t.k), e), e);
                }
#pragma unroll
                for (int c = 0; c < DIM; c++) fs[c * m + s] = ml(cs, d[c]);
                if (SAMPLE) w = ml(d[0], ml(cs, d[0]));
            } else if constexpr (PREC == LSM_PREC_FAST64) {
                const double ir = rsqrt(r2);
                cs = fma(-t.kr0, ir, t.k);  // k (r - r0) / r = k - k r0 / r
                if (SAMPLE) {
                    const double e = fma(r2, ir, -t.r0);
                    u = 0.5 * t.k * e * e;
                }
#pragma unroll
                for (int c = 0; c < DIM; c++) fs[c * m + s] = cs * d[c];
                if (SAMPLE) w = d[0] * (cs * d[0]);
            } else {  // LSM_PREC_F32: spring vector in double, force in float
                float df[DIM];
#pragma unroll
                for (int c = 0; c < DIM; c++) df[c] = (float)d[c];
                float r2f = df[0] * df[0];
#pragma unroll
                for (int c = 1; c < DIM; c++) r2f = fmaf(df[c], df[c], r2f);
                const float ir = rsqrtf(r2f);
                const float csf = fmaf(-(float)t.kr0, ir, (float)t.k);
                if (SAMPLE) {
                    const float e = fmaf(r2f, ir, -(float)t.r0);
                    u = 0.5 * t.k * (double)e * (double)e;
                }
#pragma unroll
                for (int c = 0; c < DIM; c++) fs[c * m + s] = (double)(csf * df[c]);
                if (SAMPLE) w = d[0] * (double)(csf * df[0]);
            }
        }
    }
    if (SAMPLE) {
        const double tw = block_sum(w, sh);
        const double tu = block_sum(u, sh);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = tw;
            part[nblk + blockIdx.x] = tu;
        }
    }
}

// ---------------------------------------------------------- particle pass
enum { G_END = 0, G_DRIFT = 1, G_INIT = 2, G_OBSERVE = 3 };

template <int DIM, int MODE, bool SAMPLE>
__global__ void __launch_bounds__(TPB)
k_gather(int64_t n, int64_t m, const int64_t *__restrict__ row, const uint32_t *__restrict__ inc,
         const double *__restrict__ fs, double *__restrict__ x, double *__restrict__ v,
         double *__restrict__ a, const double *__restrict__ mass, const uint8_t *__restrict__ fixm,
         const uint8_t *__restrict__ grip, double dt, double hdt, double gamma,
         double *__restrict__ part, int64_t nblk, int *__restrict__ status,
         long long *__restrict__ d_step)
{
    __shared__ double sh[TPB / 32];
    const int64_t p = (int64_t)blockIdx.x * TPB + threadIdx.x;
    double mvx2 = 0.0, ke = 0.0, react = 0.0, res = 0.0;
    if ((MODE == G_END || MODE == G_DRIFT) && p == 0) *d_step += 1;
    if (p < n) {
        double F[DIM];
#pragma unroll
        for (int c = 0; c < DIM; c++) F[c] = 0.0;
        const int64_t e0 = row[p], e1 = row[p + 1];
        for (int64_t e = e0; e < e1; e++) {
            const uint32_t word = inc[e];
            const int64_t s = word >> 1;
            if (word & 1u) {
#pragma unroll
                for (int c = 0; c < DIM; c++) F[c] = sb(F[c], fs[c * m + s]);
            } else {
#pragma unroll
                for (int c = 0; c < DIM; c++) F[c] = ad(F[c], fs[c * m + s]);
            }
        }
        const uint8_t fx = fixm[p];
        const double mp = mass[p];
        bool bad = false;
#pragma unroll
        for (int c = 0; c < DIM; c++) {
            const int64_t q = c * n + p;
            if (SAMPLE && c == 0 && grip[p] == 2) react = sb(react, F[0]);
            if (fx & (1u << c)) continue;
            if constexpr (MODE == G_INIT) {
                a[q] = dv(sb(F[c], ml(gamma, v[q])), mp);
            } else if constexpr (MODE == G_OBSERVE) {
                const double vn = v[q];
                if (SAMPLE) {
                    res = fmax(res, fmax(fabs(F[c]), fabs(vn)));
                    ke += 0.5 * mp * vn * vn;
                    if (c == 0) mvx2 += mp * vn * vn;
                }
            } else {
                const double vh = v[q];
                const double acc = dv(sb(F[c], ml(gamma, vh)), mp);
                const double vn = ad(vh, ml(hdt, acc));
                if (SAMPLE) {
                    res = fmax(res, fmax(fabs(F[c]), fabs(vn)));
                    ke += 0.5 * mp * vn * vn;
                    if (c == 0) mvx2 += mp * vn * vn;
                    bad |= !isfinite(vn) || !isfinite(x[q]);
                }
                if constexpr (MODE == G_DRIFT) {
                    const double vh2 = ad(vn, ml(hdt, acc));
                    v[q] = vh2;
                    x[q] = ad(x[q], ml(dt, vh2));
                } else {
                    a[q] = acc;
                    v[q] = vn;
                }
            }
        }
        if (SAMPLE && bad) atomicOr(status, 1);
    }
    if (SAMPLE) {
        const double t0 = block_sum(mvx2, sh);
        const double t1 = block_sum(ke, sh);
        const double t2 = block_sum(react, sh);
        const double t3 = block_max(res, sh);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = t0;
            part[nblk + blockIdx.x] = t1;
            part[2 * nblk + blockIdx.x] = t2;
            part[3 * nblk + blockIdx.x] = t3;
        }
    }
}

// First half-kick and drift of a call (Eq. 3): vh = v + dt/2 a; x += dt vh.
template <int DIM>
__global__ void __launch_bounds__(TPB)
k_drift(int64_t n, double *__restrict__ x, double *__restrict__ v, const double *__restrict__ a,
        const uint8_t *__restrict__ fixm, double dt, double hdt)
{
    const int64_t p = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (p >= n) return;
    const uint8_t fx = fixm[p];
#pragma unroll
    for (int c = 0; c < DIM; c++) {
        if (fx & (1u << c)) continue;
        const int64_t q = c * n + p;
        const double vh = ad(v[q], ml(hdt, a[q]));
        v[q] = vh;
        x[q] = ad(x[q], ml(dt, vh));
    }
}

// Constant strain rate (Section 3.1): before the spring pass of the step that
// completes step count s, each grip's x takes the strain eps0 + (s - s0) rdt
// (the steps completed so far are *d_step; no other kernel of the step runs
// concurrently). xf: the fixed-point copy, when the path keeps one.
__global__ void k_rate_grips(int64_t ng, int64_t n, const int32_t *__restrict__ glist, double *__restrict__ x,
                             const double *__restrict__ Xx, const long long *__restrict__ d_step, double eps0,
                             long long s0, double rdt, double xc, long long *__restrict__ xf, int S,
                             int *__restrict__ status)
{
    const int64_t q = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (q >= ng) return;
    const int64_t p = glist[q];
    const double eps = ad(eps0, ml((double)(*d_step + 1 - s0), rdt));
    const double X = Xx[p];
    const double xp = ad(X, ml(eps, sb(X, xc)));
    x[p] = xp;
    if (xf) {
        bool over = false;
        xf[p] = dbl_to_fix(xp, S, over);
        if (over) atomicOr(status, 2);
    }
}

// Load increment (Sections 2.3, 3.1).
__global__ void __launch_bounds__(TPB)
k_apply_strain(int64_t n, double *__restrict__ x, double *__restrict__ v, double *__restrict__ a,
               const double *__restrict__ Xx, const uint8_t *__restrict__ fixm, double xc,
               double scale, double eps, int affine, double *__restrict__ d_eps)
{
    const int64_t p = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (p == 0) *d_eps = eps;
    if (p >= n) return;
    double xp = x[p];
    if (affine) xp = ad(xc, ml(sb(xp, xc), scale));
    if (fixm[p] & 1u) {
        const double X = Xx[p];
        xp = ad(X, ml(eps, sb(X, xc)));
        v[p] = 0.0;
        a[p] = 0.0;
    }
    x[p] = xp;
}

// Fold the per-block partials into one sample, in a fixed order.
__global__ void __launch_bounds__(RED_THREADS)
k_reduce(const double *__restrict__ ps, int64_t nbs, const double *__restrict__ pp, int64_t nbp,
         double *d_eps, const unsigned long long *__restrict__ nbroken,
         long long *__restrict__ d_step, long long add_steps, double omega, double grip_area,
         DeviceSample *__restrict__ dst, long long *__restrict__ counter, int64_t cap, int rate_on,
         double rate_eps0, long long rate_step0, double rate_dt)
{
    constexpr int NW = RED_THREADS / 32;
    __shared__ double sh[6][NW];
    __shared__ double tot[6];
    double acc[6];
    for (int q = 0; q < 6; q++) acc[q] = 0.0;
    for (int64_t b = threadIdx.x; b < nbs; b += RED_THREADS) {
        acc[0] += ps[b];
        acc[1] += ps[nbs + b];
    }
    for (int64_t b = threadIdx.x; b < nbp; b += RED_THREADS) {
        acc[2] += pp[b];
        acc[3] += pp[nbp + b];
        acc[4] += pp[2 * nbp + b];
        acc[5] = fmax(acc[5], pp[3 * nbp + b]);
    }
    // the six block reductions of block_sum / block_max side by side (same
    // order: a warp xor tree, then the warps in order, one value per thread)
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 5; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        acc[5] = fmax(acc[5], __shfl_xor_sync(0xffffffffu, acc[5], o));
    }
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 6; q++) sh[q][threadIdx.x >> 5] = acc[q];
    __syncthreads();
    if (threadIdx.x < 6) {
        const int q = threadIdx.x;
        double t = 0.0;
        for (int k = 0; k < NW; k++) t = q == 5 ? fmax(t, sh[q][k]) : t + sh[q][k];
        tot[q] = t;
    }
    __syncthreads();
    const double W = tot[0], U = tot[1], MV = tot[2], KE = tot[3], R = tot[4], RES = tot[5];
    if (threadIdx.x == 0) {
        DeviceSample smp;
        const long long stp = *d_step + add_steps;
        if (rate_on) *d_eps = ad(rate_eps0, ml((double)(stp - rate_step0), rate_dt));
        smp.eps = *d_eps;
        smp.sigma_vir = (W - MV) / omega;
        smp.sigma_grip = R / grip_area;
        smp.pe = U;
        smp.ke = KE;
        smp.residual = RES;
        smp.n_broken = (long long)*nbroken;
        *d_step = stp;
        smp.step = stp;
        if (counter) {
            const long long k = *counter;
            if (k < cap) dst[k] = smp;
            *counter = k + 1;
        } else {
            dst[0] = smp;
        }
    }
}

// --------------------------------------------------------------- host side

static inline unsigned grid_of(int64_t cnt) { return (unsigned)((cnt + TPB - 1) / TPB); }

thread_local const char *g_fail_site = "";

const char *last_fail_site() { return g_fail_site; }

#define LSM_TRY(x)                                \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) {                  \
            g_fail_site = #x;                     \
            return e_;                            \
        }                                         \
    } while (0)

template <typename T>
static cudaError_t dalloc(T **p, size_t count)
{
    return lsm::dev_malloc((void **)p, (count ? count : 1) * sizeof(T));
}

void free_device(Ctx &c)
{
    fields_free(c);
    for (auto &kv : c.graphs) cudaGraphExecDestroy(kv.second);
    c.graphs.clear();
    if (c.rb_stream) {
        cudaStreamSynchronize(c.rb_stream);
        cudaStreamDestroy(c.rb_stream);
        c.rb_stream = nullptr;
    }
    for (int k = 0; k < 2; k++) {
        if (c.rb_buf[k]) cudaFree(c.rb_buf[k]);
        if (c.rb_ready[k]) cudaEventDestroy(c.rb_ready[k]);
        if (c.rb_done[k]) cudaEventDestroy(c.rb_done[k]);
        c.rb_buf[k] = nullptr;
        c.rb_ready[k] = c.rb_done[k] = nullptr;
        c.rb_used[k] = false;
    }
    void *ptrs[] = {c.x, c.v, c.a, c.mass, c.Xx, c.fixm, c.grip, c.si, c.sj, c.stype, c.types,
                    c.state, c.brk, c.row, c.inc, c.fs, c.part_s, c.part_p, c.d_step,
                    c.d_first_break, c.d_nbroken, c.d_status, c.d_eps, c.d_nsamples, c.samples,
                    c.scratch_sample};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *tptrs[] = {c.tx[0], c.tx[1], c.tvh[0], c.tvh[1], c.tvobs, c.tph, c.tmask, c.tbrk, c.tmass,
                     c.tinvm, c.tdf, c.tsbase, c.texport, c.texport_brk, c.xf, c.sdir, c.imass, c.fsx,
                     c.tmask3, c.grip_list};
    for (void *p : tptrs)
        if (p) cudaFree(p);
    c.tsbase = nullptr;
    c.xf = nullptr;
    c.sdir = nullptr;
    c.imass = nullptr;
    c.fsx = nullptr;
    c.texport = nullptr;
    c.texport_brk = nullptr;
    c.tx[0] = c.tx[1] = c.tvh[0] = c.tvh[1] = c.tvobs = c.tmass = c.tinvm = nullptr;
    c.tdf = nullptr;
    c.tph = c.tmask = nullptr;
    c.tmask3 = nullptr;
    c.grip_list = nullptr;
    c.tbrk = nullptr;
    c.x = c.v = c.a = c.mass = c.Xx = nullptr;
    c.fixm = c.grip = nullptr;
    c.si = c.sj = nullptr;
    c.stype = nullptr;
    c.types = nullptr;
    c.state = nullptr;
    c.brk = nullptr;
    c.row = nullptr;
    c.inc = nullptr;
    c.fs = c.part_s = c.part_p = nullptr;
    c.d_step = nullptr;
    c.d_first_break = c.d_nbroken = nullptr;
    c.d_status = nullptr;
    c.d_eps = nullptr;
    c.d_nsamples = nullptr;
    c.samples = c.scratch_sample = nullptr;
}

static cudaError_t upload_common(Ctx &c)
{
    LSM_TRY(dalloc(&c.d_step, 1));
    LSM_TRY(dalloc(&c.d_first_break, 1));
    LSM_TRY(dalloc(&c.d_nbroken, 1));
    LSM_TRY(dalloc(&c.d_status, 1));
    LSM_TRY(dalloc(&c.d_eps, 1));
    LSM_TRY(dalloc(&c.d_nsamples, 1));
    c.sample_cap = 1024;
    LSM_TRY(dalloc(&c.samples, c.sample_cap));
    LSM_TRY(dalloc(&c.scratch_sample, 1));
    LSM_TRY(dalloc(&c.types, c.h.types.size()));
    cudaStream_t st = c.stream;
    LSM_TRY(cudaMemcpyAsync(c.types, c.h.types.data(), c.h.types.size() * sizeof(SpringType),
                            cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemsetAsync(c.d_step, 0, sizeof(long long), st));
    LSM_TRY(cudaMemsetAsync(c.d_first_break, 0xff, sizeof(unsigned long long), st));
    LSM_TRY(cudaMemsetAsync(c.d_nbroken, 0, sizeof(unsigned long long), st));
    LSM_TRY(cudaMemsetAsync(c.d_status, 0, sizeof(int), st));
    LSM_TRY(cudaMemsetAsync(c.d_eps, 0, sizeof(double), st));
    LSM_TRY(cudaMemsetAsync(c.d_nsamples, 0, sizeof(long long), st));
    return cudaSuccess;
}

// Nearest double-float of a double: hi = float(v), lo = float(v - hi).
static ff split_ff(double v)
{
    const float hi = (float)v;
    return ff{hi, (float)(v - (double)hi)};
}

// Tile path: state on the 2D pixel grid, both ping-pong buffers at the
// reference lattice, velocities zero, no spring broken.
static cudaError_t upload_tile(Ctx &c)
{
    const HostNet &h = c.h;
    // the tile grid: the pixel grid, or the triangular packing's sites (rows
    // of nx sites at y = iy h; odd rows use the first nx - 1, shifted by a/2)
    const double hrow = h.a * std::sqrt(3.0) * 0.5;
    c.tgnx = h.nx;
    c.tgny = h.ny;
    c.tgidx.assign(h.n, 0);
    std::vector<uint8_t> gphase;
    if (c.tri) {
        int64_t rows = 0;
        for (int64_t p = 0; p < h.n; p++) rows = std::max<int64_t>(rows, std::llround(h.X[h.n + p] / hrow) + 1);
        c.tgny = (int)rows;
        gphase.assign((size_t)c.tgnx * c.tgny, 0);
        for (int64_t p = 0; p < h.n; p++) {
            const int64_t iy = std::llround(h.X[h.n + p] / hrow);
            const int64_t ix = std::llround(h.X[p] / h.a - ((iy & 1) ? 0.5 : 0.0));
            c.tgidx[p] = iy * c.tgnx + ix;
            gphase[c.tgidx[p]] = h.phase[h.pix[p]];
        }
    } else {
        for (int64_t p = 0; p < h.n; p++) c.tgidx[p] = h.pix[p];
    }
    const uint8_t *gph = c.tri ? gphase.data() : h.phase.data();
    const int64_t np = (int64_t)c.tgnx * c.tgny;
    c.tnp = np;
    c.tile_nphase = h.nphase;
    c.ntiles = c.tri ? 0 : tile_count(c);
    if (c.strip) {
        bool fills = true;
        LSM_TRY(strip_geometry(c, &fills));
        if (!fills && !c.tri && !c.strip_forced) {  // small image: the tile kernel
            c.strip = false;
            c.nstrips = 0;
        }
    }
    if (c.tri) c.ntiles = c.nstrips;  // the packing's samples all come from the strip kernel
    std::vector<double> X(2 * np);
    for (int64_t g = 0; g < np; g++) {
        const int64_t ix = g % c.tgnx, iy = g / c.tgnx;
        X[g] = c.tri ? (ix + ((iy & 1) ? 0.5 : 0.0)) * h.a : ix * h.a;
        X[np + g] = c.tri ? iy * hrow : iy * h.a;
    }
    std::vector<double> mtab(h.nphase, 1.0), itab(h.nphase, 1.0);
    for (int64_t p = 0; p < h.n; p++) mtab[gph[c.tgidx[p]] - 1] = h.mass[p];
    itab.assign(4 * h.nphase, 0.0);  // per phase: 1 - dt g/m, dt/m, 1 - dt/2 g/m, dt/2 / m
    for (int q = 0; q < h.nphase; q++) {
        const double dt = h.dt, hdt = 0.5 * h.dt, g = h.damping, m = mtab[q];
        itab[4 * q + 0] = 1.0 - dt * g / m;
        itab[4 * q + 1] = dt / m;
        itab[4 * q + 2] = 1.0 - hdt * g / m;
        itab[4 * q + 3] = hdt / m;
    }
    // fixed-point scale: |x| stays below 2^(62 - S) for strains up to +300%,
    // spring vectors up to 2 r0 of the diagonal spring (a sqrt 2) and up to
    // every critical length stay below 2^(48 - S), where their conversion to
    // double-float is exact
    const double extent = 4.0 * (double)(h.nx > h.ny ? h.nx : h.ny) * h.a + 16.0;
    c.fix_S = 61 - (int)std::ceil(std::log2(extent));
    c.fix_S = std::min(c.fix_S, 47 - (int)std::ceil(std::log2(h.a * std::sqrt(2.0))));
    c.fix_S = std::min(c.fix_S, 47 - (int)std::floor(std::log2(max_critical_length(h.types))));
    c.a_fix = std::llround(std::ldexp(h.a, c.fix_S));
    c.h_fix = std::llround(std::ldexp(hrow, c.fix_S));
    std::vector<int64_t> sbase(np, 0);
    for (int64_t s = h.m - 1; s >= 0; s--) sbase[c.tgidx[h.si[s]]] = s;
    std::vector<TypeDF> tdf(h.types.size());
    for (size_t q = 0; q < h.types.size(); q++) {
        const SpringType &t = h.types[q];
        // the type's lattice vector o as the F32 kernels use it (fixed point):
        // square lattice (a, 0) or (a, a) by shell; triangular packing (a, 0)
        // for the row spring, (a/2, h) for the other two
        const double ox = std::ldexp((double)(c.tri && (q & 1) ? (c.a_fix >> 1) : c.a_fix), -c.fix_S);
        const double oy = (q & 1) ? std::ldexp((double)(c.tri ? c.h_fix : c.a_fix), -c.fix_S) : 0.0;
        // |o|^2 - r0^2 with the products' rounding errors kept (fma)
        const double p = t.r0 * t.r0, pe = std::fma(t.r0, t.r0, -p);
        const double o2 = ox * ox + oy * oy, o2e = std::fma(ox, ox, -(ox * ox)) + std::fma(oy, oy, -(oy * oy));
        // DF kernels hold lengths in units of 2^(24-S): r0 and rc^2 scaled
        // exactly by powers of two (F32 keeps the plain values)
        const double ul = h.precision == LSM_PREC_DF ? std::ldexp(1.0, c.fix_S - 24) : 1.0;
        tdf[q].k = split_ff(t.k);
        tdf[q].r0 = split_ff(t.r0 * ul);
        tdf[q].rc2 = split_ff(t.rc2 * ul * ul);
        tdf[q].cor = split_ff((o2 - p) + (o2e - pe));
    }
    for (int b = 0; b < 2; b++) {
        LSM_TRY(dalloc(&c.tx[b], 2 * np));
        LSM_TRY(dalloc(&c.tvh[b], 2 * np));
    }
    LSM_TRY(dalloc(&c.tvobs, 2 * np));
    LSM_TRY(dalloc(&c.tph, np));
    LSM_TRY(dalloc(&c.tmask, np));
    LSM_TRY(dalloc(&c.tbrk, 4 * np));
    LSM_TRY(dalloc(&c.tmass, h.nphase));
    LSM_TRY(dalloc(&c.tinvm, 4 * h.nphase));
    LSM_TRY(dalloc(&c.tdf, tdf.size()));
    LSM_TRY(dalloc(&c.tsbase, np));
    {  // partial sums: per tile (tile kernel samples) or per strip (strip samples)
        const int64_t np_ = std::max<int64_t>(c.ntiles, c.nstrips);
        LSM_TRY(dalloc(&c.part_s, 2 * np_));
        LSM_TRY(dalloc(&c.part_p, 4 * np_));
    }
    LSM_TRY(upload_common(c));
    cudaStream_t st = c.stream;
    for (int b = 0; b < 2; b++) {
        LSM_TRY(cudaMemcpyAsync(c.tx[b], X.data(), 2 * np * sizeof(double), cudaMemcpyHostToDevice, st));
        LSM_TRY(cudaMemsetAsync(c.tvh[b], 0, 2 * np * sizeof(double), st));
    }
    LSM_TRY(cudaMemsetAsync(c.tvobs, 0, 2 * np * sizeof(double), st));
    LSM_TRY(cudaMemcpyAsync(c.tph, gph, np, cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemsetAsync(c.tmask, 0, np, st));
    LSM_TRY(cudaMemsetAsync(c.tbrk, 0xff, 4 * np * sizeof(long long), st));
    LSM_TRY(cudaMemcpyAsync(c.tmass, mtab.data(), h.nphase * sizeof(double), cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemcpyAsync(c.tinvm, itab.data(), 4 * h.nphase * sizeof(double), cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemcpyAsync(c.tdf, tdf.data(), tdf.size() * sizeof(TypeDF), cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemcpyAsync(c.tsbase, sbase.data(), np * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    c.tcur = 0;
    LSM_TRY(cudaStreamSynchronize(st));
    return cudaSuccess;
}

cudaError_t upload(Ctx &c)
{
    const HostNet &h = c.h;
    c.dim = h.dim;
    c.n = h.n;
    c.m = h.m;
    if (c.tile && c.dim == 3) {
        LSM_TRY(upload_common(c));
        return tile3_upload(c);
    }
    if (c.tile) return upload_tile(c);
    const int64_t n = c.n, m = c.m, dn = (int64_t)h.dim * n;
    c.nblk_s = (m + TPB - 1) / TPB;
    c.nblk_p = (n + TPB - 1) / TPB;

    // incidence CSR: each particle's springs by ascending spring index
    std::vector<int64_t> row(n + 1, 0);
    for (int64_t s = 0; s < m; s++) {
        row[h.si[s] + 1]++;
        row[h.sj[s] + 1]++;
    }
    for (int64_t p = 0; p < n; p++) row[p + 1] += row[p];
    std::vector<uint32_t> inc(2 * m);
    std::vector<int64_t> fill(row.begin(), row.end() - 1);
    for (int64_t s = 0; s < m; s++) {
        inc[fill[h.si[s]]++] = (uint32_t)(s << 1);
        inc[fill[h.sj[s]]++] = (uint32_t)((s << 1) | 1);
    }
    std::vector<double> Xx(h.X.begin(), h.X.begin() + n);

    LSM_TRY(dalloc(&c.x, dn));
    LSM_TRY(dalloc(&c.v, dn));
    LSM_TRY(dalloc(&c.a, dn));
    LSM_TRY(dalloc(&c.mass, n));
    LSM_TRY(dalloc(&c.Xx, n));
    LSM_TRY(dalloc(&c.fixm, n));
    LSM_TRY(dalloc(&c.grip, n));
    LSM_TRY(dalloc(&c.si, m));
    LSM_TRY(dalloc(&c.sj, m));
    LSM_TRY(dalloc(&c.stype, m));
    LSM_TRY(dalloc(&c.state, m));
    LSM_TRY(dalloc(&c.brk, m));
    LSM_TRY(dalloc(&c.row, n + 1));
    LSM_TRY(dalloc(&c.inc, 2 * m));
    LSM_TRY(dalloc(&c.fs, (size_t)h.dim * (m ? m : 1)));
    LSM_TRY(dalloc(&c.part_s, 2 * (c.nblk_s > 0 ? c.nblk_s : 1)));
    LSM_TRY(dalloc(&c.part_p, 4 * c.nblk_p));
    LSM_TRY(upload_common(c));

    cudaStream_t st = c.stream;
    LSM_TRY(cudaMemcpyAsync(c.x, h.X.data(), dn * sizeof(double), cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemsetAsync(c.v, 0, dn * sizeof(double), st));
    LSM_TRY(cudaMemsetAsync(c.a, 0, dn * sizeof(double), st));
    LSM_TRY(cudaMemcpyAsync(c.mass, h.mass.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemcpyAsync(c.Xx, Xx.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemcpyAsync(c.fixm, h.fixm.data(), n, cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemcpyAsync(c.grip, h.grip.data(), n, cudaMemcpyHostToDevice, st));
    if (m) {
        LSM_TRY(cudaMemcpyAsync(c.si, h.si.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        LSM_TRY(cudaMemcpyAsync(c.sj, h.sj.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        LSM_TRY(cudaMemcpyAsync(c.stype, h.stype.data(), m * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
        LSM_TRY(cudaMemcpyAsync(c.inc, inc.data(), 2 * m * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    }
    LSM_TRY(cudaMemcpyAsync(c.row, row.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemsetAsync(c.state, 0, m ? m : 1, st));
    LSM_TRY(cudaMemsetAsync(c.brk, 0xff, (m ? m : 1) * sizeof(long long), st));
    LSM_TRY(cudaMemsetAsync(c.fs, 0, (size_t)h.dim * (m ? m : 1) * sizeof(double), st));
    // host vectors above must stay alive until the copies finish
    LSM_TRY(cudaStreamSynchronize(st));
    {  // particles with a prescribed x (constant strain-rate loading)
        std::vector<int32_t> gl;
        for (int64_t p = 0; p < n; p++)
            if (h.fixm[p] & 1u) gl.push_back((int32_t)p);
        c.ngrip = (int64_t)gl.size();
        LSM_TRY(dalloc(&c.grip_list, gl.size()));
        if (!gl.empty())
            LSM_TRY(cudaMemcpyAsync(c.grip_list, gl.data(), gl.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        LSM_TRY(cudaStreamSynchronize(st));
    }
    c.fixcsr = (h.precision == LSM_PREC_F32 || h.precision == LSM_PREC_DF) && !h.offv.empty() &&
               (int64_t)h.sdir.size() == m;
    if (c.fixcsr) LSM_TRY(fixcsr_upload(c));
    return cudaSuccess;
}

// Launch helpers --------------------------------------------------------------

template <int DIM, bool BREAK, bool SAMPLE>
static void springs(Ctx &c)
{
    if (c.fixcsr) {
        springs_fix<DIM, BREAK, SAMPLE>(c);
        return;
    }
    if (c.m == 0) {
        if (SAMPLE) cudaMemsetAsync(c.part_s, 0, 2 * sizeof(double), c.stream);
        return;
    }
    const unsigned g = grid_of(c.m);
#define LSM_SPR(P)                                                                              \
    k_springs<DIM, P, BREAK, SAMPLE><<<g, TPB, 0, c.stream>>>(                                  \
        c.m, c.n, c.si, c.sj, c.stype, c.types, c.state, c.brk, c.x, c.fs, c.d_step,           \
        c.d_first_break, c.d_nbroken, c.part_s, c.nblk_s)
    switch (c.h.precision) {
    case LSM_PREC_FAST64: LSM_SPR(LSM_PREC_FAST64); break;
    case LSM_PREC_DF: LSM_SPR(LSM_PREC_FAST64); break;
    case LSM_PREC_F32: LSM_SPR(LSM_PREC_F32); break;
    default: LSM_SPR(LSM_PREC_EXACT64); break;
    }
#undef LSM_SPR
}

template <int DIM, int MODE, bool SAMPLE>
static void gather(Ctx &c)
{
    if (c.fixcsr) {
        gather_fix<DIM, MODE, SAMPLE>(c);
        return;
    }
    const double dt = c.h.dt, hdt = 0.5 * c.h.dt;
    k_gather<DIM, MODE, SAMPLE><<<grid_of(c.n), TPB, 0, c.stream>>>(
        c.n, c.m, c.row, c.inc, c.fs, c.x, c.v, c.a, c.mass, c.fixm, c.grip, dt, hdt,
        c.h.damping, c.part_p, c.nblk_p, c.d_status, c.d_step);
}

// Fold the partial sums of the last sample kernel into one sample. strips:
// they came from a strip-kernel step (one partial per strip), not from the
// tile kernel (one per tile) or the spring-list kernels (one per block).
static void reduce(Ctx &c, DeviceSample *dst, long long *counter, long long add_steps, bool strips = false)
{
    const int64_t nbs = strips ? c.nstrips : c.tile ? c.ntiles : (c.m ? c.nblk_s : 1);
    const int64_t nbp = strips ? c.nstrips : c.tile ? c.ntiles : c.nblk_p;
    k_reduce<<<1, RED_THREADS, 0, c.stream>>>(c.part_s, nbs, c.part_p, nbp, c.d_eps, c.d_nbroken,
                                              c.d_step, add_steps, c.h.omega, c.h.grip_area, dst,
                                              counter, c.sample_cap, c.rate_on, c.rate_eps0, c.rate_step0,
                                              c.rate_dt);
}

template <int DIM>
static void enqueue_steps(Ctx &c, int64_t nsteps, bool record)
{
    const double dt = c.h.dt, hdt = 0.5 * c.h.dt;
    k_drift<DIM><<<grid_of(c.n), TPB, 0, c.stream>>>(c.n, c.x, c.v, c.a, c.fixm, dt, hdt);
    if (c.fixcsr) fixcsr_refresh(c);
    for (int64_t t = 0; t < nsteps; t++) {
        const bool last = t == nsteps - 1;
        if (c.rate_on && c.ngrip)
            k_rate_grips<<<grid_of(c.ngrip), TPB, 0, c.stream>>>(c.ngrip, c.n, c.grip_list, c.x, c.Xx, c.d_step,
                                                                c.rate_eps0, c.rate_step0, c.rate_dt, c.h.xc,
                                                                c.fixcsr ? c.xf : nullptr, c.fix_S, c.d_status);
        if (last) {
            springs<DIM, true, true>(c);
            gather<DIM, G_END, true>(c);
        } else {
            springs<DIM, true, false>(c);
            gather<DIM, G_DRIFT, false>(c);
        }
    }
    if (record)
        reduce(c, c.samples, c.d_nsamples, 0);
    else
        reduce(c, c.scratch_sample, nullptr, 0);
}

static cudaError_t enqueue_tile_steps(Ctx &c, int64_t nsteps, bool record)
{
    cudaError_t e = c.dim == 3 ? tile3_enqueue_steps(c, nsteps, c.tcur) : tile_enqueue_steps(c, nsteps, c.tcur);
    if (e != cudaSuccess) return e;
    const bool strips = c.dim == 2 && c.strip;  // the sample step ran on the strip kernel
    if (record)
        reduce(c, c.samples, c.d_nsamples, nsteps, strips);
    else
        reduce(c, c.scratch_sample, nullptr, nsteps, strips);
    return cudaGetLastError();
}

cudaError_t launch_steps(Ctx &c, int64_t nsteps, bool record)
{
    const int64_t key = nsteps * 4 + (record ? 2 : 0) + (c.tile ? c.tcur : 0);
    auto it = c.graphs.find(key);
    if (it == c.graphs.end()) {
        cudaGraph_t g;
        LSM_TRY(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t ee = cudaSuccess;
        if (c.tile)
            ee = enqueue_tile_steps(c, nsteps, record);
        else if (c.dim == 3)
            enqueue_steps<3>(c, nsteps, record);
        else
            enqueue_steps<2>(c, nsteps, record);
        cudaError_t e = cudaStreamEndCapture(c.stream, &g);
        if (ee != cudaSuccess) {
            if (e == cudaSuccess) cudaGraphDestroy(g);
            return ee;
        }
        if (e != cudaSuccess) return e;
        size_t nodes = 0;
        cudaGraphGetNodes(g, nullptr, &nodes);
        c.graph_nodes[key] = (int64_t)nodes;
        cudaGraphExec_t ex;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        it = c.graphs.emplace(key, ex).first;
    }
    LSM_TRY(cudaGraphLaunch(it->second, c.stream));
    c.launches += c.graph_nodes[key];
    if (c.tile) c.tcur ^= (int)(nsteps & 1);
    return cudaGetLastError();
}

cudaError_t launch_init_accel(Ctx &c)
{
    if (c.tile) return c.dim == 3 ? tile3_init_accel(c) : tile_init_accel(c);
    if (c.fixcsr) {
        const cudaError_t e = fixcsr_refresh(c);  // positions may have been replaced
        if (e != cudaSuccess) return e;
    }
    if (c.dim == 3) {
        springs<3, false, false>(c);
        gather<3, G_INIT, false>(c);
    } else {
        springs<2, false, false>(c);
        gather<2, G_INIT, false>(c);
    }
    return cudaGetLastError();
}

cudaError_t launch_observe(Ctx &c, DeviceSample *dst)
{
    if (c.tile) {
        cudaError_t e = c.dim == 3 ? tile3_observe(c) : tile_observe(c);
        if (e != cudaSuccess) return e;
        reduce(c, dst, nullptr, 0);
        return cudaGetLastError();
    }
    if (c.dim == 3) {
        springs<3, false, true>(c);
        gather<3, G_OBSERVE, true>(c);
    } else {
        springs<2, false, true>(c);
        gather<2, G_OBSERVE, true>(c);
    }
    reduce(c, dst, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_apply_strain(Ctx &c, double eps_old, double eps_new)
{
    if (c.tile) {
        c.launches += 1;
        return tile_apply_strain(c, eps_old, eps_new);
    }
    const double scale = (1.0 + eps_new) / (1.0 + eps_old);
    k_apply_strain<<<grid_of(c.n), TPB, 0, c.stream>>>(c.n, c.x, c.v, c.a, c.Xx, c.fixm, c.h.xc,
                                                       scale, eps_new, c.h.load_mode == 0,
                                                       c.d_eps);
    c.launches += 1;
    if (c.fixcsr) {
        c.launches += 1;
        return fixcsr_refresh(c);
    }
    return cudaGetLastError();
}

}  // namespace lsm
