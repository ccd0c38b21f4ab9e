// csr_fix.cu -- the spring-list path in the fixed-point modes (F32, DF).
//
// Same structure as the spring-list FP64 kernels (one thread per spring, then
// one thread per particle gathering its springs in ascending spring order),
// with the arithmetic of the 2D tile kernel's fixed-point modes: positions
// carry a 64-bit fixed-point copy xf = x 2^S, written wherever x changes; a
// spring's vector is the exact integer difference xf_j - xf_i, split into its
// lattice vector o (known from the spring's offset index) and the deviation e;
// the force is evaluated in single precision (F32) or double-float (DF) from
// (2 o + e).e = r^2 - |o|^2, which has no cancellation; forces are gathered in
// the same precision and integrated in FP64. Used for image builds whose tile
// kernel does not apply (3D volumes, path 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "dfloat.cuh"
#include "lsm_internal.h"

namespace lsm {

constexpr int FTPB = 256;

struct FixTab {
    long long o[9][3];  // lattice offset index -> o * 2^S
    ff of[9][3];        // o as double-floats
    ff oo[9];           // |o|^2
    int S;
    float p24, p0;
};

namespace {

__device__ __forceinline__ double fbsum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < FTPB / 32; q++) t += sh[q];
    return t;
}

__device__ __forceinline__ double fbmax(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < FTPB / 32; q++) t = fmax(t, sh[q]);
    return t;
}

}  // namespace

// xf = x 2^S for every component (status bit 2 if out of range)
__global__ void k_fix(int64_t total, const double *__restrict__ x, long long *__restrict__ xf, int S, int *status)
{
    const int64_t i = (int64_t)blockIdx.x * FTPB + threadIdx.x;
    if (i >= total) return;
    bool over = false;
    xf[i] = dbl_to_fix(x[i], S, over);
    if (over) atomicOr(status, 2);
}

template <int DIM, int PREC, bool BREAK, bool SAMPLE>
__global__ void __launch_bounds__(FTPB)
k_springs_fix(int64_t m, int64_t n, const int32_t *__restrict__ si, const int32_t *__restrict__ sj,
              const uint16_t *__restrict__ stype, const uint8_t *__restrict__ sdir, const TypeDF *__restrict__ tdf,
              uint8_t *__restrict__ state, long long *__restrict__ brk, const long long *__restrict__ xf, void *fsv,
              const long long *__restrict__ d_step, unsigned long long *__restrict__ first_break,
              unsigned long long *__restrict__ nbroken, double *__restrict__ part, int64_t nblk, FixTab T)
{
    using FT = typename std::conditional<PREC == LSM_PREC_F32, float, ff>::type;
    FT *fs = (FT *)fsv;
    __shared__ double sh[FTPB / 32];
    const int64_t s = (int64_t)blockIdx.x * FTPB + threadIdx.x;
    double w = 0.0, u = 0.0;
    if (s < m && !state[s]) {
        const int32_t i = si[s], j = sj[s];
        const int dir = PREC == LSM_PREC_F32 ? sdir[s] : 0;
        const TypeDF t = tdf[stype[s]];
        bool brk_now = false;
        FT f[DIM];
        if constexpr (PREC == LSM_PREC_F32) {
            // deviation e = d - o from the lattice vector o, exact in fixed
            // point: r^2 - r0^2 = (2 o + e).e + |o|^2 - r0^2 has no cancellation
            long long ef[DIM];
#pragma unroll
            for (int c = 0; c < DIM; c++) ef[c] = xf[c * n + j] - xf[c * n + i] - T.o[dir][c];
            const ff cor = ff_add(T.oo[dir], t.cor);  // |o|^2 - r0^2 (t.cor holds -r0^2)
            float e[DIM], d[DIM], s2 = 0.0f;
#pragma unroll
            for (int c = 0; c < DIM; c++) {
                e[c] = fix_to_float_i2f(ef[c], T.p24, T.p0);
                const float o = T.of[dir][c].hi;
                d[c] = o + e[c];
                s2 = fmaf(2.0f * o + e[c], e[c], s2);
            }
            const float r2 = T.oo[dir].hi + s2;  // r^2 = |o|^2 + (2 o + e).e
            const float num = s2 + cor.hi;       // r^2 - r0^2
            if (BREAK && r2 > t.rc2.hi) {
                brk_now = true;
            } else {
                const float ir = rsqrtf(r2);
                const float st = __fdividef(num, fmaf(r2, ir, t.r0.hi));
                const float cc = t.k.hi * st * ir;
#pragma unroll
                for (int c = 0; c < DIM; c++) f[c] = cc * d[c];
                if (SAMPLE) {
                    u = 0.5 * (double)t.k.hi * (double)st * (double)st;
                    w = (double)d[0] * (double)f[0];
                }
            }
        } else {
            // the spring vector d = x_j - x_i as an exact fixed-point
            // difference, converted to a double-float; 1/r by a Newton step
            // and the force k (1 - r0 / r) d (the tile kernels' arithmetic)
            ff d[DIM];
#pragma unroll
            for (int c = 0; c < DIM; c++) d[c] = fix_to_ff_i2f2(xf[c * n + j] - xf[c * n + i], T.p24, T.p0);
            ff r2;
            if constexpr (DIM == 3) r2 = ff_norm3_un(d[0], d[1], d[2]);
            else r2 = ff_norm2_un(d[0], d[1]);
            if (BREAK && ff_gt_un(r2, t.rc2)) {
                brk_now = true;
            } else {
                ff y;
                const ff g = ff_spring_g(r2, t.r0, SAMPLE ? &y : nullptr);
                const ff cc = ff_mul_un(t.k, g);  // unnormalised: only multiplied or summed further
#pragma unroll
                for (int c = 0; c < DIM; c++) f[c] = ff_mul_un(cc, d[c]);
                if (SAMPLE) {
                    const double st = ff_to_double(ff_mul(ff_mul(r2, y), g));  // r - r0
                    u = 0.5 * ff_to_double(t.k) * st * st;
                    w = ff_to_double(d[0]) * ff_to_double(f[0]);
                }
            }
        }
        if (brk_now) {
            state[s] = 1;
            const long long st = *d_step;
            brk[s] = st;
            atomicMin(first_break, (unsigned long long)st);
            atomicAdd(nbroken, 1ull);
#pragma unroll
            for (int c = 0; c < DIM; c++) f[c] = FT{};
        }
#pragma unroll
        for (int c = 0; c < DIM; c++) fs[c * m + s] = f[c];
    }
    if (SAMPLE) {
        const double tw = fbsum(w, sh);
        const double tu = fbsum(u, sh);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = tw;
            part[nblk + blockIdx.x] = tu;
        }
    }
}

enum { FG_END = 0, FG_DRIFT = 1, FG_INIT = 2, FG_OBSERVE = 3 };

template <int DIM, int PREC, int MODE, bool SAMPLE>
__global__ void __launch_bounds__(FTPB)
k_gather_fix(int64_t n, int64_t m, const int64_t *__restrict__ row, const uint32_t *__restrict__ inc, const void *fsv,
             double *__restrict__ x, double *__restrict__ v, double *__restrict__ a, long long *__restrict__ xf,
             const double *__restrict__ mass, const double *__restrict__ imass, const uint8_t *__restrict__ fixm,
             const uint8_t *__restrict__ grip, double dt, double hdt, double gamma, double *__restrict__ part,
             int64_t nblk, int *__restrict__ status, long long *__restrict__ d_step, int S)
{
    using FT = typename std::conditional<PREC == LSM_PREC_F32, float, ff>::type;
    const FT *fs = (const FT *)fsv;
    __shared__ double sh[FTPB / 32];
    const int64_t p = (int64_t)blockIdx.x * FTPB + threadIdx.x;
    double mvx2 = 0.0, ke = 0.0, react = 0.0, res = 0.0;
    bool bad = false, over = false;
    if ((MODE == FG_END || MODE == FG_DRIFT) && p == 0) *d_step += 1;
    if (p < n) {
        FT Fa[DIM];
#pragma unroll
        for (int c = 0; c < DIM; c++) Fa[c] = FT{};
        const int64_t e0 = row[p], e1 = row[p + 1];
        // unrolled so that the loads of several incident springs are in
        // flight together (the sum keeps its order)
#pragma unroll 4
        for (int64_t e = e0; e < e1; e++) {
            const uint32_t word = inc[e];
            const int64_t s = word >> 1;
#pragma unroll
            for (int c = 0; c < DIM; c++) {
                const FT f = fs[c * m + s];
                if constexpr (PREC == LSM_PREC_F32)
                    Fa[c] = (word & 1u) ? Fa[c] - f : Fa[c] + f;
                else
                    Fa[c] = ff_add_sloppy(Fa[c], (word & 1u) ? ff_neg(f) : f);
            }
        }
        double F[DIM];
#pragma unroll
        for (int c = 0; c < DIM; c++) {
            if constexpr (PREC == LSM_PREC_F32)
                F[c] = f2d_force(Fa[c]);
            else
                F[c] = f2d_force(Fa[c].hi) + f2d_force(Fa[c].lo);
        }
        const uint8_t fx = fixm[p];
        const double mp = mass[p], im = imass[p];
#pragma unroll
        for (int c = 0; c < DIM; c++) {
            const int64_t q = c * n + p;
            if (SAMPLE && c == 0 && grip[p] == 2) react -= F[0];
            if (fx & (1u << c)) continue;
            if constexpr (MODE == FG_INIT) {
                a[q] = fma(-gamma, v[q], F[c]) * im;
            } else if constexpr (MODE == FG_OBSERVE) {
                const double vn = v[q];
                if (SAMPLE) {
                    res = fmax(res, fmax(fabs(F[c]), fabs(vn)));
                    ke += 0.5 * mp * vn * vn;
                    if (c == 0) mvx2 += mp * vn * vn;
                }
            } else {
                const double vh = v[q];
                const double acc = fma(-gamma, vh, F[c]) * im;
                const double vn = fma(hdt, acc, vh);
                if (SAMPLE) {
                    res = fmax(res, fmax(fabs(F[c]), fabs(vn)));
                    ke += 0.5 * mp * vn * vn;
                    if (c == 0) mvx2 += mp * vn * vn;
                    bad |= !isfinite(vn) || !isfinite(x[q]);
                }
                if constexpr (MODE == FG_DRIFT) {
                    const double vh2 = fma(hdt, acc, vn);
                    const double xn = fma(dt, vh2, x[q]);
                    v[q] = vh2;
                    x[q] = xn;
                    xf[q] = dbl_to_fix(xn, S, over);
                } else {
                    a[q] = acc;
                    v[q] = vn;
                }
            }
        }
        if (over) atomicOr(status, 2);
        if (SAMPLE && bad) atomicOr(status, 1);
    }
    if (SAMPLE) {
        const double t0 = fbsum(mvx2, sh);
        const double t1 = fbsum(ke, sh);
        const double t2 = fbsum(react, sh);
        const double t3 = fbmax(res, sh);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = t0;
            part[nblk + blockIdx.x] = t1;
            part[2 * nblk + blockIdx.x] = t2;
            part[3 * nblk + blockIdx.x] = t3;
        }
    }
}

// ------------------------------------------------------------------ host

static ff split_ff_c(double v)
{
    const float hi = (float)v;
    return ff{hi, (float)(v - (double)hi)};
}

static FixTab fix_tab(const Ctx &c)
{
    FixTab T{};
    T.S = c.fix_S;
    T.p24 = ldexpf(1.0f, 24 - c.fix_S);
    T.p0 = ldexpf(1.0f, -c.fix_S);
    const int no = (int)c.h.offv.size() / 3;
    for (int q = 0; q < no && q < 9; q++) {
        double oo = 0.0;
        for (int k = 0; k < 3; k++) {
            T.o[q][k] = std::llround(std::ldexp(c.h.offv[3 * q + k], c.fix_S));
            const double of = std::ldexp((double)T.o[q][k], -c.fix_S);  // exact
            T.of[q][k] = split_ff_c(of);
            oo += of * of;
        }
        T.oo[q] = split_ff_c(oo);
    }
    return T;
}

cudaError_t fixcsr_upload(Ctx &c)
{
    const HostNet &h = c.h;
    const int64_t n = c.n, m = c.m, dn = (int64_t)h.dim * n;
    int maxext = std::max(h.nx, std::max(h.ny, h.nz));
    const double extent = 4.0 * maxext * h.a + 16.0;
    // also every intact spring vector (up to the longest critical length)
    // below 2^48 in fixed point, so that it converts to a double-float in two
    // exact 24-bit chunks
    c.fix_S = std::min({52, 61 - (int)std::ceil(std::log2(extent)),
                        47 - (int)std::ceil(std::log2(h.a * std::sqrt(2.0))),
                        47 - (int)std::floor(std::log2(max_critical_length(h.types)))});
    c.a_fix = std::llround(std::ldexp(h.a, c.fix_S));
    std::vector<TypeDF> tdf(h.types.size());
    for (size_t q = 0; q < h.types.size(); q++) {
        const SpringType &t = h.types[q];
        // -r0^2 to double-float accuracy: r0^2 = p + pe exactly (fma)
        const double p = t.r0 * t.r0, pe = std::fma(t.r0, t.r0, -p);
        const float hi = (float)(-p);
        tdf[q].k = split_ff_c(t.k);
        tdf[q].r0 = split_ff_c(t.r0);
        tdf[q].rc2 = split_ff_c(t.rc2);
        tdf[q].cor = ff{hi, (float)((-p - (double)hi) - pe)};
    }
    std::vector<double> im(n);
    for (int64_t p = 0; p < n; p++) im[p] = 1.0 / h.mass[p];
    const size_t fsz = c.h.precision == LSM_PREC_F32 ? sizeof(float) : sizeof(ff);
    cudaError_t e;
    if ((e = lsm::dev_malloc((void **)&c.xf, (dn ? dn : 1) * sizeof(long long))) != cudaSuccess) return e;
    if ((e = lsm::dev_malloc((void **)&c.sdir, m ? m : 1)) != cudaSuccess) return e;
    if ((e = lsm::dev_malloc((void **)&c.imass, (n ? n : 1) * sizeof(double))) != cudaSuccess) return e;
    if ((e = lsm::dev_malloc((void **)&c.tdf, (tdf.size() ? tdf.size() : 1) * sizeof(TypeDF))) != cudaSuccess) return e;
    if ((e = lsm::dev_malloc(&c.fsx, (size_t)h.dim * (m ? m : 1) * fsz)) != cudaSuccess) return e;
    cudaStream_t st = c.stream;
    if (m && (e = cudaMemcpyAsync(c.sdir, h.sdir.data(), m, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(c.imass, im.data(), n * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(c.tdf, tdf.data(), tdf.size() * sizeof(TypeDF), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(c.fsx, 0, (size_t)h.dim * (m ? m : 1) * fsz, st)) != cudaSuccess) return e;
    if ((e = fixcsr_refresh(c)) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t fixcsr_refresh(Ctx &c)
{
    const int64_t total = (int64_t)c.dim * c.n;
    if (total == 0) return cudaSuccess;
    k_fix<<<(unsigned)((total + FTPB - 1) / FTPB), FTPB, 0, c.stream>>>(total, c.x, c.xf, c.fix_S, c.d_status);
    return cudaGetLastError();
}

template <int DIM, int PREC, bool BREAK, bool SAMPLE>
static void springs_fix_p(Ctx &c)
{
    if (c.m == 0) {
        if (SAMPLE) cudaMemsetAsync(c.part_s, 0, 2 * sizeof(double), c.stream);
        return;
    }
    k_springs_fix<DIM, PREC, BREAK, SAMPLE><<<(unsigned)((c.m + FTPB - 1) / FTPB), FTPB, 0, c.stream>>>(
        c.m, c.n, c.si, c.sj, c.stype, c.sdir, c.tdf, c.state, c.brk, c.xf, c.fsx, c.d_step, c.d_first_break,
        c.d_nbroken, c.part_s, c.nblk_s, fix_tab(c));
}

template <int DIM, bool BREAK, bool SAMPLE>
void springs_fix(Ctx &c)
{
    if (c.h.precision == LSM_PREC_F32)
        springs_fix_p<DIM, LSM_PREC_F32, BREAK, SAMPLE>(c);
    else
        springs_fix_p<DIM, LSM_PREC_DF, BREAK, SAMPLE>(c);
}

template <int DIM, int MODE, bool SAMPLE>
void gather_fix(Ctx &c)
{
    const double dt = c.h.dt, hdt = 0.5 * c.h.dt;
    const unsigned g = (unsigned)((c.n + FTPB - 1) / FTPB);
    if (c.h.precision == LSM_PREC_F32)
        k_gather_fix<DIM, LSM_PREC_F32, MODE, SAMPLE><<<g, FTPB, 0, c.stream>>>(
            c.n, c.m, c.row, c.inc, c.fsx, c.x, c.v, c.a, c.xf, c.mass, c.imass, c.fixm, c.grip, dt, hdt,
            c.h.damping, c.part_p, c.nblk_p, c.d_status, c.d_step, c.fix_S);
    else
        k_gather_fix<DIM, LSM_PREC_DF, MODE, SAMPLE><<<g, FTPB, 0, c.stream>>>(
            c.n, c.m, c.row, c.inc, c.fsx, c.x, c.v, c.a, c.xf, c.mass, c.imass, c.fixm, c.grip, dt, hdt,
            c.h.damping, c.part_p, c.nblk_p, c.d_status, c.d_step, c.fix_S);
}

// explicit instantiations used by kernels.cu
template void springs_fix<2, true, true>(Ctx &);
template void springs_fix<2, true, false>(Ctx &);
template void springs_fix<2, false, true>(Ctx &);
template void springs_fix<2, false, false>(Ctx &);
template void springs_fix<3, true, true>(Ctx &);
template void springs_fix<3, true, false>(Ctx &);
template void springs_fix<3, false, true>(Ctx &);
template void springs_fix<3, false, false>(Ctx &);
template void gather_fix<2, FG_END, true>(Ctx &);
template void gather_fix<2, FG_DRIFT, false>(Ctx &);
template void gather_fix<2, FG_INIT, false>(Ctx &);
template void gather_fix<2, FG_OBSERVE, true>(Ctx &);
template void gather_fix<3, FG_END, true>(Ctx &);
template void gather_fix<3, FG_DRIFT, false>(Ctx &);
template void gather_fix<3, FG_INIT, false>(Ctx &);
template void gather_fix<3, FG_OBSERVE, true>(Ctx &);

}  // namespace lsm
