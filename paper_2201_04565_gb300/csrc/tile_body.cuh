// tile_body.cuh -- the per-tile time step shared by the single-specimen and
// the batched 2D kernels (see tile2d.cu for the method and the layout).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "dfloat.cuh"
#include "lsm_internal.h"

namespace lsm {


namespace {

// Threads per CTA for a tile of height TY: one warp per tile row, up to 16
// warps for the double-float time step (16- and 32-row tiles of the batched
// kernel) and 8 otherwise (fewer warps per barrier; the sample step needs
// more registers).
template <int TY, int PREC, bool SAMPLE>
__host__ __device__ constexpr int tile_threads()
{
    return 32 * (TY < (PREC == LSM_PREC_DF && !SAMPLE ? 16 : 8) ? TY : (PREC == LSM_PREC_DF && !SAMPLE ? 16 : 8));
}

__device__ __forceinline__ double ad(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sb(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ml(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dv(double a, double b) { return __ddiv_rn(a, b); }

template <int NWARP>
__device__ __forceinline__ double bsum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NWARP; q++) t += sh[q];
    return t;
}

template <int NWARP>
__device__ __forceinline__ double bmax(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NWARP; q++) t = fmax(t, sh[q]);
    return t;
}

// Fixed-order block sum of a double-float per thread: the warp tree in
// double-float arithmetic (FP32 pipe), then the warps' totals in FP64 by
// thread 0. Deterministic for a given block size.
template <int NWARP>
__device__ __forceinline__ double bsum_ff(ff v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) {
        const ff w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = ff_add_sloppy(v, w);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ff_to_double(v);
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NWARP; q++) t += sh[q];
    return t;
}

template <int NWARP>
__device__ __forceinline__ double bmax_f(float v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = f2d_bits(v);
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NWARP; q++) t = fmax(t, sh[q]);
    return t;
}

}  // namespace

enum { T_STEP = 0, T_INIT = 1, T_OBSERVE = 2 };

// Per-phase integration coefficients: vh' = c1 vh + c2 F is vh + dt (F - g vh)/m,
// and c1h, c2h the same for a half step.
struct Coef4 {
    double c1, c2, c1h, c2h;
};

struct TileArgs {
    int nx, ny, nphase;
    int64_t np;
    const double *x_in, *vh_in;
    double *x_out, *vh_out, *v_obs;
    const uint8_t *phase;
    uint8_t *mask;
    long long *brk;  // [4][np]
    const SpringType *types;
    const TypeDF *tdf;         // double-float copies of the spring types
    const double *mass;        // per phase
    const Coef4 *coef;         // per phase integration coefficients
    int S;                     // fixed-point scale: positions as x * 2^S
    long long a_fix;           // lattice spacing in fixed point
    long long h_fix;           // triangular packing: row height a sqrt(3)/2 in fixed point
    double hrow;               // triangular packing: row height
    float p24, p0;             // 2^(24-S), 2^-S
    unsigned df_bias;          // DF: f2d_force_scaled bias for forces held in units of p24
    double dt, hdt, gamma, a;
    int grip_mode;
    int rate_on;               // constant strain rate: grips at rate_eps0 + (s - rate_step0) rate_dt
    double rate_eps0, rate_dt, xc;
    long long rate_step0;
    const long long *d_step;  // steps completed before this graph launch
    int64_t t_off;            // index of this step within the launch
    unsigned long long *first_break, *nbroken;
    int *status;
    double *part_s, *part_p;
    int64_t ntiles;
};

// CTAs per SM the 8- and 16-row tile kernels are compiled for: 3 of 16
// warps for the 16-row double-float time step, 6 of 8 warps for the other
// double-float, FP32 and FAST64 steps, 5 for the exact FP64 step, 4 of 8
// warps for every sample step (the register budgets that leave, 42, 51 and 64
// per thread, hold each kernel without spills, up to 12 bytes in the batched
// FP32 step)
template <int TY, int PREC, bool SAMPLE>
__host__ __device__ constexpr int tile_min_ctas()
{
    return TY != 8 && TY != 16       ? 1
           : SAMPLE                  ? 4
           : PREC == LSM_PREC_DF     ? (TY == 16 ? 3 : 6)
           : PREC == LSM_PREC_EXACT64 ? 5
                                     : 6;
}

// Cascaded double-float sum (Ogita, Rump and Oishi, 2005) of a particle's
// spring forces in the canonical order: a TwoSum chain over the high parts,
// with their errors and the low parts summed in float. value() is the sum
// as a double (exact conversion of both parts, one FP64 addition).
struct DfSum {
    float hs, el;
    __device__ __forceinline__ void first_neg(ff t)
    {
        hs = -t.hi;
        el = -t.lo;
    }
    __device__ __forceinline__ void sub(ff o)
    {
        const ff t = two_sum(hs, -o.hi);
        hs = t.hi;
        el = __fadd_rn(el, __fsub_rn(t.lo, o.lo));
    }
    __device__ __forceinline__ void add(ff o)
    {
        const ff t = two_sum(hs, o.hi);
        hs = t.hi;
        el = __fadd_rn(el, __fadd_rn(t.lo, o.lo));
    }
    // the sum as a double; bias: the unit the terms are held in (f2d_force_scaled)
    __device__ __forceinline__ double value(unsigned bias) const
    {
        return f2d_force_scaled(hs, bias) + f2d_force_scaled(el, bias);
    }
};

// The fixed-point modes' spring arithmetic, shared by every 2D kernel that
// evaluates springs (tile, strip and batched kernels), so that all of them
// produce the same bits. Input: the exact fixed-point spring vector
// (dxq, dyq) = x_q - x_p of an intact spring of type t in forward slot
// `slot`. Returns true when the break test (TEST) fires: r^2 > rc^2, the
// force is then left at zero. Otherwise writes the force on the lower
// endpoint, f = k (1 - r0/r) d (Eq. 2), and with SAMPLE the spring's x
// component d_x and its stretch r - r0.

// Double-float force: d as a double-float (two exact 24-bit chunks), 1/r by
// one double-float Newton step, k (r - r0) / r = k (1 - r0 / r). Lengths are
// held in units of 2^(24-S) (fix_to_ff_u24; the type table's r0 and rc^2 are
// scaled to match on the host), so the force, d_x and r - r0 come out in that
// unit too: exactly the unscaled values times 2^(S-24).
template <bool TEST, bool SAMPLE>
__device__ __forceinline__ bool spring_df(long long dxq, long long dyq, const TypeDF &t, const TileArgs &A,
                                          ff &fx, ff &fy, ff &dx, ff &st)
{
    const ff dxf = fix_to_ff_u24(dxq);
    const ff dyf = fix_to_ff_u24(dyq);
    const ff r2 = ff_norm2_un(dxf, dyf);
    if (TEST && ff_gt_un(r2, t.rc2)) return true;
    ff y;
    const ff g = ff_spring_g(r2, t.r0, SAMPLE ? &y : nullptr);
    const ff c = ff_mul_un(t.k, g);  // the products stay unnormalised: they are only
    fx = ff_mul_un(c, dxf);          // multiplied or summed further (DfSum)
    fy = ff_mul_un(c, dyf);
    if (SAMPLE) {
        dx = dxf;
        st = ff_mul(ff_mul(r2, y), g);  // r - r0
    }
    return false;
}

// Single-precision force: the deviation e = d - o from the slot's lattice
// vector o is exact in fixed point, so r^2 - |o|^2 = (2 o + e).e carries no
// cancellation in float. Products are explicitly rounded (no contraction
// with the caller's sums, whatever the kernel).
// (ofx, ofy): the slot's lattice vector in fixed point, (ox, oy, oo) the
// same as floats with |o|^2; t.cor = |o|^2 - r0^2 for that vector.
template <bool TEST, bool SAMPLE>
__device__ __forceinline__ bool spring_f32_o(long long dxq, long long dyq, long long ofx, long long ofy, float ox,
                                             float oy, float oo, const TypeDF &t, const TileArgs &A, float &fx,
                                             float &fy, float &dx, float &st)
{
    const long long exf = dxq - ofx;
    const long long eyf = dyq - ofy;
    const float ex = fix_to_float_i2f(exf, A.p24, A.p0), ey = fix_to_float_i2f(eyf, A.p24, A.p0);
    const float dxf = __fadd_rn(ox, ex), dyf = __fadd_rn(oy, ey);
    const float num = __fmaf_rn(__fadd_rn(__fmul_rn(2.0f, ox), ex), ex,
                                __fmaf_rn(__fadd_rn(__fmul_rn(2.0f, oy), ey), ey, t.cor.hi));
    const float r2f = __fadd_rn(oo, num);
    if (TEST && r2f > t.rc2.hi) return true;
    const float ir = rsqrt_approx(r2f);
    const float s = __fdividef(num, __fmaf_rn(r2f, ir, t.r0.hi));  // r - r0
    const float c = __fmul_rn(__fmul_rn(t.k.hi, s), ir);
    fx = __fmul_rn(c, dxf);
    fy = __fmul_rn(c, dyf);
    if (SAMPLE) {
        dx = dxf;
        st = s;
    }
    return false;
}

// The square lattice's forward slots (+1,0), (-1,+1), (0,+1), (+1,+1).
template <bool TEST, bool SAMPLE>
__device__ __forceinline__ bool spring_f32(long long dxq, long long dyq, int slot, const TypeDF &t,
                                           const ff (*soff)[3], const TileArgs &A, float &fx, float &fy,
                                           float &dx, float &st)
{
    const int ox_i = slot == 0 ? 1 : (slot == 1 ? -1 : (slot == 2 ? 0 : 1));
    const int oy_i = slot == 0 ? 0 : 1;
    return spring_f32_o<TEST, SAMPLE>(dxq, dyq, (long long)ox_i * A.a_fix, (long long)oy_i * A.a_fix,
                                      soff[slot][0].hi, soff[slot][1].hi, soff[slot][2].hi, t, A, fx, fy, dx, st);
}

// Force on the lower endpoint of one spring (rp -> rq, forward slot), with
// the break test. Writes the force into sf; OWNER adds the sample sums and
// records a break (only the tile owning the lower endpoint does).
template <int PREC, int MODE, bool SAMPLE, bool OWNER, int NR, int NS, typename FT, typename AT>
__device__ __forceinline__ void eval_spring(const TileArgs &A, int rp, int rq, int slot, const double *sx,
                                            const double *sy, const long long *sxf, const long long *syf,
                                            const uint8_t *sph, const uint8_t *smk, FT *sf,
                                            const SpringType *stab, const TypeDF *sdf, const ff (*soff)[3],
                                            int *snew, int64_t gsrc, long long step_now, AT &w_acc,
                                            AT &u_acc)
{
    FT fx{}, fy{};
    const uint8_t pp = sph[rp], pq = sph[rq];
    const uint8_t mk = smk[rp];
    if (pp && pq && !((mk >> slot) & 1)) {
        const int ti = (((pp - 1) * A.nphase) + (pq - 1)) * 2 + (slot & 1);
        bool brk_now = false;
        if constexpr (PREC == LSM_PREC_EXACT64) {
            const SpringType t = stab[ti];
            const double ddx = sb(sx[rq], sx[rp]), ddy = sb(sy[rq], sy[rp]);
            const double r2 = ad(ml(ddx, ddx), ml(ddy, ddy));
            if (MODE == T_STEP && r2 > t.rc2) {
                brk_now = true;
            } else {
                const double r = __dsqrt_rn(r2);
                const double c = dv(ml(t.k, sb(r, t.r0)), r);
                fx = ml(c, ddx);
                fy = ml(c, ddy);
                if (SAMPLE && OWNER) {
                    const double st = sb(r, t.r0);
                    u_acc += ml(ml(ml(0.5, t.k), st), st);
                    w_acc += ml(ddx, ml(c, ddx));
                }
            }
        } else if constexpr (PREC == LSM_PREC_FAST64) {
            const SpringType t = stab[ti];
            const double ddx = sx[rq] - sx[rp], ddy = sy[rq] - sy[rp];
            const double r2 = fma(ddx, ddx, ddy * ddy);
            if (MODE == T_STEP && r2 > t.rc2) {
                brk_now = true;
            } else {
                const double ir = rsqrt(r2);
                const double c = fma(-t.kr0, ir, t.k);
                fx = c * ddx;
                fy = c * ddy;
                if (SAMPLE && OWNER) {
                    const double st = fma(r2, ir, -t.r0);
                    u_acc += 0.5 * t.k * st * st;
                    w_acc += ddx * fx;
                }
            }
        } else {
            const TypeDF t = sdf[ti];
            if constexpr (PREC == LSM_PREC_F32) {
                float dxf, st;
                brk_now = spring_f32<MODE == T_STEP, SAMPLE && OWNER>(sxf[rq] - sxf[rp], syf[rq] - syf[rp], slot,
                                                                      t, soff, A, fx, fy, dxf, st);
                if (SAMPLE && OWNER && !brk_now) {  // double-float sums: no FP64 pipe work per spring
                    u_acc = ff_add_f(u_acc, 0.5f * t.k.hi * st * st);
                    w_acc = ff_add_f(w_acc, dxf * fx);
                }
            } else {  // LSM_PREC_DF
                ff dxf, st;
                brk_now = spring_df<MODE == T_STEP, SAMPLE && OWNER>(sxf[rq] - sxf[rp], syf[rq] - syf[rp], t, A,
                                                                     fx, fy, dxf, st);
                if (SAMPLE && OWNER && !brk_now) {  // double-float sums: no FP64 pipe work per spring
                    u_acc = ff_add_sloppy(u_acc, ff_mul(ff_mul_f(t.k, 0.5f), ff_sqr(st)));
                    w_acc = ff_add_sloppy(w_acc, ff_mul(dxf, fx));
                }
            }
        }
        if (OWNER && brk_now) {
            atomicOr(&snew[rp], 1 << slot);
            A.brk[(int64_t)slot * A.np + gsrc] = step_now;
            atomicMin(A.first_break, (unsigned long long)step_now);
            atomicAdd(A.nbroken, 1ull);
        }
    }
    sf[(0 * 4 + slot) * NS + rp] = fx;
    sf[(1 * 4 + slot) * NS + rp] = fy;
}

// Constant strain rate: x of a grip in column gx at the strain of the step
// being computed, eps = eps0 + (s - s0) rate dt, x = X + eps (X - xc)
// (correctly rounded operations); the kernels evaluate it for the two grip
// columns once and pass the results to the region load.
__device__ __forceinline__ double tile_rate_x(const TileArgs &A, int gx)
{
    const long long s = *A.d_step + A.t_off + 1 - A.rate_step0;
    const double eps = ad(A.rate_eps0, ml((double)s, A.rate_dt));
    const double X = ml((double)gx, A.a);
    return ad(X, ml(eps, sb(X, A.xc)));
}

// Region pixel (rx, ry) -> shared memory: phase, broken mask, and the
// positions drifted by dt vh (step mode): as doubles in the FP64 modes, as
// fixed-point copies in the F32/DF modes. The drifted position is also
// returned (the owning thread keeps it in registers for the integration).
// rate_l, rate_r: the grips' x under the constant strain rate (RATE).
template <int PREC, int MODE, int RX, bool RATE>
__device__ __forceinline__ void load_pixel(const TileArgs &A, int x0, int y0, int rx, int ry, double *sx,
                                           double *sy, long long *sxf, long long *syf, uint8_t *sph,
                                           uint8_t *smk, bool &over, double &opx, double &opy, double rate_l,
                                           double rate_r)
{
    constexpr bool FIX = PREC == LSM_PREC_F32 || PREC == LSM_PREC_DF;
    const int gx = x0 - 1 + rx, gy = y0 - 1 + ry;
    const int e = ry * RX + rx;
    uint8_t ph = 0, mk = 0;
    double px = 0.0, py = 0.0;
    if (gx >= 0 && gx < A.nx && gy >= 0 && gy < A.ny) {
        const int64_t g = (int64_t)gy * A.nx + gx;
        ph = A.phase[g];
        if (ph) {
            mk = A.mask[g];
            px = A.x_in[g];
            py = A.x_in[A.np + g];
            if (MODE == T_STEP) {
                const bool grip = gx == 0 || gx == A.nx - 1;
                if (RATE && grip) px = gx == 0 ? rate_l : rate_r;  // constant strain rate
                if (!grip) {
                    if constexpr (PREC == LSM_PREC_EXACT64) px = ad(px, ml(A.dt, A.vh_in[g]));
                    else px = fma(A.dt, A.vh_in[g], px);
                }
                if (!(grip && A.grip_mode == 1)) {
                    if constexpr (PREC == LSM_PREC_EXACT64) py = ad(py, ml(A.dt, A.vh_in[A.np + g]));
                    else py = fma(A.dt, A.vh_in[A.np + g], py);
                }
            }
        }
    }
    opx = px;
    opy = py;
    if constexpr (FIX) {
        sxf[e] = dbl_to_fix(px, A.S, over);
        syf[e] = dbl_to_fix(py, A.S, over);
    } else {
        sx[e] = px;
        sy[e] = py;
    }
    sph[e] = ph;
    smk[e] = mk;
}

// One CTA step of one 32 x TY tile (tile coordinates bx, by; tile_id indexes
// the per-tile partial sums); warp w handles tile rows w, w + 8, ...
template <int TX, int TY, int PREC, int MODE, bool SAMPLE, bool RATE = false>
__device__ __forceinline__ void tile_body(const TileArgs &A, int bx, int by, int64_t tile_id,
                                          unsigned char *smem_raw)
{
    static_assert(TX == 32, "one warp per tile row");
    constexpr int RX = TX + 2, RY = TY + 2;   // region = tile + 1-pixel halo
    constexpr int NR = RX * RY;
    constexpr int NS = RX * (TY + 1);         // spring sources: region rows 0..TY
    constexpr int NT = tile_threads<TY, PREC, SAMPLE>();
    constexpr int NW = NT / 32;
    static_assert(TY % NW == 0, "whole rows per warp");
    constexpr bool FIX = PREC == LSM_PREC_F32 || PREC == LSM_PREC_DF;
    using FT = typename std::conditional<PREC == LSM_PREC_F32, float,
               typename std::conditional<PREC == LSM_PREC_DF, ff, double>::type>::type;

    constexpr int NRD = FIX ? 0 : NR;              // FP64 modes: positions as doubles
    double *sx = (double *)smem_raw;               // [NRD] drifted positions
    double *sy = sx + NRD;                         // [NRD]
    long long *sxf = (long long *)(sy + NRD);      // [NR] fixed point (FIX modes only)
    long long *syf = sxf + (FIX ? NR : 0);         // [NR]
    FT *sf = (FT *)(syf + (FIX ? NR : 0));         // [2][4][NS] force on the lower end
    int *snew = (int *)(sf + 8 * NS);              // [NS] springs broken in this step
    uint8_t *sph = (uint8_t *)(snew + NS);         // [NR]
    uint8_t *smk = sph + NR;                       // [NR]
    __shared__ double sred[NW];
    __shared__ SpringType stab[FIX ? 1 : 128];
    __shared__ TypeDF sdf[FIX ? 128 : 1];
    __shared__ ff soff[4][3];  // per slot: o_x, o_y, |o|^2 as double-floats
    __shared__ double smass[8];
    __shared__ float smassf[8];
    __shared__ Coef4 scoef[8];  // per phase: c1, c2, c1h, c2h (vh' = c1 vh + c2 F)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = bx * TX, y0 = by * TY;
    const int nt = 2 * A.nphase * A.nphase;
    for (int q = tid; q < nt; q += NT) {
        if constexpr (FIX)
            sdf[q] = A.tdf[q];
        else
            stab[q] = A.types[q];
    }
    if (tid < A.nphase) {
        smass[tid] = A.mass[tid];
        smassf[tid] = (float)A.mass[tid];
        scoef[tid] = A.coef[tid];
    }
    if (FIX && tid < 4) {
        const int dx = tid == 0 ? 1 : (tid == 1 ? -1 : (tid == 2 ? 0 : 1));
        const int dy = tid == 0 ? 0 : 1;
        const ff ox = fix_to_ff((long long)dx * A.a_fix, A.S), oy = fix_to_ff((long long)dy * A.a_fix, A.S);
        soff[tid][0] = ox;
        soff[tid][1] = oy;
        soff[tid][2] = ff_add(ff_mul(ox, ox), ff_mul(oy, oy));
    }
    const long long step_now = MODE == T_STEP ? *A.d_step + A.t_off : 0;

    // 1. region load (+ drift): tile columns by lanes, halo columns apart
    // region rows warp, warp + NW, ...: the thread keeps its column's
    // drifted positions in registers for phase 3 (it owns those pixels)
    constexpr int KR = (RY + NW - 1) / NW;
    double opx[KR], opy[KR];
    bool over = false;
    double rate_l = 0.0, rate_r = 0.0;  // grips' x under the constant strain rate
    if constexpr (RATE && MODE == T_STEP) {
        rate_l = tile_rate_x(A, 0);
        rate_r = tile_rate_x(A, A.nx - 1);
    }
#pragma unroll
    for (int k = 0; k < KR; k++) {
        const int ry = warp + k * NW;
        if (ry < RY)
            load_pixel<PREC, MODE, RX, RATE>(A, x0, y0, lane + 1, ry, sx, sy, sxf, syf, sph, smk, over, opx[k], opy[k],
                                             rate_l, rate_r);
    }
    for (int q = tid; q < 2 * RY; q += NT) {
        double hx, hy;
        load_pixel<PREC, MODE, RX, RATE>(A, x0, y0, (q & 1) ? TX + 1 : 0, q >> 1, sx, sy, sxf, syf, sph, smk, over, hx,
                                         hy, rate_l, rate_r);
    }
    if (FIX && over) atomicOr(A.status, 2);
    for (int e = tid; e < NS; e += NT) snew[e] = 0;
    __syncthreads();

    // 2a. forward springs of the owned particles
    using AT = typename std::conditional<FIX, ff, double>::type;  // per-thread sample sums
    AT w_acc{}, u_acc{};
    constexpr int dq[4] = {1, RX - 1, RX, RX + 1};
#pragma unroll
    for (int k = 0; k < TY / NW; k++) {
        const int ry = warp + k * NW + 1, rx = lane + 1;
        const int rp = ry * RX + rx;
        const int64_t g = (int64_t)(y0 + ry - 1) * A.nx + (x0 + lane);
#pragma unroll
        for (int slot = 0; slot < 4; slot++)
            eval_spring<PREC, MODE, SAMPLE, true, NR, NS>(A, rp, rp + dq[slot], slot, sx, sy, sxf, syf, sph, smk,
                                                          sf, stab, sdf, soff, snew, g, step_now, w_acc, u_acc);
    }
    // 2b. springs from halo sources into the tile (also evaluated, with the
    // same result, by the tile that owns their lower endpoint)
    constexpr int NH = 3 * TX + 3 * TY - 2;
    for (int t = tid; t < NH; t += NT) {
        int rx, ry, slot;
        if (t < 3 * TX) {  // halo row above the tile, slots 1..3
            slot = 1 + t / TX;
            const int j = t % TX;
            rx = slot == 2 ? j + 1 : (slot == 3 ? j : j + 2);
            ry = 0;
        } else if (t < 3 * TX + TY) {  // left halo column, slot 0
            slot = 0; rx = 0; ry = 1 + (t - 3 * TX);
        } else if (t < 3 * TX + 2 * TY - 1) {  // left halo column, slot 3
            slot = 3; rx = 0; ry = 1 + (t - 3 * TX - TY);
        } else {  // right halo column, slot 1
            slot = 1; rx = TX + 1; ry = 1 + (t - 3 * TX - 2 * TY + 1);
        }
        const int rp = ry * RX + rx;
        eval_spring<PREC, MODE, SAMPLE, false, NR, NS>(A, rp, rp + dq[slot], slot, sx, sy, sxf, syf, sph, smk, sf,
                                                       stab, sdf, soff, snew, 0, step_now, w_acc, u_acc);
    }
    __syncthreads();

    // 3. gather + integrate the owned particles
    double mvx2 = 0.0, ke = 0.0, react = 0.0, res = 0.0;
    float mvx2f = 0.0f, kef = 0.0f, resf = 0.0f;  // fixed-point modes
    ff reactf{0.0f, 0.0f};
    bool bad = false;
#pragma unroll
    for (int k = 0; k < KR; k++) {
        const int ry = warp + k * NW, ly = ry - 1;  // the rows loaded into registers above
        if (ry < 1 || ry > TY) continue;
        const int gx = x0 + lane, gy = y0 + ly;
        const int rx = lane + 1;
        const int rp = ry * RX + rx;
        if (gx >= A.nx || gy >= A.ny || !sph[rp]) continue;
        const int64_t g = (int64_t)gy * A.nx + gx;
        // incoming springs come from p - o for slots 3, 2, 1, 0 (ascending
        // source index), then the outgoing ones in slot order
        const int s3 = rp - RX - 1, s2 = rp - RX, s1 = rp - RX + 1, s0 = rp - 1;
        double F[2];
        float Ff[2];  // F as floats (fixed-point modes: sample statistics without FP64 work)
        ff Fd[2];     // F as double-floats (fixed-point modes: the grip reaction)
        if constexpr (PREC == LSM_PREC_EXACT64) {
#pragma unroll
            for (int c = 0; c < 2; c++) {
                double acc = 0.0;
                acc = sb(acc, sf[(c * 4 + 3) * NS + s3]);
                acc = sb(acc, sf[(c * 4 + 2) * NS + s2]);
                acc = sb(acc, sf[(c * 4 + 1) * NS + s1]);
                acc = sb(acc, sf[(c * 4 + 0) * NS + s0]);
#pragma unroll
                for (int sl = 0; sl < 4; sl++) acc = ad(acc, sf[(c * 4 + sl) * NS + rp]);
                F[c] = acc;
            }
        } else if constexpr (PREC == LSM_PREC_DF) {
            // cascaded summation in the fixed order above (DfSum)
#pragma unroll
            for (int c = 0; c < 2; c++) {
                DfSum acc;
                acc.first_neg(sf[(c * 4 + 3) * NS + s3]);
                acc.sub(sf[(c * 4 + 2) * NS + s2]);
                acc.sub(sf[(c * 4 + 1) * NS + s1]);
                acc.sub(sf[(c * 4 + 0) * NS + s0]);
#pragma unroll
                for (int sl = 0; sl < 4; sl++) acc.add(sf[(c * 4 + sl) * NS + rp]);
                F[c] = acc.value(A.df_bias);
                Ff[c] = __fmul_rn(__fadd_rn(acc.hs, acc.el), A.p24);  // back from units of 2^(24-S)
                Fd[c] = ff{acc.hs, acc.el};                            // (in those units)
            }
        } else {
#pragma unroll
            for (int c = 0; c < 2; c++) {
                // (o0 - i3) + (o1 - i2) + (o2 - i1) + (o3 - i0), outgoing slot
                // s paired with the incoming spring of slot 3 - s
                FT acc = sf[(c * 4 + 0) * NS + rp] - sf[(c * 4 + 3) * NS + s3];
                acc += sf[(c * 4 + 1) * NS + rp] - sf[(c * 4 + 2) * NS + s2];
                acc += sf[(c * 4 + 2) * NS + rp] - sf[(c * 4 + 1) * NS + s1];
                acc += sf[(c * 4 + 3) * NS + rp] - sf[(c * 4 + 0) * NS + s0];
                if constexpr (PREC == LSM_PREC_F32) {
                    F[c] = f2d_force(acc);
                    Ff[c] = acc;
                    Fd[c] = ff{acc, 0.0f};
                } else {
                    F[c] = acc;
                }
            }
        }
        const bool grip = gx == 0 || gx == A.nx - 1;
        const bool fixx = grip, fixy = grip && A.grip_mode == 1;
        const int ph = sph[rp] - 1;
        const double m = smass[ph];
        const double xr[2] = {opx[k], opy[k]};
        if (SAMPLE && gx == A.nx - 1) {
            if constexpr (PREC == LSM_PREC_EXACT64) react = sb(react, F[0]);
            else if constexpr (FIX) reactf = ff_add_sloppy(reactf, ff_neg(Fd[0]));
            else react -= F[0];
        }
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const bool fixed = c == 0 ? fixx : fixy;
            const int64_t q = c * A.np + g;
            if (MODE == T_STEP) A.x_out[q] = xr[c];
            if (fixed) {
                if (MODE == T_STEP) A.vh_out[q] = 0.0;
                if (MODE == T_STEP && SAMPLE) A.v_obs[q] = 0.0;
                continue;
            }
            if (MODE == T_OBSERVE) {
                const double vn = A.v_obs[q];
                if (SAMPLE) {
                    if constexpr (FIX) {
                        const float vf = d2f_bits(vn);
                        resf = fmaxf(resf, fmaxf(fabsf(Ff[c]), fabsf(vf)));
                        kef = fmaf(0.5f * smassf[ph] * vf, vf, kef);
                        if (c == 0) mvx2f = fmaf(smassf[ph] * vf, vf, mvx2f);
                    } else {
                        res = fmax(res, fmax(fabs(F[c]), fabs(vn)));
                        ke += 0.5 * m * vn * vn;
                        if (c == 0) mvx2 += m * vn * vn;
                    }
                }
                continue;
            }
            const double vh = MODE == T_INIT ? A.v_obs[q] : A.vh_in[q];
            double vn, vh2;
            if constexpr (PREC == LSM_PREC_EXACT64) {
                const double acc = dv(sb(F[c], ml(A.gamma, vh)), m);
                vn = ad(vh, ml(A.hdt, acc));
                vh2 = ad(vn, ml(A.hdt, acc));
            } else {
                // vh + t (F - gamma vh) / m = (1 - t gamma / m) vh + (t / m) F
                const Coef4 k4 = scoef[ph];
                vn = fma(k4.c2h, F[c], k4.c1h * vh);
                vh2 = fma(k4.c2, F[c], k4.c1 * vh);
            }
            if (MODE == T_INIT) {
                // vh = v + dt/2 a(t) with a from the forces at the current x
                A.vh_out[q] = vn;
                continue;
            }
            A.vh_out[q] = vh2;
            if (SAMPLE) {
                A.v_obs[q] = vn;
                if constexpr (FIX) {
                    // float statistics (residual, KE, m v_x^2): 2^-24 relative,
                    // and the FP64 pipe is left to the integration
                    const float vf = d2f_bits(vn);
                    resf = fmaxf(resf, fmaxf(fabsf(Ff[c]), fabsf(vf)));
                    kef = fmaf(0.5f * smassf[ph] * vf, vf, kef);
                    if (c == 0) mvx2f = fmaf(smassf[ph] * vf, vf, mvx2f);
                    bad |= !dbl_finite_bits(vn) || !dbl_finite_bits(xr[c]);
                } else {
                    res = fmax(res, fmax(fabs(F[c]), fabs(vn)));
                    ke += 0.5 * m * vn * vn;
                    if (c == 0) mvx2 += m * vn * vn;
                    bad |= !isfinite(vn) || !isfinite(xr[c]);
                }
            }
        }
        if (MODE == T_STEP) {
            const int nb = snew[rp];
            if (nb) A.mask[g] = (uint8_t)(smk[rp] | nb);
        }
    }
    if (SAMPLE) {
        if (bad) atomicOr(A.status, 1);
        double t0, t1, t2, t3, t4, t5;
        if constexpr (FIX) {  // warp trees on the FP32 pipe
            t0 = bsum_ff<NW>(w_acc, sred);
            t1 = bsum_ff<NW>(u_acc, sred);
            t2 = bsum_ff<NW>(ff{mvx2f, 0.0f}, sred);
            t3 = bsum_ff<NW>(ff{kef, 0.0f}, sred);
            t4 = bsum_ff<NW>(reactf, sred);
            t5 = bmax_f<NW>(resf, sred);
            if constexpr (PREC == LSM_PREC_DF) {  // from units of 2^(24-S) (exact)
                const double u = (double)A.p24;
                t0 *= u * u;
                t1 *= u * u;
                t4 *= u;
            }
        } else {
            t0 = bsum<NW>(w_acc, sred);
            t1 = bsum<NW>(u_acc, sred);
            t2 = bsum<NW>(mvx2, sred);
            t3 = bsum<NW>(ke, sred);
            t4 = bsum<NW>(react, sred);
            t5 = bmax<NW>(res, sred);
        }
        if (tid == 0) {
            A.part_s[tile_id] = t0;
            A.part_s[A.ntiles + tile_id] = t1;
            A.part_p[tile_id] = t2;
            A.part_p[A.ntiles + tile_id] = t3;
            A.part_p[2 * A.ntiles + tile_id] = t4;
            A.part_p[3 * A.ntiles + tile_id] = t5;
        }
    }
}


// strip2d.cu: the register-resident time step (fixed-point modes, square
// lattice); its positions, velocities and breaks are bit-identical to the
// tile kernel's (sample sums: per strip instead of per tile).
cudaError_t launch_strip(Ctx &c, const TileArgs &A, bool sample);
cudaError_t launch_strip_mode(Ctx &c, const TileArgs &A, int mode);  // T_INIT / T_OBSERVE, triangular packing

// Pixel-grid broken flags -> canonical spring order (defined in tile2d.cu).
__global__ void k_tile_export(int nx, int ny, int64_t np, const uint8_t *__restrict__ phase,
                              const uint8_t *__restrict__ mask, const long long *__restrict__ brk,
                              const int64_t *__restrict__ sbase, uint8_t *__restrict__ out_mask,
                              long long *__restrict__ out_brk, int tri);

// Shared memory of tile_body (dynamic part).
template <int TX, int TY>
constexpr size_t tile_smem_bytes(int prec)
{
    constexpr int RX = TX + 2, RY = TY + 2, SX = TX + 2, SY = TY + 1;  // sources: region rows 0..TY
    const bool fix = prec == LSM_PREC_F32 || prec == LSM_PREC_DF;
    const size_t fsz = prec == LSM_PREC_F32 ? sizeof(float) : sizeof(double);  // ff is 8 bytes
    return (fix ? 0 : (size_t)2 * RX * RY * sizeof(double)) + (fix ? (size_t)2 * RX * RY * sizeof(long long) : 0) +
           (size_t)8 * SX * SY * fsz + (size_t)SX * SY * sizeof(int) + (size_t)2 * RX * RY + 16;
}

}  // namespace lsm
