// strip_body.cuh -- the register-resident strip sweep shared by the
// single-specimen strip kernel (strip2d.cu) and the batched one (batch.cu).
//
// One warp sweeps a strip of 32 pixel columns (lane = column) and R rows
// from top to bottom, one row per iteration. Per row y it
//   1. takes row y + 1 (phase, broken flags, x and vh, fetched one
//      iteration ahead), drifts it, x(t+dt) = x + dt vh (Eq. 3), writes the
//      drifted position of owned pixels as the step's output and converts it
//      to 64-bit fixed point; then fetches row y + 2;
//   2. evaluates the four forward springs of every pixel of row y (slots
//      (+1,0), (-1,+1), (0,+1), (+1,+1); Eq. 2 with the break test): the
//      endpoints in the neighbouring columns come from the neighbouring
//      lanes by warp shuffles, so positions never pass through shared
//      memory and no barrier is needed;
//   3. gathers each owned particle's eight spring forces in the canonical
//      order (incoming springs by ascending source: slot 3, 2, 1 of row
//      y - 1, slot 0 of row y; then the outgoing slots 0..3), applies the
//      damped half-kicks (Eqs. 4-5) and writes vh(t + 3dt/2).
// Forces of row y's slots 1-3 stay in registers for row y + 1's gather.
//
// Strips overlap by two columns: lane 0 and lane 31 hold the columns beside
// the 30 columns the warp owns (lanes 1..30). They load and evaluate springs
// like the other lanes (the springs from the left column into the strip,
// and the right column's targets), so every spring an owned particle needs
// is evaluated inside the warp; the neighbouring warp evaluates the shared
// springs too, from the same inputs, with the same result, and alone
// records their breaks. The row above the strip (y0 - 1) is evaluated
// without being owned; the row below (y1) is loaded only.
//
// Every floating-point operation is the one the tile kernel performs, in the
// same order (spring_df / spring_f32 / DfSum), so both kernels produce the
// same states and a context or batch can switch between them from one step
// to the next (the batch's sample steps stay on its tile list).
#pragma once

#include "tile_body.cuh"

namespace lsm {

namespace {

constexpr int STRIP_WARPS = 4;  // warps per CTA; each warp sweeps its own strip
constexpr int STRIP_OWN = 30;   // columns owned per strip (lanes 1..30)
constexpr unsigned FULL = 0xffffffffu;

// A pixel as the springs see it: drifted position in fixed point, and
// phase | broken flags << 8 (pm == 0: no particle).
struct PixFix {
    long long xf, yf;
    unsigned pm;
};

// A pixel as fetched from memory (x, vh as stored; ph == 0: no particle or
// outside the image).
struct PixRaw {
    double x, y, vx, vy;
    unsigned ph, mk;
};

__device__ __forceinline__ PixFix shfl_pix(const PixFix &p, int src)
{
    PixFix q;
    q.xf = __shfl_sync(FULL, p.xf, src);
    q.yf = __shfl_sync(FULL, p.yf, src);
    q.pm = __shfl_sync(FULL, p.pm, src);
    return q;
}

template <typename FT>
__device__ __forceinline__ FT shfl_ft(FT v, int src);
template <>
__device__ __forceinline__ float shfl_ft<float>(float v, int src) { return __shfl_sync(FULL, v, src); }
template <>
__device__ __forceinline__ ff shfl_ft<ff>(ff v, int src)
{
    return ff{__shfl_sync(FULL, v.hi, src), __shfl_sync(FULL, v.lo, src)};
}

// Issue the loads of pixel (gx, gy); x and the velocity are read whatever
// the phase (the state arrays cover every pixel) so that no load waits on
// another. VOBS: the full-step velocity (initial acceleration, observation)
// instead of the half-step one.
// Pixel indices are 32-bit: the kernel runs on grids of fewer than 2^30
// pixels (strip_supported), so that np + g fits too.
template <bool VOBS = false>
__device__ __forceinline__ PixRaw strip_fetch(const TileArgs &A, int gx, int gy)
{
    PixRaw r{0.0, 0.0, 0.0, 0.0, 0u, 0u};
    if (gx < 0 || gx >= A.nx || gy < 0 || gy >= A.ny) return r;
    const int g = gy * A.nx + gx, gyc = (int)A.np + g;
    r.ph = A.phase[g];
    r.mk = A.mask[g];
    r.x = A.x_in[g];
    r.y = A.x_in[gyc];
    const double *v = VOBS ? A.v_obs : A.vh_in;
    r.vx = v[g];
    r.vy = v[gyc];
    return r;
}

// The fetched pixel at the start of the step: position drifted by dt vh on
// free components (a grip's x stays, or follows the constant strain rate);
// an owned pixel's drifted position is written to x_out (pixel index g).
// Reference x of site (gx, row parity par): gx a on the square lattice,
// (gx + par / 2) a on the triangular packing.
template <int LAT>
__device__ __forceinline__ double site_X(const TileArgs &A, int gx, int par)
{
    if constexpr (LAT == 0) return ml((double)gx, A.a);
    else return ml(ad((double)gx, par ? 0.5 : 0.0), A.a);
}

// Drift (time steps only): the position moved by dt vh on free components;
// a grip (first or last site of its row, row length C) keeps its x, or
// follows the constant strain rate (rate_x: this lane's grip x at the strain
// of this step for the row's parity, from strip_rate_x).
template <bool RATE, bool SAMPLE, int LAT, int MODE>
__device__ __forceinline__ PixFix strip_make(const TileArgs &A, const PixRaw &r, int gx, int C, int g, bool own,
                                             double rate_x, bool &over, bool &bad)
{
    PixFix p{0, 0, 0u};
    if (!r.ph) return p;
    double px = r.x, py = r.y;
    const bool grip = gx == 0 || gx == C - 1;
    if (MODE == T_STEP) {
        if (RATE && grip) px = rate_x;
        if (!grip) px = fma(A.dt, r.vx, px);
        if (!(grip && A.grip_mode == 1)) py = fma(A.dt, r.vy, py);
    }
    if (MODE == T_STEP && own) {
        A.x_out[g] = px;
        A.x_out[(int)A.np + g] = py;
        if (SAMPLE) bad |= !dbl_finite_bits(px) || !dbl_finite_bits(py);
    }
    p.xf = dbl_to_fix(px, A.S, over);
    p.yf = dbl_to_fix(py, A.S, over);
    p.pm = r.ph | (r.mk << 8);
    return p;
}

// Constant strain rate: the x of a grip in column gx at the strain of the
// step being computed, eps = eps0 + (s - s0) rate dt, x = X + eps (X - xc),
// for rows of parity par (the same correctly rounded operations as the tile
// kernel). It depends on the step and the column only, so a strip computes
// it once per row parity instead of once per row.
template <int LAT>
__device__ __forceinline__ double strip_rate_x(const TileArgs &A, int gx, int par)
{
    const long long s = *A.d_step + A.t_off + 1 - A.rate_step0;
    const double eps = ad(A.rate_eps0, ml((double)s, A.rate_dt));
    const double X = site_X<LAT>(A, gx, par);
    return ad(X, ml(eps, sb(X, A.xc)));
}

// Force on the lower endpoint p of the spring p -> q in forward slot `slot`
// (zero if either pixel holds no particle or the spring is broken). Returns
// S_NONE (no spring, or broken before), S_BREAK (the break test fires in
// this step) or S_FORCE; with SAMPLE and S_FORCE also the spring's d_x, its
// stretch r - r0 and its type.
enum { S_NONE = 0, S_BREAK = 1, S_FORCE = 2 };

// Slots: square lattice (+1,0), (-1,+1), (0,+1), (+1,+1), type shell
// slot & 1; triangular packing (+1, same row), (-1/2, next row), (+1/2,
// next row), shell 0 for the row spring and 1 for the other two (their
// fixed-point lattice vectors share one |o|^2, the F32 correction term).
template <int PREC, bool SAMPLE, bool TEST, int LAT, typename FT>
__device__ __forceinline__ int strip_spring(const TileArgs &A, const PixFix &p, const PixFix &q, int slot,
                                            const TypeDF *sdf, const ff (*soff)[3], FT &fx, FT &fy, FT &dx,
                                            FT &st, TypeDF &t)
{
    fx = FT{};
    fy = FT{};
    const unsigned pp = p.pm & 0xffu, pq = q.pm & 0xffu;
    if (!pp || !pq || ((p.pm >> (8 + slot)) & 1u)) return S_NONE;
    const int shell = LAT == 0 ? (slot & 1) : (slot != 0);
    t = sdf[(((int)(pp - 1) * A.nphase) + (int)(pq - 1)) * 2 + shell];
    bool b;
    if constexpr (PREC == LSM_PREC_DF) {
        b = spring_df<TEST, SAMPLE>(q.xf - p.xf, q.yf - p.yf, t, A, fx, fy, dx, st);
    } else if constexpr (LAT == 0) {
        b = spring_f32<TEST, SAMPLE>(q.xf - p.xf, q.yf - p.yf, slot, t, soff, A, fx, fy, dx, st);
    } else {
        const long long ah = A.a_fix >> 1;
        const long long ofx = slot == 0 ? A.a_fix : (slot == 1 ? -ah : ah), ofy = slot == 0 ? 0 : A.h_fix;
        b = spring_f32_o<TEST, SAMPLE>(q.xf - p.xf, q.yf - p.yf, ofx, ofy, soff[slot][0].hi, soff[slot][1].hi,
                                       soff[slot][2].hi, t, A, fx, fy, dx, st);
    }
    return b ? S_BREAK : S_FORCE;
}

// The sample sums of one intact spring: the potential energy and the
// virial term d_x f_x (the tile kernel's terms). The double-float form sums
// k (r - r0)^2, halved once at the end (exactly), with the one-TwoSum
// addition: its error, a few units of 2^-48 of the terms' magnitudes per
// addition, stays near 3e-12 of the sum over the up to ~200 terms a lane
// accumulates along its strip.
template <typename FT>
__device__ __forceinline__ void spring_sample(ff &u, ff &w, const TypeDF &t, FT dx, FT fx, FT st);
template <>
__device__ __forceinline__ void spring_sample<ff>(ff &u, ff &w, const TypeDF &t, ff dx, ff fx, ff st)
{
    u = ff_add_sloppy(u, ff_mul(t.k, ff_sqr(st)));
    w = ff_add_sloppy(w, ff_mul(dx, fx));
}
template <>
__device__ __forceinline__ void spring_sample<float>(ff &u, ff &w, const TypeDF &t, float dx, float fx, float st)
{
    u = ff_add_f(u, t.k.hi * st * st);
    w = ff_add_f(w, dx * fx);
}

__device__ __forceinline__ ff warp_sum_ff(ff v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const ff w{__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
        v = ff_add_sloppy(v, w);
    }
    return v;
}

__device__ __forceinline__ float warp_max_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// The CTA's shared tables: the double-float spring types, the per-phase
// integration coefficients and masses, and (F32) the slots' lattice vectors.
// Every thread of the CTA calls it; the caller synchronises before use.
template <int PREC, int LAT>
__device__ __forceinline__ void strip_tables(const TileArgs &A, TypeDF *sdf, Coef4 *scoef, float *smassf,
                                             ff (*soff)[3])
{
    const int tid = threadIdx.x;
    const int nt = 2 * A.nphase * A.nphase;
    for (int q = tid; q < nt; q += blockDim.x) sdf[q] = A.tdf[q];
    if (tid < A.nphase) {
        scoef[tid] = A.coef[tid];
        smassf[tid] = (float)A.mass[tid];
    }
    if (PREC == LSM_PREC_F32 && tid < 4) {
        long long ofx, ofy;
        if (LAT == 0) {
            ofx = (tid == 0 ? 1 : (tid == 1 ? -1 : (tid == 2 ? 0 : 1))) * A.a_fix;
            ofy = (tid == 0 ? 0 : 1) * A.a_fix;
        } else {
            const long long ah = A.a_fix >> 1;
            ofx = tid == 0 ? A.a_fix : (tid == 1 ? -ah : ah);
            ofy = tid == 0 ? 0 : A.h_fix;
        }
        const ff ox = fix_to_ff(ofx, A.S), oy = fix_to_ff(ofy, A.S);
        soff[tid][0] = ox;
        soff[tid][1] = oy;
        soff[tid][2] = ff_add(ff_mul(ox, ox), ff_mul(oy, oy));
    }
}

// LAT: 0 square lattice (4 forward slots), 1 triangular packing (3; rows
// alternate between nx sites and nx - 1 sites shifted by half a spacing).
// MODE: T_STEP (a time step), T_INIT (the initial acceleration: half-step
// velocity from the current forces, no drift, no break test), T_OBSERVE (the
// sample of the current state). SAMPLE: the last step of an lsm_step call,
// or an observation, also writes the full-step velocity v(t+dt) = vh + dt/2
// a (steps) and the strip's partial sums of the sample (virial and
// potential energy of the owned springs, m v_x^2, kinetic energy,
// right-grip reaction, residual) at index `part` of the partial arrays
// (stride A.ntiles), as the tile kernel does per tile.
// One warp sweeps the strip of columns sx * 30 - 1 .. sx * 30 + 30 and rows
// y0 .. y0 + R - 1 (y0 < A.ny), with the CTA's shared tables.
template <int PREC, bool RATE, bool SAMPLE, int LAT, int MODE>
__device__ __forceinline__ void strip_run(const TileArgs &A, int R, int sx, int y0, int64_t part, const TypeDF *sdf,
                                          const Coef4 *scoef, const float *smassf, const ff (*soff)[3])
{
    using FT = typename std::conditional<PREC == LSM_PREC_F32, float, ff>::type;
    constexpr bool TEST = MODE == T_STEP;
    constexpr bool VOBS = MODE != T_STEP;
    const int lane = threadIdx.x & 31;
    const int y1 = min(y0 + R, A.ny);
    const int gx = sx * STRIP_OWN - 1 + lane;  // lanes 0 and 31: the neighbour columns
    const bool owner = lane >= 1 && lane <= STRIP_OWN && gx < A.nx;
    const long long step_now = MODE == T_STEP ? *A.d_step + A.t_off : 0;
    bool over = false, bad = false;
    // sample sums; m v_x^2 and the kinetic energy are float terms (2^-24
    // relative each, as in the tile kernel) summed as double-floats
    ff w_acc{0.0f, 0.0f}, u_acc{0.0f, 0.0f}, reactf{0.0f, 0.0f}, mvx2{0.0f, 0.0f}, ke{0.0f, 0.0f};
    float resf = 0.0f;
    // row length (sites) of row y: nx, or nx - 1 on odd rows of the packing
    auto row_len = [&](int y) { return LAT == 0 ? A.nx : A.nx - (y & 1); };

    // grip x under the constant strain rate, per row parity (used by grip lanes)
    double rate_x0 = 0.0, rate_x1 = 0.0;
    if constexpr (RATE && MODE == T_STEP) {
        rate_x0 = strip_rate_x<LAT>(A, gx, 0);
        rate_x1 = LAT == 0 ? rate_x0 : strip_rate_x<LAT>(A, gx, 1);
    }
    // row y0 - 1: its springs into row y0 are evaluated, it is not owned
    PixRaw raw = strip_fetch<VOBS>(A, gx, y0 - 1);
    PixFix P = strip_make<RATE, SAMPLE, LAT, MODE>(A, raw, gx, row_len(y0 - 1), 0, false, ((y0 - 1) & 1) ? rate_x1 : rate_x0,
                                                   over, bad);
    raw = strip_fetch<VOBS>(A, gx, y0);
    double vcx = 0.0, vcy = 0.0;
    FT p1x{}, p1y{}, p2x{}, p2y{}, p3x{}, p3y{};  // previous row's forces (slots 1..3)
    // square lattice: the slot-0 target (gx + 1, y) is the previous row's
    // slot-3 target (gx + 1, (y - 1) + 1), kept from its shuffle (not in the
    // sample step, whose sums need the registers)
    constexpr bool CARRY = LAT == 0 && !SAMPLE;
    PixFix q0n;
    if constexpr (CARRY) {
        q0n = shfl_pix(P, lane + 1);
        if (lane == 31) q0n.pm = 0u;
    }

    for (int y = y0 - 1; y < y1; y++) {
        const bool own = y >= y0;  // warp-uniform
        const int par = y & 1;     // row parity (triangular packing)
        // 1. row y + 1 (fetched last iteration), then fetch row y + 2
        const double vnx = raw.vx, vny = raw.vy;
        const PixFix N = strip_make<RATE, SAMPLE, LAT, MODE>(A, raw, gx, row_len(y + 1), (y + 1) * A.nx + gx,
                                                             owner && y + 1 < y1, par ? rate_x0 : rate_x1, over, bad);
        raw = strip_fetch<VOBS>(A, gx, y + 2 <= y1 ? y + 2 : -1);

        // 2. the forward springs of row y; the shuffles that wrap around the
        // warp (lane 31's right and lane 0's left neighbour) carry no particle
        PixFix q0;
        if constexpr (CARRY) {
            q0 = q0n;
        } else {
            q0 = shfl_pix(P, lane + 1);
            if (lane == 31) q0.pm = 0u;
        }
        PixFix q1, q3;
        if constexpr (LAT == 0) {
            q1 = shfl_pix(N, lane - 1);
            q3 = shfl_pix(N, lane + 1);
            if (lane == 31) q3.pm = 0u;
            if (lane == 0) q1.pm = 0u;
        } else {  // targets (gx - 1 + par, y + 1) and (gx + par, y + 1)
            q1 = shfl_pix(N, lane - 1 + par);
            q3 = par ? shfl_pix(N, lane + 1) : N;
            if (lane == 0 && !par) q1.pm = 0u;
            if (lane == 31 && par) q3.pm = 0u;
        }
        const bool sum_springs = SAMPLE && own && owner;
        FT f0x, f0y, dx, st;
        TypeDF t;
        const int s0 = strip_spring<PREC, SAMPLE, TEST, LAT>(A, P, q0, 0, sdf, soff, f0x, f0y, dx, st, t);
        if (sum_springs && s0 == S_FORCE) spring_sample(u_acc, w_acc, t, dx, f0x, st);
        const FT i0x = shfl_ft(f0x, lane - 1), i0y = shfl_ft(f0y, lane - 1);
        // incoming springs of row y - 1
        FT i3x, i3y, i1x, i1y, i2x, i2y;
        if constexpr (LAT == 0) {
            i3x = shfl_ft(p3x, lane - 1);
            i3y = shfl_ft(p3y, lane - 1);
            i1x = shfl_ft(p1x, lane + 1);
            i1y = shfl_ft(p1y, lane + 1);
            i2x = p2x;
            i2y = p2y;
        } else {  // from (gx - pp, y - 1) in slot 2 and (gx + 1 - pp, y - 1) in slot 1, pp = (y - 1) & 1
            const int pp = par ^ 1;
            i2x = shfl_ft(p2x, lane - pp);
            i2y = shfl_ft(p2y, lane - pp);
            i1x = shfl_ft(p1x, lane + 1 - pp);
            i1y = shfl_ft(p1y, lane + 1 - pp);
        }

        DfSum ax, ay;
        float sx_ = 0.0f, sy_ = 0.0f;
        if constexpr (PREC == LSM_PREC_DF) {
            if constexpr (LAT == 0) {  // canonical: slot 3, 2, 1 of row y - 1, slot 0 of row y
                ax.first_neg(i3x);
                ax.sub(i2x);
                ay.first_neg(i3y);
                ay.sub(i2y);
            } else {  // canonical: slot 2, slot 1 of row y - 1, slot 0 of row y
                ax.first_neg(i2x);
                ay.first_neg(i2y);
            }
            ax.sub(i1x);
            ax.sub(i0x);
            ax.add(f0x);
            ay.sub(i1y);
            ay.sub(i0y);
            ay.add(f0y);
        } else {
            if constexpr (LAT == 0) {
                sx_ = f0x - i3x;
                sy_ = f0y - i3y;
            } else {
                sx_ = f0x - i2x;
                sy_ = f0y - i2y;
            }
        }
        FT f1x, f1y, f2x, f2y, f3x{}, f3y{};
        int s1, s2, s3 = S_NONE;
        if constexpr (LAT == 0) {
            s1 = strip_spring<PREC, SAMPLE, TEST, LAT>(A, P, q1, 1, sdf, soff, f1x, f1y, dx, st, t);
            if (sum_springs && s1 == S_FORCE) spring_sample(u_acc, w_acc, t, dx, f1x, st);
            s2 = strip_spring<PREC, SAMPLE, TEST, LAT>(A, P, N, 2, sdf, soff, f2x, f2y, dx, st, t);
            if (sum_springs && s2 == S_FORCE) spring_sample(u_acc, w_acc, t, dx, f2x, st);
            s3 = strip_spring<PREC, SAMPLE, TEST, LAT>(A, P, q3, 3, sdf, soff, f3x, f3y, dx, st, t);
            if (sum_springs && s3 == S_FORCE) spring_sample(u_acc, w_acc, t, dx, f3x, st);
        } else {
            s1 = strip_spring<PREC, SAMPLE, TEST, LAT>(A, P, q1, 1, sdf, soff, f1x, f1y, dx, st, t);
            if (sum_springs && s1 == S_FORCE) spring_sample(u_acc, w_acc, t, dx, f1x, st);
            s2 = strip_spring<PREC, SAMPLE, TEST, LAT>(A, P, q3, 2, sdf, soff, f2x, f2y, dx, st, t);
            if (sum_springs && s2 == S_FORCE) spring_sample(u_acc, w_acc, t, dx, f2x, st);
        }

        // 3. gather + integrate the owned particle (gx, y)
        if (own) {
            double F[2];
            float Ff[2];  // F as floats (sample statistics without FP64 work)
            ff Fx;        // F_x as a double-float (the grip reaction)
            if constexpr (PREC == LSM_PREC_DF) {
                ax.add(f1x);
                ax.add(f2x);
                ay.add(f1y);
                ay.add(f2y);
                if constexpr (LAT == 0) {
                    ax.add(f3x);
                    ay.add(f3y);
                }
                F[0] = ax.value(A.df_bias);
                F[1] = ay.value(A.df_bias);
                Ff[0] = __fmul_rn(__fadd_rn(ax.hs, ax.el), A.p24);  // back from units of 2^(24-S)
                Ff[1] = __fmul_rn(__fadd_rn(ay.hs, ay.el), A.p24);
                Fx = ff{ax.hs, ax.el};  // (in those units)
            } else {
                if constexpr (LAT == 0) {
                    sx_ += f1x - i2x;
                    sy_ += f1y - i2y;
                    sx_ += f2x - i1x;
                    sy_ += f2y - i1y;
                    sx_ += f3x - i0x;
                    sy_ += f3y - i0y;
                } else {
                    sx_ += f1x - i1x;
                    sy_ += f1y - i1y;
                    sx_ += f2x - i0x;
                    sy_ += f2y - i0y;
                }
                F[0] = f2d_force(sx_);
                F[1] = f2d_force(sy_);
                Ff[0] = sx_;
                Ff[1] = sy_;
                Fx = ff{sx_, 0.0f};
            }
            if (owner && (P.pm & 0xffu)) {
                const int g = y * A.nx + gx;
                const int ph = (int)(P.pm & 0xffu) - 1;
                const Coef4 k4 = scoef[ph];
                const bool grip = gx == 0 || gx == row_len(y) - 1;
                const bool fixy = grip && A.grip_mode == 1;
                if (SAMPLE && gx == row_len(y) - 1) reactf = ff_add(reactf, ff_neg(Fx));  // right grip
                const double vh[2] = {vcx, vcy};
                const bool fixed[2] = {grip, fixy};
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const int q = c * (int)A.np + g;
                    if (fixed[c]) {
                        if (MODE == T_STEP) A.vh_out[q] = 0.0;
                        if (MODE == T_STEP && SAMPLE) A.v_obs[q] = 0.0;
                        continue;
                    }
                    double vn;
                    if (MODE == T_OBSERVE) {
                        vn = vh[c];  // the stored full-step velocity
                    } else {
                        vn = fma(k4.c2h, F[c], k4.c1h * vh[c]);
                        if (MODE == T_INIT) {
                            A.vh_out[q] = vn;  // vh = v + dt/2 a(x)
                            continue;
                        }
                        A.vh_out[q] = fma(k4.c2, F[c], k4.c1 * vh[c]);
                    }
                    if (SAMPLE) {
                        if (MODE == T_STEP) A.v_obs[q] = vn;
                        // float statistics (residual, KE, m v_x^2), as the tile kernel
                        const float vf = d2f_bits(vn);
                        resf = fmaxf(resf, fmaxf(fabsf(Ff[c]), fabsf(vf)));
                        const float mv2 = __fmul_rn(__fmul_rn(smassf[ph], vf), vf);
                        ke = ff_add_f(ke, __fmul_rn(0.5f, mv2));
                        if (c == 0) mvx2 = ff_add_f(mvx2, mv2);
                        if (MODE == T_STEP) bad |= !dbl_finite_bits(vn);
                    }
                }
                const int nb = (int)(s0 == S_BREAK) | ((int)(s1 == S_BREAK) << 1) | ((int)(s2 == S_BREAK) << 2) |
                               ((int)(s3 == S_BREAK) << 3);
                if (MODE == T_STEP && nb) {
                    A.mask[g] = (uint8_t)((P.pm >> 8) | (unsigned)nb);
#pragma unroll
                    for (int slot = 0; slot < 4; slot++) {
                        if ((nb >> slot) & 1) {
                            A.brk[(int64_t)slot * A.np + g] = step_now;
                            atomicMin(A.first_break, (unsigned long long)step_now);
                            atomicAdd(A.nbroken, 1ull);
                        }
                    }
                }
            }
        }

        // carry to row y + 1
        p1x = f1x;
        p1y = f1y;
        p2x = f2x;
        p2y = f2y;
        p3x = f3x;
        p3y = f3y;
        P = N;
        if constexpr (CARRY) q0n = q3;
        vcx = vnx;
        vcy = vny;
    }
    if (__any_sync(FULL, over) && lane == 0) atomicOr(A.status, 2);
    if (SAMPLE) {
        if (__any_sync(FULL, bad) && lane == 0) atomicOr(A.status, 1);
        const ff tw = warp_sum_ff(w_acc), tu = warp_sum_ff(u_acc), tr = warp_sum_ff(reactf);
        const ff tm = warp_sum_ff(mvx2), tk = warp_sum_ff(ke);
        const float tres = warp_max_f(resf);
        if (lane == 0) {
            // DF: virial, energy and reaction from units of 2^(24-S) (exact)
            const double u = PREC == LSM_PREC_DF ? (double)A.p24 : 1.0;
            A.part_s[part] = ff_to_double(tw) * (u * u);
            A.part_s[A.ntiles + part] = 0.5 * ff_to_double(tu) * (u * u);  // the 1/2 of 1/2 k (r - r0)^2, exact
            A.part_p[part] = ff_to_double(tm);
            A.part_p[A.ntiles + part] = ff_to_double(tk);
            A.part_p[2 * A.ntiles + part] = ff_to_double(tr) * u;
            A.part_p[3 * A.ntiles + part] = f2d_bits(tres);
        }
    }
}

}  // namespace

// CTAs per SM the strip kernels are compiled for: 5 of 128 threads (up to
// 102 registers) for the DF time step and every sample step, 6 (up to 85)
// for the F32 time step; each fits its budget without spills.
template <int PREC, bool SAMPLE>
constexpr int strip_min_ctas() { return PREC == LSM_PREC_DF || SAMPLE ? 5 : 6; }

}  // namespace lsm
