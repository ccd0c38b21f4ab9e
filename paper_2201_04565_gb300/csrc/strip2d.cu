// strip2d.cu -- register-resident time step for 2D square-lattice images in
// the fixed-point modes (F32, DF).
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
// same bits and the sample steps can stay on the tile kernel.
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

// Issue the loads of pixel (gx, gy); x and vh are read whatever the phase
// (the state arrays cover every pixel) so that no load waits on another.
__device__ __forceinline__ PixRaw strip_fetch(const TileArgs &A, int gx, int gy)
{
    PixRaw r{0.0, 0.0, 0.0, 0.0, 0u, 0u};
    if (gx < 0 || gx >= A.nx || gy < 0 || gy >= A.ny) return r;
    const int64_t g = (int64_t)gy * A.nx + gx;
    r.ph = A.phase[g];
    r.mk = A.mask[g];
    r.x = A.x_in[g];
    r.y = A.x_in[A.np + g];
    r.vx = A.vh_in[g];
    r.vy = A.vh_in[A.np + g];
    return r;
}

// The fetched pixel at the start of the step: position drifted by dt vh on
// free components (a grip's x stays, or follows the constant strain rate);
// an owned pixel's drifted position is written to x_out (pixel index g).
template <bool RATE>
__device__ __forceinline__ PixFix strip_make(const TileArgs &A, const PixRaw &r, int gx, int64_t g, bool own,
                                             bool &over)
{
    PixFix p{0, 0, 0u};
    if (!r.ph) return p;
    double px = r.x, py = r.y;
    const bool grip = gx == 0 || gx == A.nx - 1;
    if (RATE && grip) {  // constant strain rate: grip x at the strain of this step
        const long long s = *A.d_step + A.t_off + 1 - A.rate_step0;
        const double eps = ad(A.rate_eps0, ml((double)s, A.rate_dt));
        const double X = ml((double)gx, A.a);
        px = ad(X, ml(eps, sb(X, A.xc)));
    }
    if (!grip) px = fma(A.dt, r.vx, px);
    if (!(grip && A.grip_mode == 1)) py = fma(A.dt, r.vy, py);
    if (own) {
        A.x_out[g] = px;
        A.x_out[A.np + g] = py;
    }
    p.xf = dbl_to_fix(px, A.S, over);
    p.yf = dbl_to_fix(py, A.S, over);
    p.pm = r.ph | (r.mk << 8);
    return p;
}

// Force on the lower endpoint p of the spring p -> q in forward slot `slot`
// (zero if either pixel holds no particle or the spring is broken); returns
// true when the break test fires in this step.
template <int PREC, typename FT>
__device__ __forceinline__ bool strip_spring(const TileArgs &A, const PixFix &p, const PixFix &q, int slot,
                                             const TypeDF *sdf, const ff (*soff)[3], FT &fx, FT &fy)
{
    fx = FT{};
    fy = FT{};
    const unsigned pp = p.pm & 0xffu, pq = q.pm & 0xffu;
    if (!pp || !pq || ((p.pm >> (8 + slot)) & 1u)) return false;
    const TypeDF t = sdf[(((int)(pp - 1) * A.nphase) + (int)(pq - 1)) * 2 + (slot & 1)];
    if constexpr (PREC == LSM_PREC_DF) {
        ff dx, st;
        return spring_df<true, false>(q.xf - p.xf, q.yf - p.yf, t, A, fx, fy, dx, st);
    } else {
        float dx, st;
        return spring_f32<true, false>(q.xf - p.xf, q.yf - p.yf, slot, t, soff, A, fx, fy, dx, st);
    }
}

}  // namespace

// CTAs per SM the strip kernel is compiled for (its register budget without
// spills: 80 registers in F32, 102 in DF).
template <int PREC>
constexpr int strip_min_ctas() { return PREC == LSM_PREC_DF ? 5 : 6; }

template <int PREC, bool RATE>
__global__ void __launch_bounds__(32 * STRIP_WARPS, strip_min_ctas<PREC>())
k_strip2d(TileArgs A, int R, int nsx)
{
    using FT = typename std::conditional<PREC == LSM_PREC_F32, float, ff>::type;
    __shared__ TypeDF sdf[128];
    __shared__ Coef4 scoef[8];
    __shared__ ff soff[4][3];  // per slot: o_x, o_y, |o|^2 (F32)
    const int tid = threadIdx.x, lane = tid & 31;
    const int nt = 2 * A.nphase * A.nphase;
    for (int q = tid; q < nt; q += 32 * STRIP_WARPS) sdf[q] = A.tdf[q];
    if (tid < A.nphase) scoef[tid] = A.coef[tid];
    if (PREC == LSM_PREC_F32 && tid < 4) {
        const int dx = tid == 0 ? 1 : (tid == 1 ? -1 : (tid == 2 ? 0 : 1));
        const int dy = tid == 0 ? 0 : 1;
        const ff ox = fix_to_ff((long long)dx * A.a_fix, A.S), oy = fix_to_ff((long long)dy * A.a_fix, A.S);
        soff[tid][0] = ox;
        soff[tid][1] = oy;
        soff[tid][2] = ff_add(ff_mul(ox, ox), ff_mul(oy, oy));
    }
    __syncthreads();

    const int strip = blockIdx.x * STRIP_WARPS + (tid >> 5);
    const int sx = strip % nsx, sy = strip / nsx;
    const int y0 = sy * R;
    if (y0 >= A.ny) return;  // whole warps only
    const int y1 = min(y0 + R, A.ny);
    const int gx = sx * STRIP_OWN - 1 + lane;  // lanes 0 and 31: the neighbour columns
    const bool owner = lane >= 1 && lane <= STRIP_OWN && gx < A.nx;
    const long long step_now = *A.d_step + A.t_off;
    bool over = false;

    // row y0 - 1: its springs into row y0 are evaluated, it is not owned
    PixRaw raw = strip_fetch(A, gx, y0 - 1);
    PixFix P = strip_make<RATE>(A, raw, gx, 0, false, over);
    raw = strip_fetch(A, gx, y0);
    double vcx = 0.0, vcy = 0.0;
    FT p1x{}, p1y{}, p2x{}, p2y{}, p3x{}, p3y{};  // previous row's slot 1-3 forces

    for (int y = y0 - 1; y < y1; y++) {
        const bool own = y >= y0;  // warp-uniform
        // 1. row y + 1 (fetched last iteration), then fetch row y + 2
        const double vnx = raw.vx, vny = raw.vy;
        const PixFix N = strip_make<RATE>(A, raw, gx, (int64_t)(y + 1) * A.nx + gx, owner && y + 1 < y1, over);
        raw = strip_fetch(A, gx, y + 2 < y1 + 1 ? y + 2 : -1);

        // 2. the forward springs of row y; the shuffles that wrap around the
        // warp (lane 31's right and lane 0's left neighbour) carry no particle
        PixFix q0 = shfl_pix(P, lane + 1);
        PixFix q1 = shfl_pix(N, lane - 1);
        PixFix q3 = shfl_pix(N, lane + 1);
        if (lane == 31) q0.pm = q3.pm = 0u;
        if (lane == 0) q1.pm = 0u;
        FT f0x, f0y;
        const bool b0 = strip_spring<PREC>(A, P, q0, 0, sdf, soff, f0x, f0y);
        const FT i0x = shfl_ft(f0x, lane - 1), i0y = shfl_ft(f0y, lane - 1);
        const FT i3x = shfl_ft(p3x, lane - 1), i3y = shfl_ft(p3y, lane - 1);
        const FT i1x = shfl_ft(p1x, lane + 1), i1y = shfl_ft(p1y, lane + 1);

        DfSum ax, ay;
        float sx_ = 0.0f, sy_ = 0.0f;
        if constexpr (PREC == LSM_PREC_DF) {
            ax.first_neg(i3x);
            ax.sub(p2x);
            ax.sub(i1x);
            ax.sub(i0x);
            ax.add(f0x);
            ay.first_neg(i3y);
            ay.sub(p2y);
            ay.sub(i1y);
            ay.sub(i0y);
            ay.add(f0y);
        } else {
            sx_ = f0x - i3x;
            sy_ = f0y - i3y;
        }
        FT f1x, f1y, f2x, f2y, f3x, f3y;
        const bool b1 = strip_spring<PREC>(A, P, q1, 1, sdf, soff, f1x, f1y);
        const bool b2 = strip_spring<PREC>(A, P, N, 2, sdf, soff, f2x, f2y);
        const bool b3 = strip_spring<PREC>(A, P, q3, 3, sdf, soff, f3x, f3y);

        // 3. gather + integrate the owned particle (gx, y)
        if (own) {
            double F[2];
            if constexpr (PREC == LSM_PREC_DF) {
                ax.add(f1x);
                ax.add(f2x);
                ax.add(f3x);
                ay.add(f1y);
                ay.add(f2y);
                ay.add(f3y);
                F[0] = ax.value();
                F[1] = ay.value();
            } else {
                sx_ += f1x - p2x;
                sy_ += f1y - p2y;
                sx_ += f2x - i1x;
                sy_ += f2y - i1y;
                sx_ += f3x - i0x;
                sy_ += f3y - i0y;
                F[0] = f2d_bits(sx_);
                F[1] = f2d_bits(sy_);
            }
            if (owner && (P.pm & 0xffu)) {
                const int64_t g = (int64_t)y * A.nx + gx;
                const Coef4 k4 = scoef[(P.pm & 0xffu) - 1];
                const bool grip = gx == 0 || gx == A.nx - 1;
                const bool fixy = grip && A.grip_mode == 1;
                A.vh_out[g] = grip ? 0.0 : fma(k4.c2, F[0], k4.c1 * vcx);
                A.vh_out[A.np + g] = fixy ? 0.0 : fma(k4.c2, F[1], k4.c1 * vcy);
                const int nb = (int)b0 | ((int)b1 << 1) | ((int)b2 << 2) | ((int)b3 << 3);
                if (nb) {
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
        vcx = vnx;
        vcy = vny;
    }
    if (__any_sync(FULL, over) && lane == 0) atomicOr(A.status, 2);
}

// ------------------------------------------------------------------ host

namespace {

template <int PREC, bool RATE>
cudaError_t launch_strip_t(Ctx &c, const TileArgs &A)
{
    auto kern = k_strip2d<PREC, RATE>;
    static int resident = 0;  // warps per device of this instance (occupancy x SMs)
    if (!resident) {
        int dev = 0, nsm = 0, nb = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 32 * STRIP_WARPS, 0);
        if (e != cudaSuccess) return e;
        resident = std::max(1, nb * STRIP_WARPS * nsm);
    }
    // strip height: one warp per strip, as many strips as fit on the device
    // at once (one wave), but at least 8 rows per strip
    const int nsx = (c.h.nx + STRIP_OWN - 1) / STRIP_OWN;
    const int rows_target = std::max(1, resident / nsx);
    const int R = std::max(8, (c.h.ny + rows_target - 1) / rows_target);
    const int nsy = (c.h.ny + R - 1) / R;
    const int64_t nstrips = (int64_t)nsx * nsy;
    const unsigned grid = (unsigned)((nstrips + STRIP_WARPS - 1) / STRIP_WARPS);
    kern<<<grid, 32 * STRIP_WARPS, 0, c.stream>>>(A, R, nsx);
    return cudaSuccess;
}

}  // namespace

bool strip_supported(const Ctx &c)
{
    return c.dim == 2 && c.h.lattice == 0 &&
           (c.h.precision == LSM_PREC_DF || c.h.precision == LSM_PREC_F32);
}

cudaError_t launch_strip(Ctx &c, const TileArgs &A)
{
    const bool rate = c.rate_on;
    if (c.h.precision == LSM_PREC_DF)
        return rate ? launch_strip_t<LSM_PREC_DF, true>(c, A) : launch_strip_t<LSM_PREC_DF, false>(c, A);
    return rate ? launch_strip_t<LSM_PREC_F32, true>(c, A) : launch_strip_t<LSM_PREC_F32, false>(c, A);
}

}  // namespace lsm
