// tile2d.cu -- fused one-launch-per-time-step kernel for 2D image lattices.
//
// A CTA owns a TX x TY tile of pixels. Per time step it
//   1. loads positions and half-step velocities of the tile plus a one-pixel
//      halo into shared memory and drifts them, x(t+dt) = x + dt vh (Eq. 3);
//   2. evaluates every spring that touches the tile once (Eq. 2, break test
//      on the squared length), writing the force on the spring's lower
//      endpoint into shared memory; springs that cross the tile edge are also
//      evaluated by the neighbouring tile, with bit-identical results, so no
//      cross-CTA communication is needed;
//   3. gathers each owned particle's eight spring forces in a fixed order
//      (the order of the canonical spring list: incoming springs by ascending
//      source, then outgoing springs by ascending target), applies the viscous
//      half-kick (Eqs. 4-5) and the next half-kick, and writes x(t+dt) and
//      vh(t+3dt/2) to the other buffer of a ping-pong pair.
// State lives on the pixel grid (void pixels carry no particle and are never
// read). Springs of pixel p are the forward offsets sorted by raster distance:
// slot 0 (+1,0), slot 1 (-1,+1), slot 2 (0,+1), slot 3 (+1,+1); their broken
// flags are the low 4 bits of mask[p], written only by the tile owning p.
//
// Precision modes: EXACT64 performs the same correctly rounded operations in
// the same order as the sequential FP64 definition (bit-identical state);
// FAST64 uses fused multiply-add and a reciprocal square root; F32 and DF form
// the spring vector exactly from 64-bit fixed-point positions and evaluate the
// force in single precision or in double-float arithmetic, integrating in FP64.
#include "tile_body.cuh"

#include <cmath>

namespace lsm {

template <int TX, int TY, int PREC, int MODE, bool SAMPLE, bool RATE>
__global__ void __launch_bounds__(tile_threads<TY, PREC, SAMPLE>(), (tile_min_ctas<TY, PREC, SAMPLE>()))
k_tile2d(TileArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_body<TX, TY, PREC, MODE, SAMPLE, RATE>(A, blockIdx.x, blockIdx.y,
                                                (int64_t)blockIdx.y * gridDim.x + blockIdx.x, smem_raw);
}

// Load increment on the pixel grid, or on the triangular packing's sites
// (tri: rows alternate between nx sites at x = ix a and nx - 1 sites at
// x = (ix + 1/2) a; a row's first and last site are its grips) (Sections
// 2.3, 3.1).
__global__ void k_tile_strain(int nx, int ny, int64_t np, double *x, double *vh, double *v_obs,
                              const uint8_t *phase, double a, double xc, double scale, double eps,
                              int affine, double *d_eps, int tri)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0) *d_eps = eps;
    if (g >= np || !phase[g]) return;
    const int gx = (int)(g % nx);
    const int odd = tri ? (int)((g / nx) & 1) : 0;
    double xp = x[g];
    if (affine) xp = ad(xc, ml(sb(xp, xc), scale));
    if (gx == 0 || gx == nx - 1 - odd) {
        const double X = odd ? ml(ad((double)gx, 0.5), a) : gx * a;
        xp = ad(X, ml(eps, sb(X, xc)));
        vh[g] = 0.0;
        v_obs[g] = 0.0;
    }
    x[g] = xp;
}

// Pixel-grid broken flags / break steps -> canonical spring order. sbase[g]
// is the canonical index of pixel g's first forward spring; its springs follow
// in slot order, which is the canonical order of their upper endpoints.
__global__ void k_tile_export(int nx, int ny, int64_t np, const uint8_t *__restrict__ phase,
                              const uint8_t *__restrict__ mask, const long long *__restrict__ brk,
                              const int64_t *__restrict__ sbase, uint8_t *__restrict__ out_mask,
                              long long *__restrict__ out_brk, int tri)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= np || !phase[g]) return;
    const int gx = (int)(g % nx), gy = (int)(g / nx);
    int64_t b = sbase[g];
    const uint8_t mk = mask[g];
    const int odd = gy & 1;
#pragma unroll
    for (int slot = 0; slot < 4; slot++) {
        // square: (+1,0), (-1,+1), (0,+1), (+1,+1); packing: (+1, same row),
        // then the next row's sites at x -/+ a/2 (no fourth slot); the
        // packing's padding site (last of an odd row) has phase 0
        if (tri && slot == 3) break;
        const int dx = tri ? (slot == 0 ? 1 : (slot == 1 ? odd - 1 : odd))
                           : (slot == 0 ? 1 : (slot == 1 ? -1 : (slot == 2 ? 0 : 1)));
        const int dy = slot == 0 ? 0 : 1;
        const int qx = gx + dx, qy = gy + dy;
        if (qx < 0 || qx >= nx || qy >= ny || !phase[(int64_t)qy * nx + qx]) continue;
        if (out_mask) out_mask[b] = (mk >> slot) & 1u;
        if (out_brk) out_brk[b] = brk[(int64_t)slot * np + g];
        b++;
    }
}

cudaError_t tile_export(Ctx &c, bool steps)
{
    if (c.dim == 3) return tile3_export(c, steps);
    if (c.m == 0) return cudaSuccess;
    if (!c.texport) {
        cudaError_t e = lsm::dev_malloc((void **)&c.texport, c.m);
        if (e != cudaSuccess) return e;
    }
    if (steps && !c.texport_brk) {
        cudaError_t e = lsm::dev_malloc((void **)&c.texport_brk, c.m * sizeof(long long));
        if (e != cudaSuccess) return e;
    }
    const unsigned g = (unsigned)((c.tnp + 255) / 256);
    k_tile_export<<<g, 256, 0, c.stream>>>(c.tgnx, c.tgny, c.tnp, c.tph, c.tmask, c.tbrk, c.tsbase,
                                           steps ? nullptr : c.texport, steps ? c.texport_brk : nullptr,
                                           c.tri ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host


constexpr int TILE_X = 32;

// Tile height: 8 rows of one warp each (6 CTAs per SM) for the double-float
// steps without a sample, 16 rows otherwise (measured fastest per mode on the
// 2048 x 2048 composite). Only sample steps write per-tile partial sums, so
// the partials always come from 16-row tiles (half as many block reductions
// as 8-row tiles would need).
constexpr int TILE_Y_SAMPLE = 16;
template <int PREC, bool SAMPLE>
constexpr int tile_y() { return PREC == LSM_PREC_DF && !SAMPLE ? 8 : TILE_Y_SAMPLE; }

static TileArgs tile_args(Ctx &c)
{
    TileArgs A;
    A.nx = c.tgnx;
    A.ny = c.tgny;
    A.nphase = c.tile_nphase;
    A.np = c.tnp;
    A.x_in = c.tx[c.tcur];
    A.vh_in = c.tvh[c.tcur];
    A.x_out = c.tx[c.tcur ^ 1];
    A.vh_out = c.tvh[c.tcur ^ 1];
    A.v_obs = c.tvobs;
    A.phase = c.tph;
    A.mask = c.tmask;
    A.brk = c.tbrk;
    A.types = c.types;
    A.tdf = c.tdf;
    A.mass = c.tmass;
    A.coef = (const Coef4 *)c.tinvm;
    A.S = c.fix_S;
    A.a_fix = c.a_fix;
    A.h_fix = c.h_fix;
    A.hrow = c.h.a * std::sqrt(3.0) * 0.5;
    A.p24 = ldexpf(1.0f, 24 - c.fix_S);
    A.p0 = ldexpf(1.0f, -c.fix_S);
    A.df_bias = (unsigned)(896 + 24 - c.fix_S) << 20;
    A.dt = c.h.dt;
    A.hdt = 0.5 * c.h.dt;
    A.gamma = c.h.damping;
    A.a = c.h.a;
    A.grip_mode = c.h.grip_mode;
    A.rate_on = c.rate_on;
    A.rate_eps0 = c.rate_eps0;
    A.rate_dt = c.rate_dt;
    A.rate_step0 = c.rate_step0;
    A.xc = c.h.xc;
    A.d_step = c.d_step;
    A.t_off = 0;
    A.first_break = c.d_first_break;
    A.nbroken = c.d_nbroken;
    A.status = c.d_status;
    A.part_s = c.part_s;
    A.part_p = c.part_p;
    A.ntiles = c.ntiles;
    return A;
}

template <int PREC, int MODE, bool SAMPLE, bool RATE>
static cudaError_t launch_tile(Ctx &c, TileArgs A)
{
    constexpr int TILE_Y = tile_y<PREC, SAMPLE>();
    auto kern = k_tile2d<TILE_X, TILE_Y, PREC, MODE, SAMPLE, RATE>;
    const size_t smem = tile_smem_bytes<TILE_X, TILE_Y>(PREC);
    static bool configured = false;  // per template instance
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // all of the unified L1 / shared storage as shared memory: the CTAs per
        // SM are bounded by shared memory and registers, not by the carveout
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((c.h.nx + TILE_X - 1) / TILE_X, (c.h.ny + TILE_Y - 1) / TILE_Y);
    kern<<<grid, tile_threads<TILE_Y, PREC, SAMPLE>(), smem, c.stream>>>(A);
    return cudaSuccess;
}

// constant strain-rate loading is a separate instance of the time step, so
// that the ordinary step carries none of its code (registers)
template <int MODE, bool SAMPLE, bool RATE>
static cudaError_t launch_tile_p(Ctx &c, TileArgs A)
{
    switch (c.h.precision) {
    case LSM_PREC_FAST64: return launch_tile<LSM_PREC_FAST64, MODE, SAMPLE, RATE>(c, A);
    case LSM_PREC_F32: return launch_tile<LSM_PREC_F32, MODE, SAMPLE, RATE>(c, A);
    case LSM_PREC_DF: return launch_tile<LSM_PREC_DF, MODE, SAMPLE, RATE>(c, A);
    default: return launch_tile<LSM_PREC_EXACT64, MODE, SAMPLE, RATE>(c, A);
    }
}

template <int MODE, bool SAMPLE>
static cudaError_t launch_tile_prec(Ctx &c, TileArgs A)
{
    if (MODE == T_STEP && c.rate_on) return launch_tile_p<MODE, SAMPLE, true>(c, A);
    return launch_tile_p<MODE, SAMPLE, false>(c, A);
}

cudaError_t tile_enqueue_steps(Ctx &c, int64_t nsteps, int start_buf)
{
    int cur = start_buf;
    for (int64_t t = 0; t < nsteps; t++) {
        TileArgs A = tile_args(c);
        A.t_off = t;
        A.x_in = c.tx[cur];
        A.vh_in = c.tvh[cur];
        A.x_out = c.tx[cur ^ 1];
        A.vh_out = c.tvh[cur ^ 1];
        const bool last = t == nsteps - 1;
        cudaError_t e = c.strip ? launch_strip(c, A, last)
                        : last  ? launch_tile_prec<T_STEP, true>(c, A)
                                : launch_tile_prec<T_STEP, false>(c, A);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    return cudaGetLastError();
}

cudaError_t tile_init_accel(Ctx &c)
{
    TileArgs A = tile_args(c);
    A.vh_out = c.tvh[c.tcur];  // vh = v + dt/2 a, written in place of the current buffer
    cudaError_t e = c.tri ? launch_strip_mode(c, A, T_INIT) : launch_tile_prec<T_INIT, false>(c, A);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t tile_observe(Ctx &c)
{
    TileArgs A = tile_args(c);
    cudaError_t e = c.tri ? launch_strip_mode(c, A, T_OBSERVE) : launch_tile_prec<T_OBSERVE, true>(c, A);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t tile_apply_strain(Ctx &c, double eps_old, double eps_new)
{
    const double scale = (1.0 + eps_new) / (1.0 + eps_old);
    const unsigned g = (unsigned)((c.tnp + 255) / 256);
    k_tile_strain<<<g, 256, 0, c.stream>>>(c.tgnx, c.tgny, c.tnp, c.tx[c.tcur], c.tvh[c.tcur], c.tvobs,
                                           c.tph, c.h.a, c.h.xc, scale, eps_new, c.h.load_mode == 0,
                                           c.d_eps, c.tri ? 1 : 0);
    return cudaGetLastError();
}

int64_t tile_count(const Ctx &c)
{
    return (int64_t)((c.h.nx + TILE_X - 1) / TILE_X) * ((c.h.ny + TILE_Y_SAMPLE - 1) / TILE_Y_SAMPLE);
}

}  // namespace lsm
