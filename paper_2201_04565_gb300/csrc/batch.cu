// batch.cu -- many 2D specimens stepped by one launch per time step.
//
// Specimens are concatenated pixel grids (specimen s owns pixels
// [pbase_s, pbase_s + nx_s ny_s) of every per-pixel array, and the blocks
// [2 pbase_s, 2 pbase_s + 2 np_s) of the two-component arrays). Each time
// step is one launch of k_tile2d_batch over a global tile list; CTAs walk the
// list with a grid stride, so the grid can be one CTA per tile or a
// persistent grid. Every specimen has its own ping-pong parity, step counter
// and "active" flag (relax stops stepping converged specimens); a tiny kernel
// after each step flips the parity of the active ones. Samples are folded per
// specimen from that specimen's contiguous range of per-tile partial sums, in
// a fixed order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/lsm_nn.h"
#include "strip_body.cuh"

namespace lsm {

struct SpecDesc {
    int nx, ny;
    int64_t pbase;    // first pixel of the specimen in the concatenated grids
    int64_t tbase;    // first tile of the specimen in the tile list
    int64_t ntiles;   // tiles of the specimen
    int64_t sbase;    // first tile of the specimen in the sample-step tile list
    int64_t nstiles;  // its tiles there
    double xc, omega, grip_area;
    double eps;       // applied strain
    int cur;          // current ping-pong buffer
    int active;       // 1 = stepping
    long long steps;  // time steps taken
};

struct BatchTile {
    int spec, bx, by, pad;
};

struct BatchCtx {
    std::string err;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int S = 0;                       // specimens
    int prec = LSM_PREC_DF;
    int nphase = 1;
    double dt = 0.01, damping = 0.0, a = 1.0;
    int grip_mode = 0, load_mode = 0;
    std::vector<int> nx, ny;
    std::vector<int64_t> n, m, pbase;
    std::vector<std::vector<int64_t>> pix;  // particle -> pixel (empty: identity)
    std::vector<double> eps;                // host mirror
    int64_t NP = 0;                         // pixels in all specimens
    // schedule: tiles of tile_y rows, or (strip_r > 0, fixed-point modes)
    // the plain steps on strips of strip_r rows
    int tile_y = 16, grid = 0, order = 0, strip_r = 0;
    int64_t T = 0;
    BatchTile *strips = nullptr;  // (spec, sx, sy) of every strip
    int64_t NSTRIP = 0;
    // device memory
    double *X[2] = {nullptr, nullptr}, *VH[2] = {nullptr, nullptr}, *VOBS = nullptr;
    uint8_t *PH = nullptr, *MASK = nullptr;
    long long *BRK = nullptr;
    int64_t *SBASE = nullptr;
    SpecDesc *specs = nullptr;
    BatchTile *tiles = nullptr;
    BatchTile *stiles = nullptr;  // 16-row tiles of the sample steps (== tiles when tile_y is 16)
    int64_t TS = 0;               // tiles in that list (the per-tile partials)
    double *part_s = nullptr, *part_p = nullptr;
    unsigned long long *fb = nullptr, *nb = nullptr;
    int *status = nullptr, *nactive = nullptr;
    long long *d_nsamp = nullptr;
    DeviceSample *samples = nullptr;  // [S][cap]
    DeviceSample *scratch = nullptr;  // [S]
    double *d_eps2 = nullptr;         // [2][S] new strain, affine scale
    SpringType *types = nullptr;
    TypeDF *tdf = nullptr;
    double *tmass = nullptr, *tcoef = nullptr;
    uint8_t *export_buf = nullptr;
    int64_t export_cap = 0;
    int64_t cap = 0, nsamples = 0;
    int fix_S = 40;
    long long a_fix = 0;
    int64_t spring_updates = 0, launches = 0;
    std::map<int64_t, cudaGraphExec_t> graphs;
    std::map<int64_t, int64_t> graph_nodes;
    double relax_tol = -1.0;  // tolerance baked into the cached relax graphs
};

// ----------------------------------------------------------------- kernels

template <int TY, int PREC, int MODE, bool SAMPLE>
__global__ void __launch_bounds__(tile_threads<TY, PREC, SAMPLE>(), (tile_min_ctas<TY, PREC, SAMPLE>()))
k_tile2d_batch(TileArgs base, const BatchTile *__restrict__ tiles, int64_t t0, int64_t t1,
               const SpecDesc *__restrict__ specs, double *X0, double *X1, double *V0, double *V1, double *VOBS,
               const uint8_t *PH, uint8_t *MASK, long long *BRK, unsigned long long *fb,
               unsigned long long *nb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int64_t t = t0 + blockIdx.x; t < t1; t += gridDim.x) {
        const BatchTile bt = tiles[t];
        const SpecDesc &sd = specs[bt.spec];
        if (MODE == T_STEP && !sd.active) continue;  // uniform over the CTA
        TileArgs A = base;
        const int64_t P = sd.pbase;
        A.nx = sd.nx;
        A.ny = sd.ny;
        A.np = (int64_t)sd.nx * sd.ny;
        double *xa = (sd.cur ? X1 : X0) + 2 * P, *xb = (sd.cur ? X0 : X1) + 2 * P;
        double *va = (sd.cur ? V1 : V0) + 2 * P, *vb = (sd.cur ? V0 : V1) + 2 * P;
        A.x_in = xa;
        A.vh_in = va;
        A.x_out = xb;
        A.vh_out = MODE == T_INIT ? va : vb;
        A.v_obs = VOBS + 2 * P;
        A.phase = PH + P;
        A.mask = MASK + P;
        A.brk = BRK + 4 * P;
        A.first_break = fb + bt.spec;
        A.nbroken = nb + bt.spec;
        A.d_step = &specs[bt.spec].steps;
        A.t_off = 0;
        tile_body<32, TY, PREC, MODE, SAMPLE>(A, bt.bx, bt.by, t, smem_raw);
        __syncthreads();
    }
}

// A time step of the batch on strips: one warp per strip of 30 owned
// columns and R rows of one specimen (entries (spec, sx, sy) of `strips`;
// the schedule's grid does not apply), the single-specimen strip kernel's
// sweep on that specimen's arrays; a sample step writes the strip's partial
// sums at its index q in the strip list (stride base.ntiles, the number of
// strips; each specimen's strips are contiguous, its range sbase/nstiles).
// Same states as the tile kernel.
template <int PREC, bool SAMPLE>
__global__ void __launch_bounds__(32 * STRIP_WARPS, 5)
k_strip2d_batch(TileArgs base, const BatchTile *__restrict__ strips, int64_t n, int R,
                const SpecDesc *__restrict__ specs, double *X0, double *X1, double *V0, double *V1, double *VOBS,
                const uint8_t *PH, uint8_t *MASK, long long *BRK, unsigned long long *fb, unsigned long long *nb)
{
    __shared__ TypeDF sdf[128];
    __shared__ Coef4 scoef[8];
    __shared__ float smassf[8];
    __shared__ ff soff[4][3];
    strip_tables<PREC, 0>(base, sdf, scoef, smassf, soff);
    __syncthreads();
    const int64_t q = (int64_t)blockIdx.x * STRIP_WARPS + (threadIdx.x >> 5);
    if (q >= n) return;  // whole warps only
    {
        const BatchTile st = strips[q];
        const SpecDesc &sd = specs[st.spec];
        if (!sd.active) return;  // uniform over the warp
        TileArgs A = base;
        const int64_t P = sd.pbase;
        A.nx = sd.nx;
        A.ny = sd.ny;
        A.np = (int64_t)sd.nx * sd.ny;
        A.x_in = (sd.cur ? X1 : X0) + 2 * P;
        A.x_out = (sd.cur ? X0 : X1) + 2 * P;
        A.vh_in = (sd.cur ? V1 : V0) + 2 * P;
        A.vh_out = (sd.cur ? V0 : V1) + 2 * P;
        A.v_obs = VOBS + 2 * P;
        A.phase = PH + P;
        A.mask = MASK + P;
        A.brk = BRK + 4 * P;
        A.first_break = fb + st.spec;
        A.nbroken = nb + st.spec;
        A.d_step = &specs[st.spec].steps;
        A.t_off = 0;
        strip_run<PREC, false, SAMPLE, 0, T_STEP>(A, R, st.bx, st.by * R, q, sdf, scoef, smassf, soff);
    }
}

// After a step: active specimens advance their parity and step count.
__global__ void k_batch_flip(SpecDesc *specs, int S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S && specs[s].active) {
        specs[s].cur ^= 1;
        specs[s].steps += 1;
    }
}

__global__ void k_batch_set_active(SpecDesc *specs, int S, int v)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) specs[s].active = v;
}

// One block per specimen: fold its tiles' partials in a fixed order into a
// sample. relax: specimens whose residual is <= tol stop stepping; nactive
// counts the ones still active.
__global__ void __launch_bounds__(256)
k_batch_reduce(SpecDesc *specs, const double *__restrict__ ps, const double *__restrict__ pp, int64_t T,
               const unsigned long long *__restrict__ nb, DeviceSample *dst, int64_t cap,
               const long long *d_nsamp, int record, int relax, double tol, int *nactive)
{
    __shared__ double sh[8];
    const int s = blockIdx.x;
    SpecDesc &sd = specs[s];
    if (relax && !sd.active) return;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t t = sd.sbase + threadIdx.x; t < sd.sbase + sd.nstiles; t += 256) {
        acc[0] += ps[t];
        acc[1] += ps[T + t];
        acc[2] += pp[t];
        acc[3] += pp[T + t];
        acc[4] += pp[2 * T + t];
        acc[5] = fmax(acc[5], pp[3 * T + t]);
    }
    double r[6];
    for (int q = 0; q < 6; q++) r[q] = q == 5 ? bmax<8>(acc[q], sh) : bsum<8>(acc[q], sh);
    if (threadIdx.x == 0) {
        DeviceSample smp;
        smp.eps = sd.eps;
        smp.sigma_vir = (r[0] - r[2]) / sd.omega;
        smp.sigma_grip = r[4] / sd.grip_area;
        smp.pe = r[1];
        smp.ke = r[3];
        smp.residual = r[5];
        smp.n_broken = (long long)nb[s];
        smp.step = sd.steps;
        if (record) {
            const long long k = *d_nsamp;
            if (k < cap) dst[(int64_t)s * cap + k] = smp;
        } else {
            dst[s] = smp;
        }
        if (relax) {
            if (r[5] <= tol)
                sd.active = 0;
            else
                atomicAdd(nactive, 1);
        }
    }
}

__global__ void k_batch_count(long long *d_nsamp) { *d_nsamp += 1; }

// Load increment over the tile list (one CTA per tile, its owned pixels).
__global__ void __launch_bounds__(256)
k_batch_strain(const BatchTile *__restrict__ tiles, int64_t T, int TY, SpecDesc *specs, double *X0, double *X1,
               double *V0, double *V1, double *VOBS, const uint8_t *PH, const double *__restrict__ eps2, int S,
               double a, int affine)
{
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const BatchTile bt = tiles[t];
        const SpecDesc &sd = specs[bt.spec];
        const int64_t P = sd.pbase, np = (int64_t)sd.nx * sd.ny;
        double *x = (sd.cur ? X1 : X0) + 2 * P;
        double *vh = (sd.cur ? V1 : V0) + 2 * P;
        const double eps = eps2[bt.spec], scale = eps2[S + bt.spec];
        for (int e = threadIdx.x; e < 32 * TY; e += blockDim.x) {
            const int gx = bt.bx * 32 + (e & 31), gy = bt.by * TY + (e >> 5);
            if (gx >= sd.nx || gy >= sd.ny) continue;
            const int64_t g = (int64_t)gy * sd.nx + gx;
            if (!PH[P + g]) continue;
            double xp = x[g];
            if (affine) xp = ad(sd.xc, ml(sb(xp, sd.xc), scale));
            if (gx == 0 || gx == sd.nx - 1) {
                const double X = gx * a;
                xp = ad(X, ml(eps, sb(X, sd.xc)));
                vh[g] = 0.0;
                VOBS[2 * P + g] = 0.0;
            }
            x[g] = xp;
        }
    }
}

// Displacement u = x - X (and phase) of every specimen, all H x W.
__global__ void __launch_bounds__(256)
k_batch_fields(const BatchTile *__restrict__ tiles, int64_t T, int TY, const SpecDesc *__restrict__ specs,
               const double *X0, const double *X1, const uint8_t *__restrict__ PH, float *__restrict__ u,
               uint8_t *__restrict__ phase, double a)
{
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const BatchTile bt = tiles[t];
        const SpecDesc &sd = specs[bt.spec];
        const int64_t P = sd.pbase, np = (int64_t)sd.nx * sd.ny;
        const double *x = (sd.cur ? X1 : X0) + 2 * P;
        for (int e = threadIdx.x; e < 32 * TY; e += blockDim.x) {
            const int gx = bt.bx * 32 + (e & 31), gy = bt.by * TY + (e >> 5);
            if (gx >= sd.nx || gy >= sd.ny) continue;
            const int64_t g = (int64_t)gy * sd.nx + gx;
            const int64_t o = (int64_t)bt.spec * np;
            u[2 * o + g] = (float)(x[g] - gx * a);
            u[2 * o + np + g] = (float)(x[np + g] - gy * a);
            if (phase) phase[o + g] = PH[P + g];
        }
    }
}

// x += du on the free components of every specimen (all H x W).
__global__ void __launch_bounds__(256)
k_batch_add_du(const BatchTile *__restrict__ tiles, int64_t T, int TY, const SpecDesc *__restrict__ specs,
               double *X0, double *X1, const uint8_t *__restrict__ PH, const float *__restrict__ du, int grip_mode)
{
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const BatchTile bt = tiles[t];
        const SpecDesc &sd = specs[bt.spec];
        const int64_t P = sd.pbase, np = (int64_t)sd.nx * sd.ny;
        double *x = (sd.cur ? X1 : X0) + 2 * P;
        for (int e = threadIdx.x; e < 32 * TY; e += blockDim.x) {
            const int gx = bt.bx * 32 + (e & 31), gy = bt.by * TY + (e >> 5);
            if (gx >= sd.nx || gy >= sd.ny) continue;
            const int64_t g = (int64_t)gy * sd.nx + gx;
            if (!PH[P + g]) continue;
            const bool grip = gx == 0 || gx == sd.nx - 1;
            const int64_t o = (int64_t)bt.spec * np;
            if (!grip) x[g] += (double)du[2 * o + g];
            if (!(grip && grip_mode == 1)) x[np + g] += (double)du[2 * o + np + g];
        }
    }
}

__global__ void k_batch_set_eps(SpecDesc *specs, const double *eps2, int S)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) specs[s].eps = eps2[s];
}

// ------------------------------------------------------------------- host

#define BT_TRY(x)                             \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return e_;     \
    } while (0)

template <typename T>
static cudaError_t balloc(T **p, size_t count)
{
    return lsm::dev_malloc((void **)p, (count ? count : 1) * sizeof(T));
}

// Captured step graphs bake in the tile list, the grid and the buffers; any
// change of those drops them.
static void drop_graphs(BatchCtx &b)
{
    for (auto &kv : b.graphs) cudaGraphExecDestroy(kv.second);
    b.graphs.clear();
}

static void batch_free(BatchCtx &b)
{
    drop_graphs(b);
    if (b.stiles && b.stiles != b.tiles) cudaFree(b.stiles);
    b.stiles = nullptr;
    void *ptrs[] = {b.X[0], b.X[1], b.VH[0], b.VH[1], b.VOBS, b.PH, b.MASK, b.BRK, b.SBASE, b.specs, b.tiles,
                    b.strips, b.part_s, b.part_p, b.fb, b.nb, b.status, b.nactive, b.d_nsamp, b.samples,
                    b.scratch, b.d_eps2, b.types, b.tdf, b.tmass, b.tcoef, b.export_buf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

static ff split_ff_b(double v)
{
    const float hi = (float)v;
    return ff{hi, (float)(v - (double)hi)};
}

// (Re)build the tile list for tile height ty and order (0 natural, 1 largest
// specimen first), the 16-row list of the sample steps (the same list when ty
// is 16: the per-tile sample reductions would double on 8-row tiles) and the
// per-tile partial buffers, which only sample steps write. ty = -R (R 8, 16
// or 32): the plain steps run on strips of 30 owned columns and R rows, in
// the same specimen order, and the tiles (load increments, sample steps,
// fields) are 16 rows high.
static cudaError_t build_tiles(BatchCtx &b, int ty, int order)
{
    const int strip_r = ty < 0 ? -ty : 0;
    if (strip_r) ty = 16;
    constexpr int TYS = 16;
    std::vector<int> sorder(b.S);
    std::iota(sorder.begin(), sorder.end(), 0);
    if (order == 1)
        std::stable_sort(sorder.begin(), sorder.end(),
                         [&](int p, int q) { return (int64_t)b.nx[p] * b.ny[p] > (int64_t)b.nx[q] * b.ny[q]; });
    std::vector<BatchTile> tl, ts, sl;
    std::vector<SpecDesc> sd(b.S);
    BT_TRY(cudaMemcpyAsync(sd.data(), b.specs, b.S * sizeof(SpecDesc), cudaMemcpyDeviceToHost, b.stream));
    BT_TRY(cudaStreamSynchronize(b.stream));
    for (int s : sorder) {
        const int tx = (b.nx[s] + 31) / 32, tyn = (b.ny[s] + ty - 1) / ty, tys = (b.ny[s] + TYS - 1) / TYS;
        sd[s].tbase = (int64_t)tl.size();
        sd[s].ntiles = (int64_t)tx * tyn;
        for (int by = 0; by < tyn; by++)
            for (int bx = 0; bx < tx; bx++) tl.push_back(BatchTile{s, bx, by, 0});
        sd[s].sbase = (int64_t)ts.size();
        sd[s].nstiles = (int64_t)tx * tys;
        for (int by = 0; by < tys; by++)
            for (int bx = 0; bx < tx; bx++) ts.push_back(BatchTile{s, bx, by, 0});
        if (strip_r) {  // the sample steps too: the specimen's strips give its partial sums
            const int nsx = (b.nx[s] + STRIP_OWN - 1) / STRIP_OWN, nsy = (b.ny[s] + strip_r - 1) / strip_r;
            sd[s].sbase = (int64_t)sl.size();
            sd[s].nstiles = (int64_t)nsx * nsy;
            for (int sy = 0; sy < nsy; sy++)
                for (int sx = 0; sx < nsx; sx++) sl.push_back(BatchTile{s, sx, sy, 0});
        }
    }
    if (b.stiles && b.stiles != b.tiles) cudaFree(b.stiles);
    if (b.tiles) cudaFree(b.tiles);
    if (b.strips) cudaFree(b.strips);
    if (b.part_s) cudaFree(b.part_s);
    if (b.part_p) cudaFree(b.part_p);
    b.tiles = b.stiles = b.strips = nullptr;
    b.part_s = b.part_p = nullptr;
    b.NSTRIP = 0;
    if (strip_r) {
        BT_TRY(balloc(&b.strips, sl.size()));
        BT_TRY(cudaMemcpyAsync(b.strips, sl.data(), sl.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, b.stream));
        b.NSTRIP = (int64_t)sl.size();
    }
    b.T = (int64_t)tl.size();
    b.TS = strip_r ? (int64_t)sl.size() : (int64_t)ts.size();  // partial sums per sample-step unit
    BT_TRY(balloc(&b.tiles, tl.size()));
    if (ty == TYS) {
        b.stiles = b.tiles;
    } else {
        BT_TRY(balloc(&b.stiles, ts.size()));
        BT_TRY(cudaMemcpyAsync(b.stiles, ts.data(), ts.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, b.stream));
    }
    BT_TRY(balloc(&b.part_s, 2 * b.TS));
    BT_TRY(balloc(&b.part_p, 4 * b.TS));
    BT_TRY(cudaMemcpyAsync(b.tiles, tl.data(), tl.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, b.stream));
    BT_TRY(cudaMemcpyAsync(b.specs, sd.data(), b.S * sizeof(SpecDesc), cudaMemcpyHostToDevice, b.stream));
    BT_TRY(cudaStreamSynchronize(b.stream));
    b.tile_y = ty;
    b.strip_r = strip_r;
    b.order = order;
    drop_graphs(b);
    return cudaSuccess;
}

// Whether the batch can take strip schedules: the fixed-point modes, and
// specimens small enough for the strip sweep's 32-bit pixel indices.
static bool batch_strips_ok(const BatchCtx &b)
{
    if (b.prec != LSM_PREC_DF && b.prec != LSM_PREC_F32) return false;
    for (int s = 0; s < b.S; s++)
        if (2 * (int64_t)b.nx[s] * b.ny[s] >= ((int64_t)1 << 30)) return false;
    return true;
}

static TileArgs batch_base_args(BatchCtx &b)
{
    TileArgs A{};
    A.nphase = b.nphase;
    A.types = b.types;
    A.tdf = b.tdf;
    A.mass = b.tmass;
    A.coef = (const Coef4 *)b.tcoef;
    A.dt = b.dt;
    A.hdt = 0.5 * b.dt;
    A.gamma = b.damping;
    A.a = b.a;
    A.grip_mode = b.grip_mode;
    A.S = b.fix_S;
    A.a_fix = b.a_fix;
    A.p24 = ldexpf(1.0f, 24 - b.fix_S);
    A.p0 = ldexpf(1.0f, -b.fix_S);
    A.df_bias = (unsigned)(896 + 24 - b.fix_S) << 20;
    A.status = b.status;
    A.part_s = b.part_s;
    A.part_p = b.part_p;
    A.ntiles = b.TS;  // partial sums come from the sample-step tiles or strips
    return A;
}

// Whether strips of R rows outnumber the warps of the batched strip kernel
// that fit on the device at once.
static bool batch_strips_fill(const BatchCtx &b, int R)
{
    int dev = 0, nsm = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_strip2d_batch<LSM_PREC_DF, false>, 32 * STRIP_WARPS, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int64_t strips = 0;
    for (int s = 0; s < b.S; s++)
        strips += (int64_t)((b.nx[s] + STRIP_OWN - 1) / STRIP_OWN) * ((b.ny[s] + R - 1) / R);
    return strips >= (int64_t)nb * STRIP_WARPS * nsm;
}

template <int PREC, bool SAMPLE>
static cudaError_t launch_bs(BatchCtx &b)
{
    if (b.NSTRIP <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((b.NSTRIP + STRIP_WARPS - 1) / STRIP_WARPS);  // one warp per strip
    k_strip2d_batch<PREC, SAMPLE><<<grid, 32 * STRIP_WARPS, 0, b.stream>>>(batch_base_args(b), b.strips, b.NSTRIP, b.strip_r,
                                                                    b.specs, b.X[0], b.X[1], b.VH[0], b.VH[1], b.VOBS,
                                                                    b.PH, b.MASK, b.BRK, b.fb, b.nb);
    b.launches += 1;
    return cudaGetLastError();
}

template <int TY, int PREC, int MODE, bool SAMPLE>
static cudaError_t launch_bt(BatchCtx &b, const BatchTile *tiles, int64_t t0, int64_t t1)
{
    auto kern = k_tile2d_batch<TY, PREC, MODE, SAMPLE>;
    const size_t smem = tile_smem_bytes<32, TY>(PREC);
    static bool configured = false;
    if (!configured) {
        BT_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BT_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        configured = true;
    }
    const int64_t ntl = t1 - t0;
    if (ntl <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)(b.grid > 0 && b.grid < ntl ? b.grid : ntl);
    kern<<<grid, tile_threads<TY, PREC, SAMPLE>(), smem, b.stream>>>(batch_base_args(b), tiles, t0, t1, b.specs, b.X[0], b.X[1],
                                                 b.VH[0], b.VH[1], b.VOBS, b.PH, b.MASK, b.BRK, b.fb, b.nb);
    b.launches += 1;
    return cudaGetLastError();
}

// Steps without a sample run on the tile list of the schedule's height;
// sample steps on the 16-row list (t0, t1 index the list used).
template <int MODE, bool SAMPLE>
static cudaError_t launch_b(BatchCtx &b, int64_t t0, int64_t t1)
{
#define BT_PREC(TYV, TL)                                                                          \
    switch (b.prec) {                                                                             \
    case LSM_PREC_EXACT64: return launch_bt<TYV, LSM_PREC_EXACT64, MODE, SAMPLE>(b, TL, t0, t1);  \
    case LSM_PREC_FAST64: return launch_bt<TYV, LSM_PREC_FAST64, MODE, SAMPLE>(b, TL, t0, t1);    \
    case LSM_PREC_F32: return launch_bt<TYV, LSM_PREC_F32, MODE, SAMPLE>(b, TL, t0, t1);          \
    default: return launch_bt<TYV, LSM_PREC_DF, MODE, SAMPLE>(b, TL, t0, t1);                     \
    }
    if (MODE == T_STEP && b.strip_r > 0) {  // time steps on strips
        if (b.prec == LSM_PREC_F32) return launch_bs<LSM_PREC_F32, SAMPLE>(b);
        return launch_bs<LSM_PREC_DF, SAMPLE>(b);
    }
    if constexpr (SAMPLE) {
        BT_PREC(16, b.stiles)
    } else {
        if (b.tile_y == 8) { BT_PREC(8, b.tiles) }
        if (b.tile_y == 32) { BT_PREC(32, b.tiles) }
        BT_PREC(16, b.tiles)
    }
#undef BT_PREC
}

// nsteps steps (+ sample on the last) and the per-specimen reduction.
static cudaError_t enqueue_batch_steps(BatchCtx &b, int64_t nsteps, int record, int relax, double tol)
{
    const unsigned sg = (unsigned)((b.S + 255) / 256);
    for (int64_t t = 0; t < nsteps; t++) {
        cudaError_t e = t == nsteps - 1 ? launch_b<T_STEP, true>(b, 0, b.TS) : launch_b<T_STEP, false>(b, 0, b.T);
        if (e != cudaSuccess) return e;
        k_batch_flip<<<sg, 256, 0, b.stream>>>(b.specs, b.S);
        b.launches += 1;
    }
    k_batch_reduce<<<b.S, 256, 0, b.stream>>>(b.specs, b.part_s, b.part_p, b.TS, b.nb,
                                               record ? b.samples : b.scratch, b.cap, b.d_nsamp, record, relax, tol,
                                               b.nactive);
    b.launches += 1;
    if (record) {
        k_batch_count<<<1, 1, 0, b.stream>>>(b.d_nsamp);
        b.launches += 1;
    }
    return cudaGetLastError();
}

static cudaError_t batch_steps_graph(BatchCtx &b, int64_t nsteps, int record, int relax, double tol)
{
    const int64_t key = nsteps * 8 + record * 4 + relax * 2;
    if (relax && tol != b.relax_tol) {  // tol is baked into relax graphs
        for (auto q = b.graphs.begin(); q != b.graphs.end();) {
            if (q->first & 2) {
                cudaGraphExecDestroy(q->second);
                q = b.graphs.erase(q);
            } else {
                ++q;
            }
        }
        b.relax_tol = tol;
    }
    auto it = b.graphs.find(key);
    if (it == b.graphs.end()) {
        cudaGraph_t g;
        const int64_t l0 = b.launches;
        BT_TRY(cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t ee = enqueue_batch_steps(b, nsteps, record, relax, tol);
        cudaError_t e = cudaStreamEndCapture(b.stream, &g);
        b.launches = l0;
        if (ee != cudaSuccess) return ee;
        if (e != cudaSuccess) return e;
        size_t nodes = 0;
        cudaGraphGetNodes(g, nullptr, &nodes);
        cudaGraphExec_t ex;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        b.graph_nodes[key] = (int64_t)nodes;
        it = b.graphs.emplace(key, ex).first;
    }
    BT_TRY(cudaGraphLaunch(it->second, b.stream));
    b.launches += b.graph_nodes[key];
    return cudaSuccess;
}

static cudaError_t batch_upload(BatchCtx &b, const std::vector<HostNet> &nets, const HostNet &h0)
{
    const int S = b.S;
    int64_t np_all = 0;
    b.pbase.resize(S);
    for (int s = 0; s < S; s++) {
        b.pbase[s] = np_all;
        np_all += (int64_t)b.nx[s] * b.ny[s];
    }
    b.NP = np_all;
    const int64_t NP = np_all;
    // fixed-point scale from the largest specimen
    int maxext = 0;
    for (int s = 0; s < S; s++) maxext = std::max(maxext, std::max(b.nx[s], b.ny[s]));
    const double extent = 4.0 * maxext * b.a + 16.0;
    b.fix_S = std::min(61 - (int)std::ceil(std::log2(extent)), 47 - (int)std::ceil(std::log2(b.a * std::sqrt(2.0))));
    b.fix_S = std::min(b.fix_S, 47 - (int)std::floor(std::log2(max_critical_length(h0.types))));
    b.a_fix = std::llround(std::ldexp(b.a, b.fix_S));
    for (int q = 0; q < 2; q++) {
        BT_TRY(balloc(&b.X[q], 2 * NP));
        BT_TRY(balloc(&b.VH[q], 2 * NP));
    }
    BT_TRY(balloc(&b.VOBS, 2 * NP));
    BT_TRY(balloc(&b.PH, NP));
    BT_TRY(balloc(&b.MASK, NP));
    BT_TRY(balloc(&b.BRK, 4 * NP));
    BT_TRY(balloc(&b.SBASE, NP));
    BT_TRY(balloc(&b.specs, S));
    BT_TRY(balloc(&b.fb, S));
    BT_TRY(balloc(&b.nb, S));
    BT_TRY(balloc(&b.status, 1));
    BT_TRY(balloc(&b.nactive, 1));
    BT_TRY(balloc(&b.d_nsamp, 1));
    b.cap = 256;
    BT_TRY(balloc(&b.samples, (size_t)S * b.cap));
    BT_TRY(balloc(&b.scratch, S));
    BT_TRY(balloc(&b.d_eps2, 2 * S));
    BT_TRY(balloc(&b.types, h0.types.size()));
    BT_TRY(balloc(&b.tdf, h0.types.size()));
    BT_TRY(balloc(&b.tmass, b.nphase));
    BT_TRY(balloc(&b.tcoef, 4 * b.nphase));
    cudaStream_t st = b.stream;
    // per-pixel arrays
    std::vector<double> Xg(2 * NP);
    std::vector<uint8_t> ph(NP);
    std::vector<int64_t> sbase(NP, 0);
    std::vector<SpecDesc> sd(S);
    for (int s = 0; s < S; s++) {
        const HostNet &h = nets[s];
        const int64_t P = b.pbase[s], np = (int64_t)b.nx[s] * b.ny[s];
        for (int64_t g = 0; g < np; g++) {
            Xg[2 * P + g] = (g % b.nx[s]) * b.a;
            Xg[2 * P + np + g] = (g / b.nx[s]) * b.a;
        }
        std::copy(h.phase.begin(), h.phase.end(), ph.begin() + P);
        for (int64_t sp = h.m - 1; sp >= 0; sp--) sbase[P + h.pix[h.si[sp]]] = sp;
        sd[s].nx = b.nx[s];
        sd[s].ny = b.ny[s];
        sd[s].pbase = P;
        sd[s].xc = h.xc;
        sd[s].omega = h.omega;
        sd[s].grip_area = h.grip_area;
        sd[s].eps = 0.0;
        sd[s].cur = 0;
        sd[s].active = 1;
        sd[s].steps = 0;
    }
    std::vector<double> mtab(b.nphase, 1.0), coef(4 * b.nphase, 0.0);
    for (int64_t p = 0; p < h0.n; p++) mtab[h0.phase[h0.pix[p]] - 1] = h0.mass[p];
    for (int q = 0; q < b.nphase; q++) {
        const double dt = b.dt, hdt = 0.5 * b.dt, g = b.damping, m = mtab[q];
        coef[4 * q + 0] = 1.0 - dt * g / m;
        coef[4 * q + 1] = dt / m;
        coef[4 * q + 2] = 1.0 - hdt * g / m;
        coef[4 * q + 3] = hdt / m;
    }
    std::vector<TypeDF> tdf(h0.types.size());
    for (size_t q = 0; q < h0.types.size(); q++) {
        const SpringType &t = h0.types[q];
        const double shell = (q & 1) ? 2.0 : 1.0;
        const double aa = std::ldexp((double)b.a_fix, -b.fix_S);
        const double p = t.r0 * t.r0, pe = std::fma(t.r0, t.r0, -p);
        const double o2 = shell * aa * aa, o2e = shell * std::fma(aa, aa, -(aa * aa));
        // DF kernels hold lengths in units of 2^(24-S) (exact power-of-two scaling)
        const double ul = b.prec == LSM_PREC_DF ? std::ldexp(1.0, b.fix_S - 24) : 1.0;
        tdf[q].k = split_ff_b(t.k);
        tdf[q].r0 = split_ff_b(t.r0 * ul);
        tdf[q].rc2 = split_ff_b(t.rc2 * ul * ul);
        tdf[q].cor = split_ff_b((o2 - p) + (o2e - pe));
    }
    for (int q = 0; q < 2; q++) {
        BT_TRY(cudaMemcpyAsync(b.X[q], Xg.data(), 2 * NP * sizeof(double), cudaMemcpyHostToDevice, st));
        BT_TRY(cudaMemsetAsync(b.VH[q], 0, 2 * NP * sizeof(double), st));
    }
    BT_TRY(cudaMemsetAsync(b.VOBS, 0, 2 * NP * sizeof(double), st));
    BT_TRY(cudaMemcpyAsync(b.PH, ph.data(), NP, cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemsetAsync(b.MASK, 0, NP, st));
    BT_TRY(cudaMemsetAsync(b.BRK, 0xff, 4 * NP * sizeof(long long), st));
    BT_TRY(cudaMemcpyAsync(b.SBASE, sbase.data(), NP * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemcpyAsync(b.specs, sd.data(), S * sizeof(SpecDesc), cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemsetAsync(b.fb, 0xff, S * sizeof(unsigned long long), st));
    BT_TRY(cudaMemsetAsync(b.nb, 0, S * sizeof(unsigned long long), st));
    BT_TRY(cudaMemsetAsync(b.status, 0, sizeof(int), st));
    BT_TRY(cudaMemsetAsync(b.d_nsamp, 0, sizeof(long long), st));
    BT_TRY(cudaMemcpyAsync(b.types, h0.types.data(), h0.types.size() * sizeof(SpringType), cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemcpyAsync(b.tdf, tdf.data(), tdf.size() * sizeof(TypeDF), cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemcpyAsync(b.tmass, mtab.data(), b.nphase * sizeof(double), cudaMemcpyHostToDevice, st));
    BT_TRY(cudaMemcpyAsync(b.tcoef, coef.data(), 4 * b.nphase * sizeof(double), cudaMemcpyHostToDevice, st));
    BT_TRY(cudaStreamSynchronize(st));
    // default schedule: largest specimens first, plain steps on 16-row
    // strips in the fixed-point modes when the strips fill the device (what
    // the autotuner picks on the benchmark's batches; a warp sweeping a strip
    // is latency-bound when few run), 16-row tiles otherwise
    BT_TRY(build_tiles(b, batch_strips_ok(b) && batch_strips_fill(b, 16) ? -16 : 16, 1));
    // initial acceleration of every specimen (vh = v + dt/2 a(0))
    {
        cudaError_t ei = launch_b<T_INIT, false>(b, 0, b.T);
        if (ei != cudaSuccess) return ei;
    }
    BT_TRY(cudaStreamSynchronize(st));
    return cudaSuccess;
}

// Device status -> lsm_status.
static lsm_status batch_status(BatchCtx &b)
{
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, b.status, sizeof(int), cudaMemcpyDeviceToHost, b.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b.stream);
    if (e != cudaSuccess) {
        b.err = std::string("synchronize: ") + cudaGetErrorString(e);
        return LSM_ECUDA;
    }
    if (st) {
        b.err = (st & 2) ? "position outside the fixed-point range" : "non-finite position or velocity";
        return LSM_ENONFINITE;
    }
    return LSM_OK;
}

}  // namespace lsm

// =================================================================== C ABI

struct lsm_batch : public lsm::BatchCtx {};

namespace {
thread_local std::string g_batch_err;

lsm_status bfail(lsm_batch *b, lsm_status st, const std::string &msg)
{
    if (b)
        b->err = msg;
    else
        g_batch_err = msg;
    return st;
}

lsm_status bcuda(lsm_batch *b, cudaError_t e, const char *where)
{
    return bfail(b, LSM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool spec_ok(lsm_batch *b, int32_t spec) { return b && spec >= 0 && spec < b->S; }

lsm_status grow_samples(lsm_batch *b)
{
    if (b->nsamples < b->cap) return LSM_OK;
    const int64_t nc = b->cap * 2;
    lsm::DeviceSample *ns = nullptr;
    cudaError_t e = lsm::dev_malloc((void **)&ns, (size_t)b->S * nc * sizeof(lsm::DeviceSample));
    if (e != cudaSuccess) return bfail(b, LSM_ENOMEM, "sample buffer growth failed");
    e = cudaMemcpy2DAsync(ns, nc * sizeof(lsm::DeviceSample), b->samples, b->cap * sizeof(lsm::DeviceSample),
                          b->cap * sizeof(lsm::DeviceSample), b->S, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        cudaFree(ns);
        return bcuda(b, e, "sample growth");
    }
    cudaFree(b->samples);
    b->samples = ns;
    b->cap = nc;
    drop_graphs(*b);
    return LSM_OK;
}

}  // namespace

extern "C" {

lsm_status lsm_build_batch(const lsm_desc *descs, int32_t count, lsm_batch **out)
{
    lsm::NvtxRange nvtx_("lsm_build_batch");
    if (!descs || !out || count < 1) return bfail(nullptr, LSM_EINVAL, "descs, out and count >= 1 are required");
    *out = nullptr;
    const lsm_desc &d0 = descs[0];
    if (d0.precision < LSM_PREC_EXACT64 || d0.precision > LSM_PREC_DF)
        return bfail(nullptr, LSM_EINVAL, "bad precision");
    if (d0.nphase < 1 || d0.nphase > 8) return bfail(nullptr, LSM_EINVAL, "batches support 1..8 phases");
    lsm_batch *b = new (std::nothrow) lsm_batch();
    if (!b) return bfail(nullptr, LSM_ENOMEM, "host allocation failed");
    b->S = count;
    b->prec = d0.precision;
    b->nphase = d0.nphase;
    b->dt = d0.dt;
    b->damping = d0.damping;
    b->a = d0.a;
    b->grip_mode = d0.grip_mode;
    b->load_mode = d0.load_mode;
    std::vector<lsm::HostNet> nets(count);
    b->nx.resize(count);
    b->ny.resize(count);
    b->n.resize(count);
    b->m.resize(count);
    b->pix.resize(count);
    b->eps.assign(count, 0.0);
    for (int s = 0; s < count; s++) {
        const lsm_desc &d = descs[s];
        if (d.dim != 2 || d.lattice != 0 || d.nphase != d0.nphase || d.dt != d0.dt || d.damping != d0.damping || d.a != d0.a ||
            d.grip_mode != d0.grip_mode || d.load_mode != d0.load_mode || d.precision != d0.precision) {
            delete b;
            return bfail(nullptr, LSM_EINVAL, "batch specimens must be 2D square-lattice images and share nphase, dt, damping, a, "
                                              "grip/load modes and precision");
        }
        lsm_desc dd = d;
        dd.k_tab = d0.k_tab;
        dd.epsc_tab = d0.epsc_tab;
        dd.mass_tab = d0.mass_tab;
        std::string err;
        bool ok;
        try {
            ok = lsm::net_from_image(dd, nets[s], err);
        } catch (const std::bad_alloc &) {
            delete b;
            return bfail(nullptr, LSM_ENOMEM, "host allocation failed during build");
        }
        if (!ok) {
            delete b;
            return bfail(nullptr, LSM_EINVAL, "specimen " + std::to_string(s) + ": " + err);
        }
        b->nx[s] = nets[s].nx;
        b->ny[s] = nets[s].ny;
        b->n[s] = nets[s].n;
        b->m[s] = nets[s].m;
        if (nets[s].n != (int64_t)nets[s].nx * nets[s].ny) b->pix[s] = nets[s].pix;
    }
    if (d0.stream) {
        b->stream = (cudaStream_t)d0.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return bfail(nullptr, LSM_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
        }
        b->own_stream = true;
    }
    cudaGetLastError();
    cudaError_t e = lsm::batch_upload(*b, nets, nets[0]);
    if (e != cudaSuccess) {
        g_batch_err = std::string("batch upload: ") + cudaGetErrorString(e);
        lsm_status st = e == cudaErrorMemoryAllocation ? LSM_ENOMEM : LSM_ECUDA;
        lsm::batch_free(*b);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return st;
    }
    *out = b;
    return LSM_OK;
}

void lsm_batch_destroy(lsm_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    lsm::batch_free(*b);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *lsm_batch_last_error(const lsm_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

lsm_status lsm_batch_sizes(lsm_batch *b, int32_t spec, int32_t *count, int64_t *n, int64_t *m)
{
    if (!b) return bfail(nullptr, LSM_EINVAL, "null batch");
    if (count) *count = b->S;
    if (n || m) {
        if (!spec_ok(b, spec)) return bfail(b, LSM_EINVAL, "specimen index out of range");
        if (n) *n = b->n[spec];
        if (m) *m = b->m[spec];
    }
    return LSM_OK;
}

lsm_status lsm_batch_set_schedule(lsm_batch *b, int32_t tile_y, int32_t grid, int32_t order)
{
    if (!b) return bfail(nullptr, LSM_EINVAL, "null batch");
    const int ay = tile_y < 0 ? -tile_y : tile_y;
    if ((ay != 8 && ay != 16 && ay != 32) || grid < 0 || (order != 0 && order != 1))
        return bfail(b, LSM_EINVAL, "tile_y must be 8, 16 or 32 (or -8, -16, -32: strips); grid >= 0; order 0 or 1");
    if (tile_y < 0 && !lsm::batch_strips_ok(*b))
        return bfail(b, LSM_EINVAL, "strip schedules need the F32 or DF mode and specimens below 2^29 pixels");
    if (grid != b->grid) lsm::drop_graphs(*b);
    b->grid = grid;
    const int cur = b->strip_r ? -b->strip_r : b->tile_y;
    if (tile_y != cur || order != b->order) {
        cudaError_t e = lsm::build_tiles(*b, tile_y, order);
        if (e != cudaSuccess) return bcuda(b, e, "schedule");
    }
    return LSM_OK;
}

lsm_status lsm_batch_apply_strain(lsm_batch *b, const double *eps)
{
    lsm::NvtxRange nvtx_("lsm_batch_apply_strain");
    if (!b || !eps) return bfail(b, LSM_EINVAL, "null argument");
    std::vector<double> e2(2 * b->S);
    for (int s = 0; s < b->S; s++) {
        if (!std::isfinite(eps[s]) || !(1.0 + eps[s] > 0.0)) return bfail(b, LSM_EINVAL, "strain must be > -1");
        e2[s] = eps[s];
        e2[b->S + s] = (1.0 + eps[s]) / (1.0 + b->eps[s]);
    }
    cudaError_t e = cudaMemcpyAsync(b->d_eps2, e2.data(), 2 * b->S * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "apply_strain");
    const unsigned grid = (unsigned)std::min<int64_t>(b->T, 152 * 16);
    lsm::k_batch_strain<<<grid, 256, 0, b->stream>>>(b->tiles, b->T, b->tile_y, b->specs, b->X[0], b->X[1], b->VH[0],
                                                     b->VH[1], b->VOBS, b->PH, b->d_eps2, b->S, b->a,
                                                     b->load_mode == 0);
    lsm::k_batch_set_eps<<<(b->S + 255) / 256, 256, 0, b->stream>>>(b->specs, b->d_eps2, b->S);
    b->launches += 2;
    // the host array e2 must outlive the async copy
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "apply_strain");
    for (int s = 0; s < b->S; s++) b->eps[s] = eps[s];
    return LSM_OK;
}

lsm_status lsm_batch_step(lsm_batch *b, int64_t nsteps)
{
    lsm::NvtxRange nvtx_("lsm_batch_step");
    if (!b) return bfail(nullptr, LSM_EINVAL, "null batch");
    if (nsteps < 1 || nsteps > 100000) return bfail(b, LSM_EINVAL, "nsteps must be in 1..100000");
    lsm_status st = grow_samples(b);
    if (st != LSM_OK) return st;
    lsm::k_batch_set_active<<<(b->S + 255) / 256, 256, 0, b->stream>>>(b->specs, b->S, 1);
    b->launches += 1;
    cudaError_t e = lsm::batch_steps_graph(*b, nsteps, 1, 0, 0.0);
    if (e != cudaSuccess) return bcuda(b, e, "batch step");
    b->nsamples += 1;
    int64_t msum = 0;
    for (int s = 0; s < b->S; s++) msum += b->m[s];
    b->spring_updates += msum * nsteps;
    return LSM_OK;
}

lsm_status lsm_batch_relax(lsm_batch *b, double tol, int64_t max_steps, int64_t check_every, int64_t *taken,
                           int32_t *converged)
{
    lsm::NvtxRange nvtx_("lsm_batch_relax");
    if (!b) return bfail(nullptr, LSM_EINVAL, "null batch");
    if (!(tol >= 0) || max_steps < 1 || check_every < 1 || check_every > 100000)
        return bfail(b, LSM_EINVAL, "need tol >= 0, max_steps >= 1, 1 <= check_every <= 100000");
    lsm_status st = grow_samples(b);
    if (st != LSM_OK) return st;
    std::vector<lsm::SpecDesc> sd0(b->S), sd1(b->S);
    cudaError_t e = cudaMemcpyAsync(sd0.data(), b->specs, b->S * sizeof(lsm::SpecDesc), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "relax");
    lsm::k_batch_set_active<<<(b->S + 255) / 256, 256, 0, b->stream>>>(b->specs, b->S, 1);
    b->launches += 1;
    int64_t done = 0;
    int nact = b->S;
    while (done < max_steps && nact > 0) {
        const int64_t nb = std::min(check_every, max_steps - done);
        e = cudaMemsetAsync(b->nactive, 0, sizeof(int), b->stream);
        if (e == cudaSuccess) e = lsm::batch_steps_graph(*b, nb, 0, 1, tol);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nact, b->nactive, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "relax");
        st = lsm::batch_status(*b);
        if (st != LSM_OK) return st;
        done += nb;
    }
    // record one sample per specimen: every specimen's final state
    e = cudaMemcpyAsync(sd1.data(), b->specs, b->S * sizeof(lsm::SpecDesc), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "relax");
    std::vector<lsm::DeviceSample> last(b->S);
    e = cudaMemcpyAsync(last.data(), b->scratch, b->S * sizeof(lsm::DeviceSample), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "relax");
    bool all = true;
    int64_t su = 0;
    for (int s = 0; s < b->S; s++) {
        const int64_t ts = sd1[s].steps - sd0[s].steps;
        su += ts * b->m[s];
        const bool conv = sd1[s].active == 0;
        all &= conv;
        if (taken) taken[s] = ts;
        if (converged) converged[s] = conv ? 1 : 0;
        e = cudaMemcpyAsync(b->samples + (int64_t)s * b->cap + b->nsamples, &last[s], sizeof(lsm::DeviceSample),
                            cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "relax record");
    }
    const long long ns = b->nsamples + 1;
    e = cudaMemcpyAsync(b->d_nsamp, &ns, sizeof(ns), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "relax record");
    b->nsamples = ns;
    b->spring_updates += su;
    if (!all) return bfail(b, LSM_ENOTCONV, "some specimens above tolerance after max_steps");
    return LSM_OK;
}

lsm_status lsm_batch_samples(lsm_batch *b, int32_t spec, lsm_sample *out, int64_t cap, int64_t *count)
{
    if (!spec_ok(b, spec)) return bfail(b, LSM_EINVAL, "specimen index out of range");
    lsm_status st = lsm::batch_status(*b);
    if (st != LSM_OK) return st;
    const int64_t k = std::min<int64_t>(b->nsamples, cap);
    if (k > 0) {
        if (!out) return bfail(b, LSM_EINVAL, "null output");
        cudaError_t e = cudaMemcpyAsync(out, b->samples + (int64_t)spec * b->cap, k * sizeof(lsm_sample),
                                        cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "samples");
    }
    if (count) *count = b->nsamples;
    return LSM_OK;
}

static cudaError_t spec_desc(lsm_batch *b, int32_t spec, lsm::SpecDesc &sd)
{
    cudaError_t e = cudaMemcpyAsync(&sd, b->specs + spec, sizeof(sd), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e;
}

lsm_status lsm_batch_get_state(lsm_batch *b, int32_t spec, double *x, double *v)
{
    if (!spec_ok(b, spec)) return bfail(b, LSM_EINVAL, "specimen index out of range");
    lsm_status st = lsm::batch_status(*b);
    if (st != LSM_OK) return st;
    lsm::SpecDesc sd;
    cudaError_t e = spec_desc(b, spec, sd);
    if (e != cudaSuccess) return bcuda(b, e, "get_state");
    const int64_t np = (int64_t)b->nx[spec] * b->ny[spec], n = b->n[spec], P = b->pbase[spec];
    std::vector<double> gx(x ? 2 * np : 0), gv(v ? 2 * np : 0);
    if (x) e = cudaMemcpyAsync(gx.data(), b->X[sd.cur] + 2 * P, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && v)
        e = cudaMemcpyAsync(gv.data(), b->VOBS + 2 * P, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "get_state");
    const std::vector<int64_t> &pix = b->pix[spec];
    for (int c = 0; c < 2; c++)
        for (int64_t p = 0; p < n; p++) {
            const int64_t g = pix.empty() ? p : pix[p];
            if (x) x[c * n + p] = gx[c * np + g];
            if (v) v[c * n + p] = gv[c * np + g];
        }
    return LSM_OK;
}

lsm_status lsm_batch_set_state(lsm_batch *b, int32_t spec, const double *x, const double *v)
{
    if (!spec_ok(b, spec)) return bfail(b, LSM_EINVAL, "specimen index out of range");
    lsm::SpecDesc sd;
    cudaError_t e = spec_desc(b, spec, sd);
    if (e != cudaSuccess) return bcuda(b, e, "set_state");
    const int64_t np = (int64_t)b->nx[spec] * b->ny[spec], n = b->n[spec], P = b->pbase[spec];
    std::vector<double> gx(2 * np), gv(2 * np);
    e = cudaMemcpyAsync(gx.data(), b->X[sd.cur] + 2 * P, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(gv.data(), b->VOBS + 2 * P, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "set_state");
    const std::vector<int64_t> &pix = b->pix[spec];
    for (int c = 0; c < 2; c++)
        for (int64_t p = 0; p < n; p++) {
            const int64_t g = pix.empty() ? p : pix[p];
            if (x) gx[c * np + g] = x[c * n + p];
            if (v) gv[c * np + g] = v[c * n + p];
        }
    e = cudaMemcpyAsync(b->X[sd.cur] + 2 * P, gx.data(), 2 * np * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->VOBS + 2 * P, gv.data(), 2 * np * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = lsm::launch_b<lsm::T_INIT, false>(*b, sd.tbase, sd.tbase + sd.ntiles);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "set_state");
    return LSM_OK;
}

lsm_status lsm_batch_broken_mask(lsm_batch *b, int32_t spec, uint8_t *out, int64_t cap, int64_t *m,
                                 int64_t *first_break_step)
{
    if (!spec_ok(b, spec)) return bfail(b, LSM_EINVAL, "specimen index out of range");
    if (!out || cap < b->m[spec]) return bfail(b, LSM_EINVAL, "output buffer smaller than the spring count");
    lsm_status st = lsm::batch_status(*b);
    if (st != LSM_OK) return st;
    cudaError_t e = cudaSuccess;
    if (b->export_cap < b->m[spec]) {
        if (b->export_buf) cudaFree(b->export_buf);
        b->export_buf = nullptr;
        e = lsm::dev_malloc((void **)&b->export_buf, b->m[spec] ? b->m[spec] : 1);
        if (e != cudaSuccess) return bfail(b, LSM_ENOMEM, "export buffer");
        b->export_cap = b->m[spec];
    }
    const int64_t np = (int64_t)b->nx[spec] * b->ny[spec], P = b->pbase[spec];
    lsm::k_tile_export<<<(unsigned)((np + 255) / 256), 256, 0, b->stream>>>(
        b->nx[spec], b->ny[spec], np, b->PH + P, b->MASK + P, b->BRK + 4 * P, b->SBASE + P, b->export_buf, nullptr, 0);
    unsigned long long fb = 0;
    if (b->m[spec]) e = cudaMemcpyAsync(out, b->export_buf, b->m[spec], cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&fb, b->fb + spec, sizeof(fb), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "broken_mask");
    if (m) *m = b->m[spec];
    if (first_break_step) *first_break_step = fb == ~0ull ? -1 : (int64_t)fb;
    return LSM_OK;
}

lsm_status lsm_batch_counters(lsm_batch *b, int64_t *spring_updates, int64_t *kernel_launches)
{
    if (!b) return bfail(nullptr, LSM_EINVAL, "null batch");
    if (spring_updates) *spring_updates = b->spring_updates;
    if (kernel_launches) *kernel_launches = b->launches;
    return LSM_OK;
}

lsm_status lsm_batch_synchronize(lsm_batch *b)
{
    if (!b) return bfail(nullptr, LSM_EINVAL, "null batch");
    return lsm::batch_status(*b);
}

static bool uniform_size(lsm_batch *b, int32_t H, int32_t W)
{
    for (int s = 0; s < b->S; s++)
        if (b->nx[s] != W || b->ny[s] != H) return false;
    return true;
}

lsm_status lsm_batch_fields(lsm_batch *b, float *u, uint8_t *phase, int32_t H, int32_t W)
{
    lsm::NvtxRange nvtx_("lsm_batch_fields");
    if (!b || !u) return bfail(b, LSM_EINVAL, "null argument");
    if (!uniform_size(b, H, W)) return bfail(b, LSM_EINVAL, "every specimen must be H x W");
    const unsigned grid = (unsigned)std::min<int64_t>(b->T, 152 * 16);
    lsm::k_batch_fields<<<grid, 256, 0, b->stream>>>(b->tiles, b->T, b->tile_y, b->specs, b->X[0], b->X[1], b->PH, u,
                                                     phase, b->a);
    b->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LSM_OK : bcuda(b, e, "fields");
}

lsm_status lsm_batch_add_displacements(lsm_batch *b, const float *du, int32_t H, int32_t W)
{
    lsm::NvtxRange nvtx_("lsm_batch_add_displacements");
    if (!b || !du) return bfail(b, LSM_EINVAL, "null argument");
    if (!uniform_size(b, H, W)) return bfail(b, LSM_EINVAL, "every specimen must be H x W");
    const unsigned grid = (unsigned)std::min<int64_t>(b->T, 152 * 16);
    lsm::k_batch_add_du<<<grid, 256, 0, b->stream>>>(b->tiles, b->T, b->tile_y, b->specs, b->X[0], b->X[1], b->PH, du,
                                                     b->grip_mode);
    b->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = lsm::launch_b<lsm::T_INIT, false>(*b, 0, b->T);
    return e == cudaSuccess ? LSM_OK : bcuda(b, e, "add_displacements");
}

lsm_status lsm_batch_autotune(lsm_batch *b, int32_t steps_per_trial, int32_t *tile_y, int32_t *grid, int32_t *order,
                              double *ms_per_step)
{
    lsm::NvtxRange nvtx_("lsm_batch_autotune");
    if (!b) return bfail(nullptr, LSM_EINVAL, "null batch");
    if (steps_per_trial < 1 || steps_per_trial > 1000) return bfail(b, LSM_EINVAL, "steps_per_trial in 1..1000");
    // save the state the trials will advance
    const size_t x2 = 2 * b->NP * sizeof(double);
    void *bk[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    const size_t sz[7] = {x2, x2, x2, x2, x2, (size_t)b->NP, 4 * b->NP * sizeof(long long)};
    void *src[7] = {b->X[0], b->X[1], b->VH[0], b->VH[1], b->VOBS, b->MASK, b->BRK};
    std::vector<lsm::SpecDesc> sd0(b->S);
    std::vector<unsigned long long> fb0(b->S), nb0(b->S);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 7 && e == cudaSuccess; q++) {
        e = lsm::dev_malloc(&bk[q], sz[q]);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bk[q], src[q], sz[q], cudaMemcpyDeviceToDevice, b->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sd0.data(), b->specs, b->S * sizeof(lsm::SpecDesc), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fb0.data(), b->fb, b->S * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nb0.data(), b->nb, b->S * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    const int64_t launches0 = b->launches;
    double best = 1e300;
    const int cur_ty = b->strip_r ? -b->strip_r : b->tile_y;
    int bty = cur_ty, bgrid = b->grid, bord = b->order;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // tile heights 8, 16, 32, and in the fixed-point modes strips of 8, 16
    // or 32 rows (-R)
    const int tys[6] = {8, 16, 32, -8, -16, -32};
    const int nty = lsm::batch_strips_ok(*b) ? 6 : 3;
    // Two sweeps over the 18 (36) schedules, each keeping its faster trial;
    // the GPU is brought to its load clocks first (steps of the current
    // schedule), so that the first candidates are not timed at idle clocks.
    double tbest[6][2][3];
    for (int it = 0; it < 6; it++)
        for (int ord = 0; ord < 2; ord++)
            for (int gi = 0; gi < 3; gi++) tbest[it][ord][gi] = 1e300;
    if (e == cudaSuccess) e = lsm::build_tiles(*b, cur_ty, b->order);
    for (int w = 0; w < 4 && e == cudaSuccess; w++) e = lsm::batch_steps_graph(*b, steps_per_trial, 0, 0, 0.0);
    for (int sweep = 0; sweep < 2 && e == cudaSuccess; sweep++)
        for (int it = 0; it < nty && e == cudaSuccess; it++)
            for (int ord = 0; ord < 2 && e == cudaSuccess; ord++) {
                e = lsm::build_tiles(*b, tys[it], ord);
                const int grids[3] = {0, nsm * 4, nsm * 8};
                for (int gi = 0; gi < 3 && e == cudaSuccess; gi++) {
                    if (tys[it] < 0 && gi > 0) continue;  // strips: one warp each, the grid does not apply
                    b->grid = grids[gi];
                    lsm::drop_graphs(*b);  // the cached graphs hold the previous grid
                    e = lsm::batch_steps_graph(*b, steps_per_trial, 0, 0, 0.0);  // warm (captures the graph)
                    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
                    if (e == cudaSuccess) e = lsm::batch_steps_graph(*b, steps_per_trial, 0, 0, 0.0);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e == cudaSuccess && ms / steps_per_trial < tbest[it][ord][gi]) tbest[it][ord][gi] = ms / steps_per_trial;
                }
            }
    for (int it = 0; it < nty; it++)
        for (int ord = 0; ord < 2; ord++)
            for (int gi = 0; gi < 3; gi++)
                if (tbest[it][ord][gi] < best) {
                    best = tbest[it][ord][gi];
                    bty = tys[it];
                    bgrid = gi == 0 ? 0 : nsm * 4 * gi;
                    bord = ord;
                }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // restore the state and apply the winner
    for (int q = 0; q < 7; q++)
        if (bk[q] && e == cudaSuccess) e = cudaMemcpyAsync(src[q], bk[q], sz[q], cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->specs, sd0.data(), b->S * sizeof(lsm::SpecDesc), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->fb, fb0.data(), b->S * 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->nb, nb0.data(), b->S * 8, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    for (int q = 0; q < 7; q++)
        if (bk[q]) cudaFree(bk[q]);
    b->launches = launches0;
    if (e == cudaSuccess) {
        b->grid = bgrid;
        e = lsm::build_tiles(*b, bty, bord);  // also refreshes tile bases in the restored descriptors
    }
    if (e != cudaSuccess) return bcuda(b, e, "autotune");
    if (tile_y) *tile_y = bty;
    if (grid) *grid = bgrid;
    if (order) *order = bord;
    if (ms_per_step) *ms_per_step = best;
    return LSM_OK;
}

}  // extern "C"
