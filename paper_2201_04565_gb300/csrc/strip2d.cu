// strip2d.cu -- the register-resident time step for 2D images in the
// fixed-point modes (F32, DF): one warp per strip (the sweep is in
// strip_body.cuh), and the host side that chooses the strip geometry.
#include "strip_body.cuh"

namespace lsm {

// One warp per strip of the image (strips numbered row-major, nsx across);
// partial sums of a sample at index `strip`.
template <int PREC, bool RATE, bool SAMPLE, int LAT, int MODE>
__global__ void __launch_bounds__(32 * STRIP_WARPS, strip_min_ctas<PREC, SAMPLE>())
k_strip2d(TileArgs A, int R, int nsx)
{
    __shared__ TypeDF sdf[128];
    __shared__ Coef4 scoef[8];
    __shared__ float smassf[8];
    __shared__ ff soff[4][3];  // per slot: o_x, o_y, |o|^2 (F32)
    strip_tables<PREC, LAT>(A, sdf, scoef, smassf, soff);
    __syncthreads();
    const int strip = blockIdx.x * STRIP_WARPS + (threadIdx.x >> 5);
    const int sx = strip % nsx, sy = strip / nsx;
    const int y0 = sy * R;
    if (y0 >= A.ny) return;  // whole warps only
    strip_run<PREC, RATE, SAMPLE, LAT, MODE>(A, R, sx, y0, strip, sdf, scoef, smassf, soff);
}

// ------------------------------------------------------------------ host

namespace {

// Warps of a time-step kernel that fit on the device at once.
template <typename Kern>
cudaError_t kernel_resident(Kern k, int &cached, int &resident)
{
    if (!cached) {
        int dev = 0, nsm = 0, nb = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 32 * STRIP_WARPS, 0);
        if (e != cudaSuccess) return e;
        cached = std::max(1, nb * STRIP_WARPS * nsm);
    }
    resident = cached;
    return cudaSuccess;
}

template <int PREC, int LAT>
cudaError_t strip_resident(int &resident)
{
    static int cached = 0;  // per instance
    return kernel_resident(k_strip2d<PREC, false, false, LAT, T_STEP>, cached, resident);
}

// Strips of `own` columns and R rows, one wave of `resident` warps, at least
// rmin rows each; fills: strips of 8 rows would outnumber the resident warps.
void strip_shape(int nx, int ny, int own, int resident, int rmin, int &R, int &nsx, int64_t &nstrips, bool &fills)
{
    nsx = (nx + own - 1) / own;
    const int rows_target = std::max(1, resident / nsx);
    R = std::max(rmin, (ny + rows_target - 1) / rows_target);
    nstrips = (int64_t)nsx * ((ny + R - 1) / R);
    fills = (int64_t)nsx * ((ny + 7) / 8) >= resident;
}

template <int PREC, bool RATE, bool SAMPLE, int LAT, int MODE>
void launch_strip_t(Ctx &c, TileArgs A)
{
    if (SAMPLE) A.ntiles = c.nstrips;  // partial-sum stride
    const unsigned grid = (unsigned)((c.nstrips + STRIP_WARPS - 1) / STRIP_WARPS);
    k_strip2d<PREC, RATE, SAMPLE, LAT, MODE><<<grid, 32 * STRIP_WARPS, 0, c.stream>>>(A, c.strip_R, c.strip_nsx);
}

template <int PREC, int LAT>
void launch_strip_step(Ctx &c, const TileArgs &A, bool sample)
{
    if (c.rate_on) {
        if (sample) launch_strip_t<PREC, true, true, LAT, T_STEP>(c, A);
        else launch_strip_t<PREC, true, false, LAT, T_STEP>(c, A);
    } else {
        if (sample) launch_strip_t<PREC, false, true, LAT, T_STEP>(c, A);
        else launch_strip_t<PREC, false, false, LAT, T_STEP>(c, A);
    }
}

}  // namespace

bool strip_supported(const Ctx &c)
{
    return c.dim == 2 && (c.h.lattice == 0 || c.h.lattice == 1) &&
           (c.h.precision == LSM_PREC_DF || c.h.precision == LSM_PREC_F32) &&
           2 * (int64_t)c.h.nx * c.h.ny < ((int64_t)1 << 30);  // 32-bit indices (the packing has < 2 ny rows)
}

// Strip geometry: one warp per strip of 30 owned columns and R rows, as many
// strips as fit on the device at once (one wave), but at least 8 rows each
// (2 on the triangular packing, which has no tile kernel to fall back to).
// *fills: whether the image is large enough for strips of 8 rows to occupy
// the whole device (otherwise the square lattice's tile kernel, with more
// CTAs in flight, is the faster choice: a warp's row-by-row sweep is
// latency-bound when few run).
cudaError_t strip_geometry(Ctx &c, bool *fills)
{
    int resident = 0;
    const bool df = c.h.precision == LSM_PREC_DF;
    cudaError_t e = c.tri ? (df ? strip_resident<LSM_PREC_DF, 1>(resident) : strip_resident<LSM_PREC_F32, 1>(resident))
                          : (df ? strip_resident<LSM_PREC_DF, 0>(resident) : strip_resident<LSM_PREC_F32, 0>(resident));
    if (e != cudaSuccess) return e;
    bool f = false;
    strip_shape(c.tgnx, c.tgny, STRIP_OWN, resident, c.tri ? 2 : 8, c.strip_R, c.strip_nsx, c.nstrips, f);
    if (fills) *fills = f;
    return cudaSuccess;
}

cudaError_t launch_strip(Ctx &c, const TileArgs &A, bool sample)
{
    const bool df = c.h.precision == LSM_PREC_DF;
    if (c.tri) {
        if (df) launch_strip_step<LSM_PREC_DF, 1>(c, A, sample);
        else launch_strip_step<LSM_PREC_F32, 1>(c, A, sample);
    } else {
        if (df) launch_strip_step<LSM_PREC_DF, 0>(c, A, sample);
        else launch_strip_step<LSM_PREC_F32, 0>(c, A, sample);
    }
    return cudaSuccess;
}

// The triangular packing's initial acceleration and observation (the square
// lattice runs both on the tile kernel).
cudaError_t launch_strip_mode(Ctx &c, const TileArgs &A, int mode)
{
    const bool df = c.h.precision == LSM_PREC_DF;
    if (mode == T_INIT) {
        if (df) launch_strip_t<LSM_PREC_DF, false, false, 1, T_INIT>(c, A);
        else launch_strip_t<LSM_PREC_F32, false, false, 1, T_INIT>(c, A);
    } else {
        if (df) launch_strip_t<LSM_PREC_DF, false, true, 1, T_OBSERVE>(c, A);
        else launch_strip_t<LSM_PREC_F32, false, true, 1, T_OBSERVE>(c, A);
    }
    return cudaSuccess;
}

}  // namespace lsm
