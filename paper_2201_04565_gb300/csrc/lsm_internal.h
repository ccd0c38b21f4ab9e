// lsm_internal.h -- device data layout and internal entry points of liblsm.
//
// Layout in HBM (one context = one specimen):
//   particles (n):   x[dim][n], v[dim][n], a[dim][n]   FP64, component-major
//                    mass[n] FP64, fixm[n] u8 (bit c = component c prescribed),
//                    grip[n] u8 (0 / 1 left / 2 right), Xx[n] FP64 reference x
//   springs (m):     si[m], sj[m] int32 (si < sj, canonical order),
//                    stype[m] u16 -> params table {k, r0, rc2, k*r0},
//                    state[m] u8 (1 = broken), brk[m] int64 (step of break or -1)
//   incidence CSR:   row[n+1] int64, inc[2m] u32 = (spring << 1) | side,
//                    side 0: particle is the lower endpoint i, 1: upper j;
//                    each row lists a particle's springs by ascending index
//   spring forces:   fs[dim][m] FP64 force on the lower endpoint (force pass
//                    output, gather input)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdlib>
#include <map>
#include <string>
#include <vector>

#include "../../include/lsm.h"
#include "nvtx_range.h"

namespace lsm {

// Every device allocation of the library. LSM_MAX_ALLOC_BYTES (environment,
// bytes; unset or 0 = no limit) caps a single allocation: larger requests
// fail as if the device were out of memory, which exercises the error and
// clean-up paths of builds without exhausting a real device (fault
// injection for tests).
inline cudaError_t dev_malloc_bytes(void **p, size_t bytes)
{
    const char *cap = std::getenv("LSM_MAX_ALLOC_BYTES");
    if (cap && *cap) {
        const unsigned long long lim = std::strtoull(cap, nullptr, 10);
        if (lim > 0 && bytes > lim) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc_bytes((void **)p, bytes);
}

struct SpringType {
    double k, r0, rc2, kr0;
};

// The longest critical length rc = sqrt(rc2) of a type table (at least 1):
// the fixed-point scale keeps every spring vector up to it exactly
// convertible.
inline double max_critical_length(const std::vector<SpringType> &types)
{
    double r = 1.0;
    for (const SpringType &t : types)
        if (t.rc2 > r * r) r = std::sqrt(t.rc2);
    return r;
}

// A double-float: the unevaluated sum hi + lo of two floats.
struct ff {
    float hi, lo;
};

// Spring type in double-float form for the fixed-point spring modes:
// cor = |o|^2 - r0^2 for the type's lattice vector o (0 up to rounding).
struct TypeDF {
    ff k, r0, rc2, cor;
};

// Reduction slots of one sample (partials are reduced in a fixed order).
enum {
    RED_W = 0,      // sum over intact springs of d_x * f_x (virial, Eq. 7)
    RED_PE,         // potential energy, Eq. 1
    RED_MVX2,       // sum m v_x^2
    RED_KE,         // kinetic energy
    RED_REACT,      // sum over right-grip particles of -F_x
    RED_RES,        // max over free components of max(|F|, |v|)  (max, not sum)
    RED_NSLOT
};

struct DeviceSample {  // mirrors lsm_sample
    double eps, sigma_vir, sigma_grip, pe, ke, residual;
    long long n_broken, step;
};

// Host-side description of a network before upload.
struct HostNet {
    int dim = 2;
    int64_t n = 0, m = 0;
    std::vector<double> X;       // dim*n
    std::vector<double> mass;    // n
    std::vector<uint8_t> fixm;   // n, bit c
    std::vector<uint8_t> grip;   // n
    std::vector<int32_t> si, sj;
    std::vector<uint16_t> stype;
    std::vector<SpringType> types;
    double dt = 0.01, damping = 0.0, xc = 0.0, omega = 1.0, grip_area = 1.0;
    int load_mode = 0;
    int precision = LSM_PREC_EXACT64;
    int grip_mode = 0;
    double a = 1.0;
    int lattice = 0;               // 0 square / cubic, 1 triangular packing (image builds)
    double cell = 1.0;             // volume per particle (lsm_fields default)
    // image geometry (0 for network builds)
    int nx = 0, ny = 0, nz = 0, nphase = 0;
    std::vector<int64_t> pix;      // pixel of each particle (image builds)
    std::vector<uint8_t> phase;    // nx*ny*nz phase image (image builds)
    std::vector<uint8_t> sdir;     // per spring: index of its lattice offset (image builds)
    std::vector<double> offv;      // lattice vectors (x, y, z) by offset index (image builds)
};

struct Ctx {
    HostNet h;  // host copy of topology (kept for queries and rebuilds)
    int dim = 2;
    int64_t n = 0, m = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    // device particle state
    double *x = nullptr, *v = nullptr, *a = nullptr;
    double *mass = nullptr, *Xx = nullptr;
    uint8_t *fixm = nullptr, *grip = nullptr;
    // device springs
    int32_t *si = nullptr, *sj = nullptr;
    uint16_t *stype = nullptr;
    SpringType *types = nullptr;
    uint8_t *state = nullptr;
    long long *brk = nullptr;
    int64_t *row = nullptr;
    uint32_t *inc = nullptr;
    double *fs = nullptr;
    // reductions
    double *part_s = nullptr;  // [2][nblk_s]   W, PE per spring block
    double *part_p = nullptr;  // [4][nblk_p]   MVX2, KE, REACT, RES per particle block
    int64_t nblk_s = 0, nblk_p = 0;
    // device scalars: step counter, first break, broken count, status, eps,
    // sample count
    long long *d_step = nullptr;
    unsigned long long *d_first_break = nullptr;
    unsigned long long *d_nbroken = nullptr;
    int *d_status = nullptr;
    double *d_eps = nullptr;
    long long *d_nsamples = nullptr;
    DeviceSample *samples = nullptr;
    int64_t sample_cap = 0;
    int64_t nsamples = 0;  // host mirror
    DeviceSample *scratch_sample = nullptr;

    // 2D tile path (image lattices): state on the pixel grid, ping-pong
    bool tile = false;
    bool strip = false;                   // 2D time steps on the strip kernel (strip2d.cu)
    bool strip_forced = false;            // path 3: the strip kernel whatever the image size
    int path_req = 0;                     // the build's path request (kept by checkpoints)
    bool tri = false;                     // tile path of the triangular packing (strip kernel only)
    int tgnx = 0, tgny = 0;               // 2D tile grid: pixels, or sites (nx per row, rows) of the packing
    std::vector<int64_t> tgidx;           // [n] grid index of each particle (host)
    long long h_fix = 0;                  // packing: row height a sqrt(3)/2 in fixed point
    int strip_R = 0, strip_nsx = 0;       // rows per strip, strips across
    int64_t nstrips = 0;                  // strips (= partial sums of a strip sample step)
    int tile_nphase = 0;
    int64_t tnp = 0;                      // pixels
    double *tx[2] = {nullptr, nullptr};   // [2][tnp] positions
    double *tvh[2] = {nullptr, nullptr};  // [2][tnp] half-step velocities
    double *tvobs = nullptr;              // [2][tnp] full-step velocities (queries)
    uint8_t *tph = nullptr, *tmask = nullptr;
    uint16_t *tmask3 = nullptr;           // 3D tile path: 9 broken flags per voxel
    long long *tbrk = nullptr;            // [4][tnp]
    double *tmass = nullptr;              // per phase
    double *tinvm = nullptr;              // per phase: 1 - dt g/m, dt/m, 1 - dt/2 g/m, dt/2 / m
    TypeDF *tdf = nullptr;                // double-float spring types
    int fix_S = 40;                       // fixed-point scale of positions
    long long a_fix = 0;                  // lattice spacing * 2^fix_S
    int64_t *tsbase = nullptr;            // [tnp] canonical index of each pixel's first spring
    // spring-list path in the fixed-point modes (image builds, F32 / DF)
    bool fixcsr = false;
    long long *xf = nullptr;              // [dim][n] positions * 2^fix_S
    uint8_t *sdir = nullptr;              // [m] lattice offset index of each spring
    double *imass = nullptr;              // [n] 1 / mass
    void *fsx = nullptr;                  // [dim][m] spring forces (float or double-float)
    // per-particle fields (allocated by the first lsm_fields call)
    double *fX = nullptr;                 // [dim][n] reference positions
    double *fx = nullptr, *fv = nullptr;  // [dim][n] compact x, v (tile path)
    double *fout = nullptr;               // [2][6][n] stress and strain
    int64_t *frow = nullptr;              // [n+1] (tile path; the spring-list path uses row)
    uint32_t *finc = nullptr;             // [2m]
    int32_t *fsi = nullptr, *fsj = nullptr;
    uint16_t *fstype = nullptr;
    double *fmass = nullptr;              // [n]
    int64_t *fpix = nullptr;              // [n] pixel of each particle
    uint8_t *texport = nullptr;           // [m] staging for canonical-order exports
    long long *texport_brk = nullptr;     // [m] staging for break steps

    // asynchronous readback (lsm_readback_async): a second stream for the
    // device-to-host copies, two device snapshots of the canonical mask with
    // their events (ready: snapshot written on `stream`; done: copied out)
    cudaStream_t rb_stream = nullptr;
    uint8_t *rb_buf[2] = {nullptr, nullptr};
    cudaEvent_t rb_ready[2] = {nullptr, nullptr}, rb_done[2] = {nullptr, nullptr};
    bool rb_used[2] = {false, false};
    int64_t rb_count = 0;
    int tcur = 0;
    int64_t ntiles = 0;

    // constant strain-rate loading: eps(s) = rate_eps0 + (s - rate_step0) rate_dt
    bool rate_on = false;
    double rate_eps0 = 0.0, rate_dt = 0.0;
    long long rate_step0 = 0;
    int32_t *grip_list = nullptr;  // spring-list path: particles with a prescribed x
    int64_t ngrip = 0;

    double eps = 0.0;  // host mirror of the applied strain
    int64_t steps = 0; // host mirror of the step counter
    int64_t launches = 0;  // kernels launched (graph nodes included)
    std::map<int64_t, int64_t> graph_nodes;  // kernels per cached graph
    std::map<int64_t, cudaGraphExec_t> graphs;
};

// checkpoint.cpp: lsm_save / lsm_load
struct CkptState {
    uint32_t path = 0, tile = 0;  // build path (0 automatic, 1 spring list); ran on a tile path
    double eps = 0.0;
    int64_t steps = 0, nsamples = 0, launches = 0;
    int32_t rate_on = 0;
    double rate_eps0 = 0.0, rate_dt = 0.0;
    long long rate_step0 = 0;
    long long d_step = 0;
    unsigned long long first_break = 0, nbroken = 0;
    int32_t status = 0;
    double d_eps = 0.0;
    long long d_nsamples = 0;
    std::vector<DeviceSample> samples;
    std::vector<std::vector<uint8_t>> bufs;  // the path's state buffers
};
// device -> file; err set (and cudaSuccess returned) on an I/O failure
cudaError_t checkpoint_save(Ctx &c, const char *path, std::string &err);
// file -> host (no device work); false with err on a malformed file
bool checkpoint_read(const char *path, HostNet &h, CkptState &s, std::string &err);
// host -> the device buffers of a context freshly built from the same network
cudaError_t checkpoint_restore(Ctx &c, const CkptState &s, std::string &err);

// api.cpp: message returned by lsm_last_error(NULL) on this thread
void set_thread_error(const char *msg);

// build.cpp
bool net_from_image(const lsm_desc &d, HostNet &out, std::string &err);
bool net_from_desc(const lsm_net_desc &d, HostNet &out, std::string &err);

// kernels.cu
cudaError_t upload(Ctx &c);
cudaError_t launch_init_accel(Ctx &c);
cudaError_t launch_steps(Ctx &c, int64_t nsteps, bool record);
cudaError_t launch_apply_strain(Ctx &c, double eps_old, double eps_new);
cudaError_t launch_observe(Ctx &c, DeviceSample *dst);
void free_device(Ctx &c);

// csr_fix.cu: spring-list path in the fixed-point modes (F32, DF)
cudaError_t fixcsr_upload(Ctx &c);   // scale, tables, fixed-point copy of x
cudaError_t fixcsr_refresh(Ctx &c);  // xf = x 2^S after x changed outside the step kernels
template <int DIM, bool BREAK, bool SAMPLE>
void springs_fix(Ctx &c);
template <int DIM, int MODE, bool SAMPLE>  // MODE: end / drift / init / observe, as the FP64 gather
void gather_fix(Ctx &c);

// fields.cu
cudaError_t fields_compute(Ctx &c, double cell);  // -> fout (device), stream ordered
void fields_free(Ctx &c);

// tile3d.cu: 3D voxel lattices in the fixed-point modes (state on the voxel grid)
cudaError_t tile3_upload(Ctx &c);
cudaError_t tile3_enqueue_steps(Ctx &c, int64_t nsteps, int start_buf);
cudaError_t tile3_init_accel(Ctx &c);
cudaError_t tile3_observe(Ctx &c);
cudaError_t tile3_export(Ctx &c, bool steps);
int64_t tile3_count(const Ctx &c);

// strip2d.cu: does this context's 2D tile path run its plain time steps on
// the register-resident strip kernel (square lattice, F32 / DF modes)?
bool strip_supported(const Ctx &c);
cudaError_t strip_geometry(Ctx &c, bool *fills);  // strip_R, strip_nsx, nstrips for this device

// tile2d.cu
cudaError_t tile_enqueue_steps(Ctx &c, int64_t nsteps, int start_buf);
cudaError_t tile_init_accel(Ctx &c);
cudaError_t tile_observe(Ctx &c);
cudaError_t tile_apply_strain(Ctx &c, double eps_old, double eps_new);
int64_t tile_count(const Ctx &c);
cudaError_t tile_export(Ctx &c, bool steps);  // canonical-order mask or break steps into staging
const char *last_fail_site();  // source text of the CUDA call that failed last

}  // namespace lsm
