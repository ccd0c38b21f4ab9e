/*
 * lsm.h -- C ABI of the GB300 lattice-spring library (liblsm.so).
 *
 * The library runs the per-timestep update of a particle-spring network built
 * from a 2D image or a 3D voxel volume (arXiv 2201.04565, "ImageMech"):
 *   - spring force, Eq. 2 (harmonic spring, Eq. 1 potential);
 *   - the sum of spring forces onto particles, done as a deterministic
 *     particle-centric gather (no floating-point atomics; Section 2.3 uses
 *     atomicAdd there);
 *   - the irreversible break test (Section 2.3 force listing: a spring longer
 *     than rc gives zero force from then on; Section 4: broken springs stay);
 *   - damped velocity Verlet in the half-step-velocity form, Eqs. 3-5
 *     (Section 2.2), under displacement-controlled loading along x
 *     (Sections 2.3 and 3.1);
 *   - the virial stress, Eq. 7, and the energies (Section 2.3, output step).
 *
 * Conventions for every call:
 *   - Every function returns an lsm_status; LSM_OK is 0, errors are negative.
 *     lsm_last_error() gives a one-line reason for the last failure on a
 *     context. A context is not thread-safe.
 *   - Host pointers are plain host memory owned by the caller. Inputs are
 *     copied during the call; outputs are written into caller buffers of the
 *     stated size. The context owns all device memory it allocates.
 *   - Particle arrays are component-major: component c of particle p is at
 *     [c * n + p]. Particles of an image build are the non-void pixels or
 *     voxels in raster order (x fastest, then y, then z). Springs are in
 *     canonical order: endpoints i < j, sorted by (i, j).
 *   - Work is ordered on the context's CUDA stream. lsm_apply_strain and
 *     lsm_step may return before the device work ends; query calls
 *     (state, masks, samples) synchronise the stream. An asynchronous device
 *     error (non-finite state) is recorded in a device status word and is
 *     returned by the next synchronising call as LSM_ENONFINITE.
 */
#ifndef LSM_H
#define LSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsm_ctx lsm_ctx;

typedef enum {
    LSM_OK = 0,
    LSM_EINVAL = -1,      /* bad argument, size or descriptor field */
    LSM_ENOMEM = -2,      /* device or host allocation failed */
    LSM_ECUDA = -3,       /* a CUDA runtime call failed */
    LSM_ENOTCONV = -4,    /* relax hit max_steps before the tolerance */
    LSM_ETIMEOUT = -5,    /* a bounded device wait gave up */
    LSM_ENONFINITE = -6,  /* the state became non-finite */
    LSM_ESTATE = -7       /* call not valid in the context's current state */
} lsm_status;

/* Arithmetic of the spring pass (force evaluation and gather).
 *  LSM_PREC_EXACT64: IEEE double with correctly rounded sqrt and divide, no
 *      fused multiply-add, gather in canonical spring order: the same
 *      operations in the same order as the plain FP64 definition, so the
 *      state is bit-identical to a sequential FP64 evaluation.
 *  LSM_PREC_FAST64: double precision throughout, reassociated (fused
 *      multiply-add, 1/r from a reciprocal square root); results agree with
 *      the exact mode to a few ulps per step.
 *  LSM_PREC_F32: spring vector formed exactly (positions in 64-bit fixed
 *      point), spring force evaluated and gathered in single precision,
 *      positions and velocities integrated in double.
 *  LSM_PREC_DF: as LSM_PREC_F32, but the spring force and the gather use
 *      double-float arithmetic (pairs of floats, 48 significant bits; 1/r by
 *      one double-float Newton step, about 2^-45), so forces carry about
 *      3e-14 relative error while the FP64 pipe only does the integration.
 *      In both fixed-point modes every spring vector up to the longest
 *      critical length converts exactly, and a non-finite force (which only
 *      positions already out of range can produce) is reported by the next
 *      step's range check as LSM_ENONFINITE. For image builds DF and F32 run on the 2D strip or
 *      tile kernels (square lattice), the strip kernel (triangular
 *      packing), the 3D voxel tile kernel, or (path 1) the spring-list
 *      kernels with the same fixed-point spring vectors.
 *      Network builds have no lattice vectors:
 *      there F32 forms the spring vector in double and DF runs as
 *      LSM_PREC_FAST64. */
enum { LSM_PREC_EXACT64 = 0, LSM_PREC_FAST64 = 1, LSM_PREC_F32 = 2, LSM_PREC_DF = 3 };

/* Image build descriptor (the paper's Img2Particle stage, Section 1 and
 * Fig. 6, on a square/cubic lattice with first and second neighbours).
 *  dim          2 or 3.
 *  nx, ny, nz   image size; nz is ignored (taken as 1) when dim == 2. nx >= 2.
 *  phase        host, nx*ny*nz bytes, x fastest: 0 = void (no particle),
 *               1..nphase = material phase. Copied during the build.
 *  nphase       number of phases (1..181: the 2 nphase^2 spring types are
 *               indexed by 16 bits; the tile kernels take up to 8).
 *  k_tab        host, nphase*nphase doubles, row-major, entry
 *               [(pi-1)*nphase + (pj-1)]: spring constant between phases pi, pj.
 *  epsc_tab     same layout: critical strain; rc = r0 (1 + eps_c) (Table of
 *               spring constants, Section 3.1, gives rc per spring type).
 *  mass_tab     host, nphase doubles, particle mass by phase (NULL = all 1).
 *  k2_ratio     multiplier on k for second-neighbour (diagonal) springs.
 *  a            lattice spacing; first-neighbour r0 = a, second = a sqrt 2.
 *  dt           time step (Section 2.2).
 *  damping      viscous coefficient gamma: a = (F - gamma vh) / m.
 *  grip_mode    0 = roller grips (x component of the first and last image
 *               column prescribed), 1 = clamped (all components).
 *  load_mode    0 = each load increment remaps x of every particle affinely
 *               about the specimen centre, then sets the grips;
 *               1 = only the grips move.
 *  precision    LSM_PREC_* (see above).
 *  path         0 = automatic: images with up to 8 phases run on the grid
 *               of their pixels or sites. Square lattice: the fused tile
 *               kernel in every mode; in the F32 and DF modes, when the
 *               image is large enough for its strips to fill the device,
 *               the time steps run on the register-resident strip kernel
 *               instead (the same positions, velocities and breaks; sample
 *               sums grouped per strip). Triangular packing (F32, DF): the
 *               strip kernel. 3D (F32, DF): the voxel tile kernel.
 *               Everything else: the general spring-list kernels.
 *               1 = always the general spring-list kernels;
 *               2 = as 0, but every square-lattice 2D step on the tile kernel;
 *               3 = as 0, but the 2D F32 / DF steps on the strip kernel
 *               whatever the image size.
 *  stream       cudaStream_t to order work on (NULL = the library creates one).
 *  lattice      0 = square (2D) / cubic (3D) lattice as above; 1 = the
 *               paper's triangular packing (2D only, Section 1: six first
 *               neighbours per interior particle, r0 = a, k2_ratio unused).
 *               Rows iy = 0..R-1 at y = iy h, h = (a sqrt 3) 0.5, for every
 *               iy with iy sqrt(3)/2 <= ny - 1; row iy has nx sites at
 *               x = ix a (even iy) or nx - 1 sites at x = (ix + 0.5) a (odd
 *               iy). A site takes the phase of its nearest pixel (column
 *               ix + (iy odd), row round(iy sqrt(3)/2)). Grips are the first
 *               and last site of each row; Omega = (nx - 1) a R h; the grip
 *               area is R h. Runs on the spring-list kernels. */
typedef struct lsm_desc {
    int32_t dim, nx, ny, nz;
    const uint8_t *phase;
    int32_t nphase;
    const double *k_tab;
    const double *epsc_tab;
    const double *mass_tab;
    double k2_ratio;
    double a;
    double dt;
    double damping;
    int32_t grip_mode;
    int32_t load_mode;
    int32_t precision;
    int32_t path;
    void *stream;
    int32_t lattice;
} lsm_desc;

/* General network descriptor (the paper's solver reads any particle/bond
 * list, Section 3.1). Springs must be in canonical order (si < sj, sorted,
 * unique). All arrays are host memory, copied during the build.
 *  X        dim*n reference (and initial) positions, component-major.
 *  mass     n masses (NULL = all 1).
 *  fix      dim*n bytes, 1 = prescribed component (NULL = none).
 *  grip     n bytes: 0 interior, 1 left grip, 2 right grip (NULL = none).
 *  si, sj, k, r0, rc2   m springs; rc2 is the squared break length
 *           (INFINITY = unbreakable).
 *  xc       load centre for the affine remap and the grip law.
 *  omega    reference volume of the virial stress, Eq. 7.
 *  grip_area  area normalising the grip reaction. */
typedef struct lsm_net_desc {
    int32_t dim;
    int64_t n, m;
    const double *X;
    const double *mass;
    const uint8_t *fix;
    const uint8_t *grip;
    const int32_t *si, *sj;
    const double *k, *r0, *rc2;
    double dt, damping, xc, omega, grip_area;
    int32_t load_mode;
    int32_t precision;
    void *stream;
} lsm_net_desc;

/* One stress-strain sample, recorded at the end of every lsm_step / lsm_relax
 * call (the paper's output callback, Section 2.3 and Fig. 1).
 *  eps         engineering strain of the last lsm_apply_strain.
 *  sigma_vir   xx virial stress, Eq. 7, over the reference box, tension > 0.
 *  sigma_grip  xx stress from the right-grip reaction over the grip area.
 *  pe, ke      potential (Eq. 1, intact springs) and kinetic energy.
 *  residual    max over free components of max(|F|, |v|).
 *  n_broken    broken springs so far.
 *  step        time steps taken so far. */
typedef struct lsm_sample {
    double eps, sigma_vir, sigma_grip, pe, ke, residual;
    int64_t n_broken, step;
} lsm_sample;

/* Build a context from an image. On success *out owns device memory until
 * lsm_destroy. Errors: LSM_EINVAL (bad descriptor), LSM_ENOMEM, LSM_ECUDA. */
lsm_status lsm_build_from_image(const lsm_desc *desc, lsm_ctx **out);

/* Build a context from an explicit spring network (see lsm_net_desc). */
lsm_status lsm_build_network(const lsm_net_desc *desc, lsm_ctx **out);

/* Release all device memory of the context. NULL is ignored. */
void lsm_destroy(lsm_ctx *ctx);

/* One-line description of the last error on ctx (never NULL). With ctx ==
 * NULL, the last build error of the calling thread. */
const char *lsm_last_error(const lsm_ctx *ctx);

/* Sizes: particles n, springs m, dimension. Any output may be NULL. */
lsm_status lsm_sizes(lsm_ctx *ctx, int64_t *n, int64_t *m, int32_t *dim);

/* Displacement-controlled load increment (Sections 2.3, 3.1): set the
 * engineering strain to eps (absolute, not a delta). In load_mode 0 the x
 * coordinate of every particle is remapped x <- xc + (x - xc)(1+eps)/(1+eps_old);
 * prescribed x components are then set to X + eps (X - xc) with zero
 * velocity and acceleration. Stream-ordered. Errors: LSM_EINVAL if
 * 1 + eps <= 0. */
lsm_status lsm_apply_strain(lsm_ctx *ctx, double eps);

/* Advance nsteps (>= 1) time steps of damped velocity Verlet with the break
 * test (Eqs. 2-5), then record one lsm_sample. Stream-ordered (the step loop
 * is a cached CUDA graph per nsteps). */
lsm_status lsm_step(lsm_ctx *ctx, int64_t nsteps);

/* Relax to a force residual (the quasi-static limit of the damped dynamics,
 * Section 2.2): run steps in batches of check_every until the residual
 * (max over free components of max(|F|, |v|)) of a batch's last step is
 * <= tol, or max_steps steps are taken; then record one sample, of the final
 * state. *taken (may be NULL) = steps run. Synchronises after every batch.
 * Returns LSM_OK, LSM_ENOTCONV after max_steps (state and sample are those
 * reached), LSM_EINVAL for tol < 0, max_steps < 0 or check_every outside
 * 1..100000, or a pending device status. */
lsm_status lsm_relax(lsm_ctx *ctx, double tol, int64_t max_steps, int64_t check_every,
                     int64_t *taken);

/* The stress-strain curve: copy up to cap recorded samples' (eps,
 * sigma_vir) pairs (applied engineering strain; xx virial stress, Eq. 7,
 * over the reference box, tension > 0) into the caller's arrays (either may
 * be NULL when cap is 0); *count = number recorded (may exceed cap).
 * Synchronises. */
lsm_status lsm_stress_strain(lsm_ctx *ctx, double *eps, double *sigma, int64_t cap,
                             int64_t *count);

/* Copy up to cap full samples (lsm_sample) into out; *count = number
 * recorded (may exceed cap). Synchronises. */
lsm_status lsm_samples(lsm_ctx *ctx, lsm_sample *out, int64_t cap, int64_t *count);

/* Copy only the most recent sample into *out (64 bytes, whatever the number
 * recorded): the per-increment read of a load curve (Section 3.1 records the
 * stress at each output step). Errors: LSM_EINVAL for a null argument or
 * when no sample has been recorded yet. Synchronises. */
lsm_status lsm_sample_last(lsm_ctx *ctx, lsm_sample *out);

/* Broken-spring mask (Section 2.3 break test; Section 4: broken springs
 * are kept and give no force) in canonical spring order: out[s] = 1 if broken.
 * cap >= m is required (LSM_EINVAL otherwise); *m = spring count;
 * *first_break_step = index of the first step in which any spring broke,
 * -1 if none. Any output pointer may be NULL except out. Synchronises. */
lsm_status lsm_broken_mask(lsm_ctx *ctx, uint8_t *out, int64_t cap, int64_t *m,
                           int64_t *first_break_step);

/* Pipelined readback of a loading loop's results (no counterpart in the
 * paper, whose program reads its outputs between steps): enqueues, behind
 * the work already on the context's stream, a snapshot of the canonical
 * broken-spring mask (as lsm_broken_mask) and a copy of it into out_mask
 * (cap >= m bytes) and of the most recent sample (as lsm_sample_last) into
 * *out_sample, and returns without synchronising. The copies run on a
 * second stream of the context and overlap the steps enqueued after this
 * call; the host buffers hold the results once lsm_readback_wait returns
 * (page-locked buffers for the overlap; pageable ones make the copy
 * synchronous). Two snapshots alternate: the third call's snapshot waits,
 * on the device, for the first call's copy. out_mask or out_sample may be
 * NULL (not both); the buffers must stay valid and unread until
 * lsm_readback_wait. Errors: LSM_EINVAL (null or short buffers, no sample
 * yet), LSM_ECUDA; a pending device status is reported by lsm_readback_wait. */
lsm_status lsm_readback_async(lsm_ctx *ctx, uint8_t *out_mask, int64_t cap, lsm_sample *out_sample);

/* Wait for every readback enqueued by lsm_readback_async, then report a
 * pending device status (LSM_ENONFINITE) like the synchronising calls. */
lsm_status lsm_readback_wait(lsm_ctx *ctx);

/* Per-spring step index of the break (-1 = intact), canonical order, m
 * entries. Synchronises. */
lsm_status lsm_break_steps(lsm_ctx *ctx, int64_t *out, int64_t cap);

/* Positions and velocities (dim*n doubles each, component-major; either may
 * be NULL). Velocities are full-step velocities v(t). Synchronises. */
lsm_status lsm_get_state(lsm_ctx *ctx, double *x, double *v);

/* Replace positions and/or velocities (NULL keeps the current array); the
 * acceleration is re-evaluated from the new state, Eq. 4. Synchronises. */
lsm_status lsm_set_state(lsm_ctx *ctx, const double *x, const double *v);

/* Spring topology in canonical order (m entries each; any may be NULL). */
lsm_status lsm_topology(lsm_ctx *ctx, int32_t *si, int32_t *sj, double *k, double *r0,
                        double *rc2);

/* Observables of the current state without advancing (same fields as a
 * recorded sample; the sample history is unchanged). Synchronises. */
lsm_status lsm_observe(lsm_ctx *ctx, lsm_sample *out);

/* Constant strain-rate loading (Section 3.1: the boundary particles are
 * displaced apart at a fixed engineering strain rate, every time step).
 * From the next lsm_step on, the time step that completes step count s
 * first prescribes the grip components to X + eps (X - xc) with zero
 * velocity, eps = eps_set + (s - s_set) (rate dt) (eps_set, s_set: the
 * applied strain and the step count when the rate was set, or at the last
 * lsm_apply_strain), then advances as usual; only the grips move. rate = 0
 * stops the ramp (the strain stays where it is). Samples report the applied
 * strain. Not available on batched contexts. Errors: LSM_EINVAL for a null
 * context or a non-finite rate. */
lsm_status lsm_set_strain_rate(lsm_ctx *ctx, double rate);

/* Per-particle fields of the current state (Section 3.2, Eqs. 7-8), for
 * post-processing such as the paper's stress and strain maps.
 *   stress  host, [ncomp][n] (ncomp = 3 in 2D: xx, yy, xy; 6 in 3D: xx, yy,
 *           zz, xy, xz, yz), particle order as lsm_get_state: the virial
 *           stress of Eq. 7 with the domain taken as one particle's cell,
 *           (1/cell) [1/2 sum over the particle's intact springs of
 *           (x_l - x_k)_a f_b - m v_a v_b], f the spring's force on the
 *           particle; tension positive.
 *   strain  host, [ncomp][n]: the Lagrangian strain (J^T J - I)/2 of Eq. 8,
 *           J the least-squares affine map of the particle's first-neighbour
 *           vectors (its springs with the smallest rest length, broken or
 *           not) from the reference lattice to the current positions; NaN
 *           where those vectors do not span the space.
 *   cell_volume  the per-particle volume; <= 0 selects a^dim for image
 *           builds and 1 for network builds.
 * Either output may be NULL. Computed on the GPU in FP64 (correctly rounded
 * operations); the first call allocates the spring lists a 2D tile-path
 * context does not otherwise keep. Synchronises. Errors: LSM_EINVAL (null
 * context), LSM_ENOMEM, LSM_ECUDA, or a pending device status. */
lsm_status lsm_fields(lsm_ctx *ctx, double cell_volume, double *stress, double *strain);

/* Block until all work queued on the context's stream is done; returns any
 * pending device status. */
lsm_status lsm_synchronize(lsm_ctx *ctx);

/* Checkpoint and resume (a lifecycle call of this library; the paper's
 * solver only writes dump files, Section 3.1). lsm_save synchronises ctx and
 * writes to `path` (overwritten) the built network and the complete dynamic
 * state: positions and velocities as the time-step kernels hold them, broken
 * flags and break steps, step count, applied strain, strain-rate settings and
 * every recorded sample, with a checksum. lsm_load rebuilds a context from
 * such a file on `stream` (a cudaStream_t; NULL = a library-owned stream)
 * and restores that state, so that every later call gives results identical
 * bit for bit to those of the saved context. Errors: LSM_EINVAL for a null
 * argument, an unreadable, truncated, corrupt or foreign file (checked before
 * any device work) or a write failure; LSM_ENONFINITE / LSM_ECUDA as
 * lsm_synchronize; LSM_ENOMEM. The file is tied to this library version and
 * byte order. */
lsm_status lsm_save(lsm_ctx *ctx, const char *path);
lsm_status lsm_load(const char *path, void *stream, lsm_ctx **out);

/* Counters for throughput accounting: time steps taken, spring updates
 * (springs x steps) and CUDA kernels launched by the library (graph nodes
 * included). Any output may be NULL. */
lsm_status lsm_counters(lsm_ctx *ctx, int64_t *steps, int64_t *spring_updates,
                        int64_t *kernel_launches);

/* Potential energy and virial sum of the intact springs of a network at
 * given positions, with no device memory allocated by the library.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- code that runs inside a memory pool or
 * budget owned by another framework, and code that must not trigger the
 * implicit device-wide synchronisation of cudaFree. It never calls
 * cudaMalloc, cudaFree or an allocating library routine.
 *
 * Arguments (all arrays are DEVICE pointers owned by the caller):
 *   dim      2 or 3; n particles, m springs (0 <= m <= 268435456).
 *   x        dim*n positions, component-major ([c * n + p]).
 *   si, sj   m spring endpoints; k, r0 m spring constants and rest lengths.
 *   broken   m bytes, nonzero = broken (skipped); NULL = all intact.
 *   out      2 doubles written: out[0] = sum 1/2 k (r - r0)^2,
 *            out[1] = sum (x_j - x_i)_x f_x with f = k (r - r0)/r (x_j - x_i)
 *            (so sigma_xx = (out[1] - sum m v_x^2) / Omega).
 *   stream   cudaStream_t (NULL = default stream). The call is stream
 *            ordered and returns before the result is ready.
 * Scratch: per-chunk partial sums live in a file-scope device array of
 * 65536 x 2 doubles (1 MiB) that every device loading the library keeps until
 * exit. The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current, so make the first call on
 * each device before any stream capture. Every call shares the array and
 * fully rewrites the part it reads; calls that overlap on the GPU race on it.
 * The looked-up address is kept for the life of the process: after a reset of
 * a device (cudaDeviceReset, or a reset of its primary context) this entry
 * point must not be called on that device again in the same process.
 * Errors: LSM_EINVAL for bad sizes or null arrays (message in
 * lsm_last_error(NULL)), LSM_ECUDA if a launch fails. */
lsm_status lsm_spring_energy_static(int32_t dim, int64_t n, int64_t m, const double *x,
                                   const int32_t *si, const int32_t *sj, const double *k,
                                   const double *r0, const uint8_t *broken, double *out,
                                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LSM_H */
