// api.cpp -- the extern "C" boundary of liblsm (declared in include/lsm.h).
//
// Argument checks, context lifetime, stream handling and host<->device
// copies. Every compute step runs in the kernels of kernels.cu.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "lsm_internal.h"

using lsm::Ctx;

struct lsm_ctx : public Ctx {};

namespace {

thread_local std::string g_build_err;

lsm_status fail(Ctx *c, lsm_status st, const std::string &msg)
{
    if (c)
        c->err = msg;
    else
        g_build_err = msg;
    return st;
}

lsm_status cuda_fail(Ctx *c, cudaError_t e, const char *where)
{
    return fail(c, LSM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Pending asynchronous device status (non-finite state).
lsm_status device_status(Ctx *c)
{
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
    if (st & 1) return fail(c, LSM_ENONFINITE, "non-finite position or velocity detected");
    if (st & 2) return fail(c, LSM_ENONFINITE, "position outside the fixed-point range of the F32/DF modes");
    return LSM_OK;
}

lsm_status finish_build(lsm_ctx *c, void *stream, lsm_ctx **out, int path = 0)
{
    // 2D square-lattice images: the fused tile kernel in every mode; 3D images:
    // the voxel tile kernel in the fixed-point modes (the FP64 modes stay on
    // the spring-list kernels, see tile3d.cu)
    const bool fixmode = c->h.precision == LSM_PREC_F32 || c->h.precision == LSM_PREC_DF;
    // the triangular packing (2D, fixed-point modes, path 0) runs on the
    // strip kernel alone, its state on the grid of its sites
    c->tri = (path == 0 || path == 3) && c->h.nx > 0 && c->h.lattice == 1 && c->h.dim == 2 && fixmode && c->h.nphase >= 1 &&
             c->h.nphase <= 8;
    c->tile = c->tri || (path != 1 && c->h.nx > 0 && c->h.lattice == 0 && c->h.nphase >= 1 && c->h.nphase <= 8 &&
                         (c->h.dim == 2 || (c->h.dim == 3 && fixmode)));
    // 2D fixed-point modes: time steps on the strip kernel when its strips
    // fill the device (path 2: the square lattice's tile kernel always; path
    // 3: the strip kernel always; same states either way)
    c->strip = c->tile && (c->tri || path != 2) && lsm::strip_supported(*c);
    c->strip_forced = path == 3;
    c->path_req = path;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_build_err = std::string("stream create: ") + cudaGetErrorString(e);
            delete c;
            return LSM_ECUDA;
        }
        c->own_stream = true;
    }
    cudaGetLastError();  // clear an error left by an unrelated earlier call
    cudaError_t e = lsm::upload(*c);
    const char *site = "upload";
    if (e != cudaSuccess) site = lsm::last_fail_site();
    if (e == cudaSuccess) {
        e = lsm::launch_init_accel(*c);
        site = "initial acceleration";
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        g_build_err = std::string("build (") + site + "): " + cudaGetErrorString(e);
        lsm_status st = e == cudaErrorMemoryAllocation ? LSM_ENOMEM : LSM_ECUDA;
        lsm::free_device(*c);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return st;
    }
    *out = c;
    return LSM_OK;
}

lsm_status ensure_sample_room(Ctx *c)
{
    if (c->nsamples < c->sample_cap) return LSM_OK;
    int64_t cap = c->sample_cap * 2;
    lsm::DeviceSample *ns = nullptr;
    cudaError_t e = lsm::dev_malloc((void **)&ns, cap * sizeof(lsm::DeviceSample));
    if (e != cudaSuccess) return fail(c, LSM_ENOMEM, "sample buffer growth failed");
    e = cudaMemcpyAsync(ns, c->samples, c->sample_cap * sizeof(lsm::DeviceSample),
                        cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    // a readback in flight may still copy a sample out of the old buffer
    if (e == cudaSuccess && c->rb_stream) e = cudaStreamSynchronize(c->rb_stream);
    if (e != cudaSuccess) {
        cudaFree(ns);
        return cuda_fail(c, e, "sample buffer growth");
    }
    cudaFree(c->samples);
    c->samples = ns;
    c->sample_cap = cap;
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);  // graphs hold the old pointer
    c->graphs.clear();
    return LSM_OK;
}

}  // namespace

void lsm::set_thread_error(const char *msg) { g_build_err = msg; }

extern "C" {

lsm_status lsm_build_from_image(const lsm_desc *desc, lsm_ctx **out)
{
    lsm::NvtxRange nvtx_("lsm_build_from_image");
    if (!desc || !out) return fail(nullptr, LSM_EINVAL, "desc and out are required");
    *out = nullptr;
    if (desc->precision < LSM_PREC_EXACT64 || desc->precision > LSM_PREC_DF)
        return fail(nullptr, LSM_EINVAL, "precision must be LSM_PREC_EXACT64, _FAST64, _F32 or _DF");
    lsm_ctx *c = new (std::nothrow) lsm_ctx();
    if (!c) return fail(nullptr, LSM_ENOMEM, "host allocation failed");
    std::string err;
    bool ok;
    try {
        ok = lsm::net_from_image(*desc, c->h, err);
    } catch (const std::bad_alloc &) {
        delete c;
        return fail(nullptr, LSM_ENOMEM, "host allocation failed during build");
    }
    if (!ok) {
        delete c;
        return fail(nullptr, LSM_EINVAL, err);
    }
    if (desc->path < 0 || desc->path > 3) {
        delete c;
        return fail(nullptr, LSM_EINVAL, "path must be 0 (automatic), 1 (spring-list kernels), 2 (2D tile kernel) or "
                                         "3 (2D strip kernel)");
    }
    return finish_build(c, desc->stream, out, desc->path);
}

lsm_status lsm_build_network(const lsm_net_desc *desc, lsm_ctx **out)
{
    lsm::NvtxRange nvtx_("lsm_build_network");
    if (!desc || !out) return fail(nullptr, LSM_EINVAL, "desc and out are required");
    *out = nullptr;
    if (desc->precision < LSM_PREC_EXACT64 || desc->precision > LSM_PREC_DF)
        return fail(nullptr, LSM_EINVAL, "precision must be LSM_PREC_EXACT64, _FAST64, _F32 or _DF");
    if (desc->load_mode != 0 && desc->load_mode != 1)
        return fail(nullptr, LSM_EINVAL, "load_mode must be 0 or 1");
    lsm_ctx *c = new (std::nothrow) lsm_ctx();
    if (!c) return fail(nullptr, LSM_ENOMEM, "host allocation failed");
    std::string err;
    bool ok;
    try {
        ok = lsm::net_from_desc(*desc, c->h, err);
    } catch (const std::bad_alloc &) {
        delete c;
        return fail(nullptr, LSM_ENOMEM, "host allocation failed during build");
    }
    if (!ok) {
        delete c;
        return fail(nullptr, LSM_EINVAL, err);
    }
    return finish_build(c, desc->stream, out, 1);
}

void lsm_destroy(lsm_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    lsm::free_device(*c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *lsm_last_error(const lsm_ctx *c)
{
    return c ? c->err.c_str() : g_build_err.c_str();
}

lsm_status lsm_sizes(lsm_ctx *c, int64_t *n, int64_t *m, int32_t *dim)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (n) *n = c->n;
    if (m) *m = c->m;
    if (dim) *dim = c->dim;
    return LSM_OK;
}

// Host mirror of the applied strain under a constant strain rate (the same
// operations as the device: eps0 + (s - s0) rdt).
static void rate_eps_sync(lsm_ctx *c)
{
    if (c->rate_on) c->eps = c->rate_eps0 + (double)(c->steps - c->rate_step0) * c->rate_dt;
}

// Graphs bake the kernel arguments; drop them when the loading changes.
static void drop_graphs(lsm_ctx *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

lsm_status lsm_apply_strain(lsm_ctx *c, double eps)
{
    lsm::NvtxRange nvtx_("lsm_apply_strain");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (!(1.0 + eps > 0.0) || !std::isfinite(eps))
        return fail(c, LSM_EINVAL, "strain must be finite with 1 + eps > 0");
    cudaError_t e = lsm::launch_apply_strain(*c, c->eps, eps);
    if (e != cudaSuccess) return cuda_fail(c, e, "apply_strain");
    c->eps = eps;
    if (c->rate_on) {  // the ramp continues from the new strain
        c->rate_eps0 = eps;
        c->rate_step0 = c->steps;
        drop_graphs(c);
    }
    return LSM_OK;
}

lsm_status lsm_set_strain_rate(lsm_ctx *c, double rate)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (!std::isfinite(rate)) return fail(c, LSM_EINVAL, "strain rate must be finite");
    c->rate_on = rate != 0.0;
    c->rate_eps0 = c->eps;
    c->rate_step0 = c->steps;
    c->rate_dt = rate * c->h.dt;
    drop_graphs(c);
    return LSM_OK;
}

lsm_status lsm_step(lsm_ctx *c, int64_t nsteps)
{
    lsm::NvtxRange nvtx_("lsm_step");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (nsteps < 1) return fail(c, LSM_EINVAL, "nsteps must be >= 1");
    if (nsteps > 100000) return fail(c, LSM_EINVAL, "nsteps per call is limited to 100000");
    lsm_status st = ensure_sample_room(c);
    if (st != LSM_OK) return st;
    cudaError_t e = lsm::launch_steps(*c, nsteps, true);
    if (e != cudaSuccess) return cuda_fail(c, e, "step");
    c->nsamples += 1;
    c->steps += nsteps;
    rate_eps_sync(c);
    return LSM_OK;
}

lsm_status lsm_relax(lsm_ctx *c, double tol, int64_t max_steps, int64_t check_every,
                     int64_t *taken)
{
    lsm::NvtxRange nvtx_("lsm_relax");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (!(tol >= 0) || max_steps < 0 || check_every < 1 || check_every > 100000)
        return fail(c, LSM_EINVAL, "need tol >= 0, max_steps >= 0, 1 <= check_every <= 100000");
    lsm_status st = ensure_sample_room(c);
    if (st != LSM_OK) return st;
    int64_t done = 0;
    lsm_status result = LSM_ENOTCONV;
    while (done < max_steps) {
        const int64_t nb = max_steps - done < check_every ? max_steps - done : check_every;
        cudaError_t e = lsm::launch_steps(*c, nb, false);
        if (e != cudaSuccess) return cuda_fail(c, e, "relax");
        done += nb;
        c->steps += nb;
        rate_eps_sync(c);
        lsm::DeviceSample smp;
        e = cudaMemcpyAsync(&smp, c->scratch_sample, sizeof(smp), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "relax readback");
        st = device_status(c);
        if (st != LSM_OK) {
            if (taken) *taken = done;
            return st;
        }
        if (smp.residual <= tol) {
            result = LSM_OK;
            break;
        }
    }
    if (done > 0) {  // record the final state's sample
        cudaError_t e = cudaMemcpyAsync(c->samples + c->nsamples, c->scratch_sample,
                                        sizeof(lsm::DeviceSample), cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "relax record");
        long long ns = c->nsamples + 1;
        e = cudaMemcpyAsync(c->d_nsamples, &ns, sizeof(ns), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "relax record");
        c->nsamples = ns;
    }
    if (taken) *taken = done;
    if (result != LSM_OK) return fail(c, LSM_ENOTCONV, "residual above tolerance after max_steps");
    return LSM_OK;
}

lsm_status lsm_samples(lsm_ctx *c, lsm_sample *out, int64_t cap, int64_t *count)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (cap < 0 || (cap > 0 && !out)) return fail(c, LSM_EINVAL, "bad output buffer");
    lsm_status st = device_status(c);
    if (st != LSM_OK) return st;
    const int64_t k = c->nsamples < cap ? c->nsamples : cap;
    if (k > 0) {
        static_assert(sizeof(lsm::DeviceSample) == sizeof(lsm_sample), "sample layout");
        cudaError_t e = cudaMemcpyAsync(out, c->samples, k * sizeof(lsm_sample),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "samples");
    }
    if (count) *count = c->nsamples;
    return LSM_OK;
}

lsm_status lsm_sample_last(lsm_ctx *c, lsm_sample *out)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (!out) return fail(c, LSM_EINVAL, "null output");
    lsm_status st = device_status(c);
    if (st != LSM_OK) return st;
    if (c->nsamples < 1) return fail(c, LSM_EINVAL, "no sample recorded yet");
    cudaError_t e = cudaMemcpyAsync(out, c->samples + (c->nsamples - 1), sizeof(lsm_sample),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sample");
    return LSM_OK;
}

lsm_status lsm_stress_strain(lsm_ctx *c, double *eps, double *sigma, int64_t cap, int64_t *count)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (cap < 0 || (cap > 0 && (!eps || !sigma))) return fail(c, LSM_EINVAL, "bad output buffers");
    std::vector<lsm_sample> tmp((size_t)(c->nsamples < cap ? c->nsamples : cap));
    int64_t cnt = 0;
    lsm_status st = lsm_samples(c, tmp.data(), (int64_t)tmp.size(), &cnt);
    if (st != LSM_OK) return st;
    for (size_t q = 0; q < tmp.size(); q++) {
        eps[q] = tmp[q].eps;
        sigma[q] = tmp[q].sigma_vir;
    }
    if (count) *count = cnt;
    return LSM_OK;
}

lsm_status lsm_broken_mask(lsm_ctx *c, uint8_t *out, int64_t cap, int64_t *m,
                           int64_t *first_break_step)
{
    lsm::NvtxRange nvtx_("lsm_broken_mask");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (!out || cap < c->m) return fail(c, LSM_EINVAL, "output buffer smaller than the spring count");
    lsm_status st = device_status(c);
    if (st != LSM_OK) return st;
    unsigned long long fb = 0;
    cudaError_t e = cudaSuccess;
    if (c->tile) {
        e = lsm::tile_export(*c, false);
        if (e == cudaSuccess && c->m)
            e = cudaMemcpyAsync(out, c->texport, c->m, cudaMemcpyDeviceToHost, c->stream);
    } else if (c->m) {
        e = cudaMemcpyAsync(out, c->state, c->m, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&fb, c->d_first_break, sizeof(fb), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "broken_mask");
    if (m) *m = c->m;
    if (first_break_step) *first_break_step = fb == ~0ull ? -1 : (int64_t)fb;
    return LSM_OK;
}

lsm_status lsm_readback_async(lsm_ctx *c, uint8_t *out_mask, int64_t cap, lsm_sample *out_sample)
{
    lsm::NvtxRange nvtx_("lsm_readback_async");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if ((!out_mask && !out_sample) || (out_mask && cap < c->m))
        return fail(c, LSM_EINVAL, "need a mask buffer of at least m bytes or a sample");
    if (out_sample && c->nsamples < 1) return fail(c, LSM_EINVAL, "no sample recorded yet");
    cudaError_t e = cudaSuccess;
    if (!c->rb_stream) {
        e = cudaStreamCreateWithFlags(&c->rb_stream, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; k++) {
            e = cudaEventCreateWithFlags(&c->rb_ready[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->rb_done[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "readback setup");
    }
    const int k = (int)(c->rb_count & 1);
    if (out_mask && c->m && !c->rb_buf[k]) {
        e = lsm::dev_malloc((void **)&c->rb_buf[k], c->m);
        if (e != cudaSuccess) return cuda_fail(c, e, "readback buffer");
    }
    // the snapshot of two readbacks ago must be copied out before it is
    // rewritten: the context's stream waits for it on the device
    if (c->rb_used[k]) e = cudaStreamWaitEvent(c->stream, c->rb_done[k], 0);
    if (e == cudaSuccess && out_mask && c->m) {
        if (c->tile) {
            // the export kernel writes the canonical mask straight into the
            // snapshot (its staging pointer is swapped for the call)
            uint8_t *staging = c->texport;
            c->texport = c->rb_buf[k];
            e = lsm::tile_export(*c, false);
            c->texport = staging;
        } else {
            e = cudaMemcpyAsync(c->rb_buf[k], c->state, c->m, cudaMemcpyDeviceToDevice, c->stream);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->rb_ready[k], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->rb_stream, c->rb_ready[k], 0);
    if (e == cudaSuccess && out_mask && c->m)
        e = cudaMemcpyAsync(out_mask, c->rb_buf[k], c->m, cudaMemcpyDeviceToHost, c->rb_stream);
    if (e == cudaSuccess && out_sample)
        e = cudaMemcpyAsync(out_sample, c->samples + (c->nsamples - 1), sizeof(lsm_sample), cudaMemcpyDeviceToHost,
                            c->rb_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->rb_done[k], c->rb_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "readback_async");
    c->rb_used[k] = true;
    c->rb_count++;
    return LSM_OK;
}

lsm_status lsm_readback_wait(lsm_ctx *c)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (c->rb_stream) {
        const cudaError_t e = cudaStreamSynchronize(c->rb_stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "readback_wait");
    }
    return device_status(c);
}

lsm_status lsm_break_steps(lsm_ctx *c, int64_t *out, int64_t cap)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (!out || cap < c->m) return fail(c, LSM_EINVAL, "output buffer smaller than the spring count");
    cudaError_t e = cudaSuccess;
    if (c->tile) {
        e = lsm::tile_export(*c, true);
        if (e == cudaSuccess && c->m)
            e = cudaMemcpyAsync(out, c->texport_brk, c->m * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    } else if (c->m) {
        e = cudaMemcpyAsync(out, c->brk, c->m * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "break_steps");
    return LSM_OK;
}

lsm_status lsm_get_state(lsm_ctx *c, double *x, double *v)
{
    lsm::NvtxRange nvtx_("lsm_get_state");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    lsm_status st = device_status(c);
    if (st != LSM_OK) return st;
    const size_t bytes = (size_t)c->dim * c->n * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (c->tile) {
        std::vector<double> gx(x ? (size_t)c->dim * c->tnp : 0), gv(v ? (size_t)c->dim * c->tnp : 0);
        if (x) e = cudaMemcpyAsync(gx.data(), c->tx[c->tcur], (size_t)c->dim * c->tnp * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && v)
            e = cudaMemcpyAsync(gv.data(), c->tvobs, (size_t)c->dim * c->tnp * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "get_state");
        for (int cc = 0; cc < c->dim; cc++)
            for (int64_t p = 0; p < c->n; p++) {
                const int64_t g = c->tgidx[p];
                if (x) x[cc * c->n + p] = gx[cc * c->tnp + g];
                if (v) v[cc * c->n + p] = gv[cc * c->tnp + g];
            }
        return LSM_OK;
    }
    if (x) e = cudaMemcpyAsync(x, c->x, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(v, c->v, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_state");
    return LSM_OK;
}

lsm_status lsm_set_state(lsm_ctx *c, const double *x, const double *v)
{
    lsm::NvtxRange nvtx_("lsm_set_state");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    const size_t bytes = (size_t)c->dim * c->n * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (c->tile) {
        // scatter onto the pixel grid (void pixels keep their placeholder)
        std::vector<double> gx, gv;
        if (x) gx.resize((size_t)c->dim * c->tnp);
        if (v) gv.resize((size_t)c->dim * c->tnp);
        if (x) e = cudaMemcpyAsync(gx.data(), c->tx[c->tcur], (size_t)c->dim * c->tnp * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && v)
            e = cudaMemcpyAsync(gv.data(), c->tvobs, (size_t)c->dim * c->tnp * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
        for (int cc = 0; cc < c->dim; cc++)
            for (int64_t p = 0; p < c->n; p++) {
                const int64_t g = c->tgidx[p];
                if (x) gx[cc * c->tnp + g] = x[cc * c->n + p];
                if (v) gv[cc * c->tnp + g] = v[cc * c->n + p];
            }
        if (x) e = cudaMemcpyAsync(c->tx[c->tcur], gx.data(), (size_t)c->dim * c->tnp * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && v)
            e = cudaMemcpyAsync(c->tvobs, gv.data(), (size_t)c->dim * c->tnp * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = lsm::launch_init_accel(*c);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
        return LSM_OK;
    }
    if (x) e = cudaMemcpyAsync(c->x, x, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(c->v, v, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = lsm::launch_init_accel(*c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
    return LSM_OK;
}

lsm_status lsm_topology(lsm_ctx *c, int32_t *si, int32_t *sj, double *k, double *r0, double *rc2)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    const lsm::HostNet &h = c->h;
    for (int64_t s = 0; s < h.m; s++) {
        const lsm::SpringType &t = h.types[h.stype[s]];
        if (si) si[s] = h.si[s];
        if (sj) sj[s] = h.sj[s];
        if (k) k[s] = t.k;
        if (r0) r0[s] = t.r0;
        if (rc2) rc2[s] = t.rc2;
    }
    return LSM_OK;
}

lsm_status lsm_observe(lsm_ctx *c, lsm_sample *out)
{
    lsm::NvtxRange nvtx_("lsm_observe");
    if (!c || !out) return fail(c, LSM_EINVAL, "null argument");
    cudaError_t e = lsm::launch_observe(*c, c->scratch_sample);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, c->scratch_sample, sizeof(lsm_sample), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "observe");
    return device_status(c);
}

lsm_status lsm_fields(lsm_ctx *c, double cell_volume, double *stress, double *strain)
{
    lsm::NvtxRange nvtx_("lsm_fields");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    lsm_status st = device_status(c);
    if (st != LSM_OK) return st;
    double cell = cell_volume;
    if (!(cell > 0.0)) cell = c->h.cell;
    cudaError_t e = lsm::fields_compute(*c, cell);
    const int nq = c->h.dim == 3 ? 6 : 3;
    const size_t bytes = (size_t)nq * c->n * sizeof(double);
    if (e == cudaSuccess && stress && c->n)
        e = cudaMemcpyAsync(stress, c->fout, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && strain && c->n)
        e = cudaMemcpyAsync(strain, c->fout + (size_t)nq * c->n, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaErrorMemoryAllocation) return fail(c, LSM_ENOMEM, "fields: device allocation failed");
    if (e != cudaSuccess) return cuda_fail(c, e, "fields");
    return LSM_OK;
}

lsm_status lsm_synchronize(lsm_ctx *c)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
    return device_status(c);
}

lsm_status lsm_save(lsm_ctx *c, const char *path)
{
    lsm::NvtxRange nvtx_("lsm_save");
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (!path) return fail(c, LSM_EINVAL, "null path");
    lsm_status st = device_status(c);
    if (st != LSM_OK) return st;
    std::string err;
    cudaError_t e;
    try {
        e = lsm::checkpoint_save(*c, path, err);
    } catch (const std::bad_alloc &) {
        return fail(c, LSM_ENOMEM, "host allocation failed during save");
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "save");
    if (!err.empty()) return fail(c, LSM_EINVAL, err);
    return LSM_OK;
}

lsm_status lsm_load(const char *path, void *stream, lsm_ctx **out)
{
    lsm::NvtxRange nvtx_("lsm_load");
    if (!path || !out) return fail(nullptr, LSM_EINVAL, "path and out are required");
    *out = nullptr;
    lsm_ctx *c = new (std::nothrow) lsm_ctx();
    if (!c) return fail(nullptr, LSM_ENOMEM, "host allocation failed");
    lsm::CkptState s;
    std::string err;
    bool ok;
    try {
        ok = lsm::checkpoint_read(path, c->h, s, err);
    } catch (const std::bad_alloc &) {
        delete c;
        return fail(nullptr, LSM_ENOMEM, "host allocation failed during load");
    }
    if (!ok) {
        delete c;
        return fail(nullptr, LSM_EINVAL, err);
    }
    lsm_ctx *built = nullptr;
    lsm_status st = finish_build(c, stream, &built, (int)s.path);  // frees c on failure
    if (st != LSM_OK) return st;
    if (built->tile != (s.tile != 0)) {
        lsm_destroy(built);
        return fail(nullptr, LSM_EINVAL, "checkpoint was written by a different kernel path");
    }
    cudaError_t e = lsm::checkpoint_restore(*built, s, err);
    if (e != cudaSuccess || !err.empty()) {
        const std::string msg = e != cudaSuccess ? std::string("load: ") + cudaGetErrorString(e) : err;
        lsm_destroy(built);
        return fail(nullptr, e != cudaSuccess ? LSM_ECUDA : LSM_EINVAL, msg);
    }
    *out = built;
    return LSM_OK;
}

lsm_status lsm_counters(lsm_ctx *c, int64_t *steps, int64_t *spring_updates,
                        int64_t *kernel_launches)
{
    if (!c) return fail(nullptr, LSM_EINVAL, "null context");
    if (steps) *steps = c->steps;
    if (spring_updates) *spring_updates = c->steps * c->m;
    if (kernel_launches) *kernel_launches = c->launches;
    return LSM_OK;
}

}  // extern "C"
