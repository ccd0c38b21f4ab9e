// checkpoint.cpp -- lsm_save / lsm_load: a context's built network and its
// complete dynamic state in one file, so that a run resumes bit for bit.
//
// File layout (little-endian, native IEEE doubles; both build hosts are
// little-endian, and the endian word rejects anything else):
//   "LSMCKPT" '\0', u32 version, u32 0x01020304
//   the HostNet: scalars in a fixed order, then each vector as u64 count +
//   raw elements (X, mass, fixm, grip, si, sj, stype, types, pix, phase,
//   sdir, offv)
//   u32 path (the build's path request: 0 kernels chosen by the build rule,
//            1 spring-list kernels, 2 2D tile kernel, 3 2D strip kernel),
//   u32 tile (the context ran on a tile path)
//   host mirrors: eps, steps, nsamples, launches, the strain-rate settings
//   device scalars: step, first break, broken count, status, eps, sample count
//   samples [nsamples]
//   the path's state buffers, each as u64 bytes + raw bytes, in the order of
//   state_buffers() below
//   u64 FNV-1a hash of every byte before it.
// The integrator state is stored as the kernels hold it (tile paths: x and
// the half-step velocity vh of the current ping-pong buffer, plus the
// full-step velocity of the last sample; spring-list path: x, v and a), so no
// quantity is recomputed on load.
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "lsm_internal.h"

namespace lsm {

namespace {

constexpr char kMagic[8] = {'L', 'S', 'M', 'C', 'K', 'P', 'T', '\0'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kEndian = 0x01020304u;

struct Hash {
    uint64_t h = 1469598103934665603ull;  // FNV-1a 64-bit offset basis
    void add(const void *p, size_t n)
    {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < n; i++) {
            h ^= b[i];
            h *= 1099511628211ull;  // FNV prime
        }
    }
};

struct Writer {
    std::FILE *f = nullptr;
    Hash hash;
    bool ok = true;
    void put(const void *p, size_t n)
    {
        if (!ok || n == 0) return;
        hash.add(p, n);
        ok = std::fwrite(p, 1, n, f) == n;
    }
    template <typename T>
    void val(const T &v) { put(&v, sizeof(T)); }
    template <typename T>
    void vec(const std::vector<T> &v)
    {
        val<uint64_t>(v.size());
        put(v.data(), v.size() * sizeof(T));
    }
};

struct Reader {
    std::FILE *f = nullptr;
    Hash hash;
    bool ok = true;
    uint64_t limit = 0;  // bytes left in the file
    void get(void *p, size_t n)
    {
        if (!ok || n == 0) return;
        if (n > limit) {
            ok = false;
            return;
        }
        ok = std::fread(p, 1, n, f) == n;
        if (ok) {
            hash.add(p, n);
            limit -= n;
        }
    }
    template <typename T>
    void val(T &v) { get(&v, sizeof(T)); }
    template <typename T>
    void vec(std::vector<T> &v)
    {
        uint64_t cnt = 0;
        val(cnt);
        if (!ok || cnt > limit / sizeof(T)) {  // a count the file cannot hold
            ok = false;
            return;
        }
        v.resize(cnt);
        get(v.data(), cnt * sizeof(T));
    }
};

template <typename IO, typename H>
void net_fields(IO &io, H &h)
{
    io.val(h.dim);
    io.val(h.n);
    io.val(h.m);
    io.val(h.dt);
    io.val(h.damping);
    io.val(h.xc);
    io.val(h.omega);
    io.val(h.grip_area);
    io.val(h.load_mode);
    io.val(h.precision);
    io.val(h.grip_mode);
    io.val(h.a);
    io.val(h.lattice);
    io.val(h.cell);
    io.val(h.nx);
    io.val(h.ny);
    io.val(h.nz);
    io.val(h.nphase);
    io.vec(h.X);
    io.vec(h.mass);
    io.vec(h.fixm);
    io.vec(h.grip);
    io.vec(h.si);
    io.vec(h.sj);
    io.vec(h.stype);
    io.vec(h.types);
    io.vec(h.pix);
    io.vec(h.phase);
    io.vec(h.sdir);
    io.vec(h.offv);
}

// Device buffers that hold the dynamic state of c's path (current buffers).
std::vector<std::pair<void *, size_t>> state_buffers(Ctx &c)
{
    std::vector<std::pair<void *, size_t>> b;
    if (c.tile) {
        const size_t g = (size_t)c.dim * c.tnp * sizeof(double);
        b.push_back({c.tx[c.tcur], g});
        b.push_back({c.tvh[c.tcur], g});
        b.push_back({c.tvobs, g});
        if (c.dim == 3) {
            b.push_back({c.tmask3, (size_t)c.tnp * sizeof(uint16_t)});
            b.push_back({c.tbrk, (size_t)9 * c.tnp * sizeof(long long)});
        } else {
            b.push_back({c.tmask, (size_t)c.tnp});
            b.push_back({c.tbrk, (size_t)4 * c.tnp * sizeof(long long)});
        }
    } else {
        const size_t g = (size_t)c.dim * c.n * sizeof(double);
        b.push_back({c.x, g});
        b.push_back({c.v, g});
        b.push_back({c.a, g});
        b.push_back({c.state, (size_t)c.m});
        b.push_back({c.brk, (size_t)c.m * sizeof(long long)});
    }
    return b;
}

}  // namespace

cudaError_t checkpoint_save(Ctx &c, const char *path, std::string &err)
{
    CkptState s;
    s.path = c.tile ? (uint32_t)c.path_req : 1;  // 0 automatic, 2 tile kernel, 3 strip kernel
    s.tile = c.tile ? 1 : 0;
    s.eps = c.eps;
    s.steps = c.steps;
    s.nsamples = c.nsamples;
    s.launches = c.launches;
    s.rate_on = c.rate_on ? 1 : 0;
    s.rate_eps0 = c.rate_eps0;
    s.rate_dt = c.rate_dt;
    s.rate_step0 = c.rate_step0;
    cudaStream_t st = c.stream;
    cudaError_t e = cudaMemcpyAsync(&s.d_step, c.d_step, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s.first_break, c.d_first_break, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s.nbroken, c.d_nbroken, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s.status, c.d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s.d_eps, c.d_eps, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s.d_nsamples, c.d_nsamples, sizeof(long long), cudaMemcpyDeviceToHost, st);
    s.samples.resize((size_t)c.nsamples);
    if (e == cudaSuccess && c.nsamples > 0)
        e = cudaMemcpyAsync(s.samples.data(), c.samples, (size_t)c.nsamples * sizeof(DeviceSample),
                            cudaMemcpyDeviceToHost, st);
    const auto bufs = state_buffers(c);
    s.bufs.resize(bufs.size());
    for (size_t q = 0; q < bufs.size() && e == cudaSuccess; q++) {
        s.bufs[q].resize(bufs[q].second);
        e = cudaMemcpyAsync(s.bufs[q].data(), bufs[q].first, bufs[q].second, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;

    std::FILE *f = std::fopen(path, "wb");
    if (!f) {
        err = std::string("cannot open ") + path + " for writing";
        return cudaSuccess;
    }
    Writer w;
    w.f = f;
    w.put(kMagic, sizeof(kMagic));
    w.val(kVersion);
    w.val(kEndian);
    net_fields(w, c.h);
    w.val(s.path);
    w.val(s.tile);
    w.val(s.eps);
    w.val(s.steps);
    w.val(s.nsamples);
    w.val(s.launches);
    w.val(s.rate_on);
    w.val(s.rate_eps0);
    w.val(s.rate_dt);
    w.val(s.rate_step0);
    w.val(s.d_step);
    w.val(s.first_break);
    w.val(s.nbroken);
    w.val(s.status);
    w.val(s.d_eps);
    w.val(s.d_nsamples);
    w.vec(s.samples);
    w.val<uint64_t>(s.bufs.size());
    for (const auto &b : s.bufs) w.vec(b);
    const uint64_t hsum = w.hash.h;
    if (w.ok) w.ok = std::fwrite(&hsum, 1, sizeof(hsum), f) == sizeof(hsum);
    if (std::fclose(f) != 0) w.ok = false;
    if (!w.ok) err = std::string("write to ") + path + " failed";
    return cudaSuccess;
}

bool checkpoint_read(const char *path, HostNet &h, CkptState &s, std::string &err)
{
    std::FILE *f = std::fopen(path, "rb");
    if (!f) {
        err = std::string("cannot open ") + path;
        return false;
    }
    Reader r;
    r.f = f;
    if (std::fseek(f, 0, SEEK_END) == 0) {
        const long sz = std::ftell(f);
        r.limit = sz > 0 ? (uint64_t)sz : 0;
    }
    std::fseek(f, 0, SEEK_SET);
    if (r.limit < sizeof(kMagic) + 8 + 8) {
        std::fclose(f);
        err = std::string(path) + " is not a checkpoint (too short)";
        return false;
    }
    r.limit -= sizeof(uint64_t);  // the trailing hash
    char magic[8];
    uint32_t version = 0, endian = 0;
    r.get(magic, sizeof(magic));
    r.val(version);
    r.val(endian);
    if (!r.ok || std::memcmp(magic, kMagic, sizeof(kMagic)) != 0) {
        std::fclose(f);
        err = std::string(path) + " is not a checkpoint";
        return false;
    }
    if (version != kVersion || endian != kEndian) {
        std::fclose(f);
        err = std::string(path) + ": unsupported checkpoint version or byte order";
        return false;
    }
    net_fields(r, h);
    r.val(s.path);
    r.val(s.tile);
    r.val(s.eps);
    r.val(s.steps);
    r.val(s.nsamples);
    r.val(s.launches);
    r.val(s.rate_on);
    r.val(s.rate_eps0);
    r.val(s.rate_dt);
    r.val(s.rate_step0);
    r.val(s.d_step);
    r.val(s.first_break);
    r.val(s.nbroken);
    r.val(s.status);
    r.val(s.d_eps);
    r.val(s.d_nsamples);
    r.vec(s.samples);
    uint64_t nb = 0;
    r.val(nb);
    if (r.ok && nb > 16) r.ok = false;
    if (r.ok) {
        s.bufs.resize(nb);
        for (auto &b : s.bufs) r.vec(b);
    }
    uint64_t hsum = 0;
    const bool tail = r.ok && std::fread(&hsum, 1, sizeof(hsum), f) == sizeof(hsum);
    std::fclose(f);
    if (!r.ok || !tail || r.limit != 0) {
        err = std::string(path) + ": truncated or malformed checkpoint";
        return false;
    }
    if (hsum != r.hash.h) {
        err = std::string(path) + ": checksum mismatch (corrupt checkpoint)";
        return false;
    }
    // the network must be self-consistent before it reaches the device
    const size_t n = (size_t)h.n, m = (size_t)h.m;
    bool fine = h.dim >= 2 && h.dim <= 3 && h.n >= 0 && h.m >= 0 && h.X.size() == (size_t)h.dim * n &&
                h.mass.size() == n && h.fixm.size() == n && h.grip.size() == n && h.si.size() == m &&
                h.sj.size() == m && h.stype.size() == m && (int64_t)s.samples.size() == s.nsamples &&
                h.precision >= LSM_PREC_EXACT64 && h.precision <= LSM_PREC_DF && s.path <= 3;
    for (size_t q = 0; fine && q < m; q++)
        fine = h.si[q] >= 0 && h.sj[q] >= 0 && (size_t)h.si[q] < n && (size_t)h.sj[q] < n &&
               h.stype[q] < h.types.size();
    if (fine && h.nx > 0)
        fine = h.pix.size() == n && h.phase.size() == (size_t)h.nx * h.ny * (h.nz > 0 ? h.nz : 1);
    if (!fine) {
        err = std::string(path) + ": inconsistent network in checkpoint";
        return false;
    }
    return true;
}

cudaError_t checkpoint_restore(Ctx &c, const CkptState &s, std::string &err)
{
    c.tcur = 0;
    const auto bufs = state_buffers(c);
    if (bufs.size() != s.bufs.size()) {
        err = "checkpoint state does not match the rebuilt context";
        return cudaSuccess;
    }
    for (size_t q = 0; q < bufs.size(); q++)
        if (bufs[q].second != s.bufs[q].size()) {
            err = "checkpoint state does not match the rebuilt context";
            return cudaSuccess;
        }
    cudaStream_t st = c.stream;
    cudaError_t e = cudaSuccess;
    if (s.nsamples > c.sample_cap) {
        int64_t cap = c.sample_cap > 0 ? c.sample_cap : 1024;
        while (cap < s.nsamples) cap *= 2;
        DeviceSample *ns = nullptr;
        e = lsm::dev_malloc((void **)&ns, (size_t)cap * sizeof(DeviceSample));
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(st);
        cudaFree(c.samples);
        c.samples = ns;
        c.sample_cap = cap;
        if (e != cudaSuccess) return e;
    }
    for (size_t q = 0; q < bufs.size() && e == cudaSuccess; q++)
        e = cudaMemcpyAsync(bufs[q].first, s.bufs[q].data(), bufs[q].second, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && s.nsamples > 0)
        e = cudaMemcpyAsync(c.samples, s.samples.data(), (size_t)s.nsamples * sizeof(DeviceSample),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_step, &s.d_step, sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.d_first_break, &s.first_break, sizeof(unsigned long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.d_nbroken, &s.nbroken, sizeof(unsigned long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_status, &s.status, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_eps, &s.d_eps, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.d_nsamples, &s.d_nsamples, sizeof(long long), cudaMemcpyHostToDevice, st);
    c.eps = s.eps;
    c.steps = s.steps;
    c.nsamples = s.nsamples;
    c.launches = s.launches;
    c.rate_on = s.rate_on != 0;
    c.rate_eps0 = s.rate_eps0;
    c.rate_dt = s.rate_dt;
    c.rate_step0 = s.rate_step0;
    if (e == cudaSuccess && c.fixcsr) e = fixcsr_refresh(c);  // fixed-point copy of the restored x
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace lsm
