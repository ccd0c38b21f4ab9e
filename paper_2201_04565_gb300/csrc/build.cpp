// build.cpp -- host-side network construction for liblsm.
//
// Image -> particle-spring network on a square (2D) or cubic (3D) lattice:
// the paper's Img2Particle stage (Section 1, Fig. 6), with first neighbours
// (r0 = a) and second neighbours (r0 = a sqrt 2), spring constant and
// critical strain by the pair of endpoint phases (Table of spring constants,
// Section 3.1), particle mass by phase (Section 2.3, "assigned according to
// their specific types").
//
// Emission order is canonical by construction: particles are visited in
// raster order and, for each, the forward neighbour offsets are visited in
// ascending raster distance, so springs come out sorted by (i, j).
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <algorithm>

#include "lsm_internal.h"

namespace lsm {

namespace {

struct Offset {
    int dx, dy, dz, shell;
    int64_t lin;
};

std::vector<Offset> forward_offsets(int dim, int nx, int ny)
{
    std::vector<Offset> o;
    // every lattice vector with squared length 1 or 2 that points "forward"
    // in raster order (positive linear index offset)
    const int zr = dim == 3 ? 1 : 0;
    for (int dz = -zr; dz <= zr; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int l2 = dx * dx + dy * dy + dz * dz;
                if (l2 < 1 || l2 > 2) continue;
                int64_t lin = dx + (int64_t)nx * (dy + (int64_t)ny * dz);
                if (lin <= 0) continue;
                o.push_back({dx, dy, dz, l2, lin});
            }
    std::sort(o.begin(), o.end(), [](const Offset &a, const Offset &b) { return a.lin < b.lin; });
    return o;
}

}  // namespace

// Exact floor(sqrt(v)), v >= 0.
int64_t isqrt64(int64_t v)
{
    int64_t r = (int64_t)std::sqrt((double)v);
    while (r > 0 && r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return r;
}

// Triangular packing (lattice 1, 2D). Rows iy = 0..R-1 at y = iy h,
// h = (a sqrt 3) 0.5, R the number of rows with iy sqrt(3)/2 <= ny - 1
// pixels; row iy has nx sites (even iy) or nx - 1 (odd iy, shifted by a/2).
// Each site takes the phase of its nearest pixel (column ix + (iy odd), row
// round(iy sqrt(3)/2), in integers). Forward neighbours, in ascending site
// order: the next site of the row, then the two sites of row iy + 1 at
// x - a/2 and x + a/2; all first neighbours, r0 = a.
bool net_from_image_tri(const lsm_desc &d, HostNet &net, std::string &err)
{
    const int nx = d.nx, ny = d.ny, np = d.nphase;
    int64_t R = 0;
    while (3 * (R + 1) * (R + 1) <= 4 * (int64_t)(ny - 1) * (ny - 1)) R++;
    R += 1;
    std::vector<int64_t> rowbase(R + 1, 0);
    for (int64_t iy = 0; iy < R; iy++) rowbase[iy + 1] = rowbase[iy] + ((iy & 1) ? nx - 1 : nx);
    const int64_t nsite = rowbase[R];
    if (nsite > ((int64_t)1 << 31) - 1) { err = "lattice larger than 2^31 - 1 sites"; return false; }
    std::vector<int64_t> pid(nsite), pixel(nsite);
    int64_t n = 0;
    for (int64_t iy = 0; iy < R; iy++) {
        const int64_t prow = (isqrt64(3 * iy * iy) + 1) / 2;
        for (int64_t ix = 0; ix < rowbase[iy + 1] - rowbase[iy]; ix++) {
            const int64_t g = prow * nx + ix + (iy & 1);
            const uint8_t ph = d.phase[g];
            if (ph > np) { err = "phase value above nphase"; return false; }
            pixel[rowbase[iy] + ix] = g;
            pid[rowbase[iy] + ix] = ph ? n++ : -1;
        }
    }
    if (n == 0) { err = "image has no particles"; return false; }
    net.types.assign((size_t)np * np * 2, SpringType{});
    for (int pi = 0; pi < np; pi++)
        for (int pj = 0; pj < np; pj++) {
            const double k = d.k_tab[pi * np + pj], ec = d.epsc_tab[pi * np + pj];
            if (!(k >= 0) || !(ec > -1.0)) { err = "k_tab must be >= 0 and epsc_tab > -1"; return false; }
            const double rc = d.a * (1.0 + ec);
            SpringType &t = net.types[((size_t)pi * np + pj) * 2];
            t.k = k;
            t.r0 = d.a;
            t.rc2 = rc * rc;
            t.kr0 = k * d.a;
            net.types[((size_t)pi * np + pj) * 2 + 1] = t;  // no second shell; kept for the type layout
        }
    const double h = d.a * std::sqrt(3.0) * 0.5;
    net.offv = {d.a, 0.0, 0.0, -0.5 * d.a, h, 0.0, 0.5 * d.a, h, 0.0};
    net.dim = 2;
    net.n = n;
    net.X.assign((size_t)2 * n, 0.0);
    net.mass.assign(n, 1.0);
    net.fixm.assign(n, 0);
    net.grip.assign(n, 0);
    net.si.clear(); net.sj.clear(); net.stype.clear(); net.sdir.clear();
    net.pix.resize(n);
    for (int64_t iy = 0; iy < R; iy++) {
        const int64_t C = rowbase[iy + 1] - rowbase[iy];
        for (int64_t ix = 0; ix < C; ix++) {
            const int64_t p = pid[rowbase[iy] + ix];
            if (p < 0) continue;
            const int ph = d.phase[pixel[rowbase[iy] + ix]];
            net.pix[p] = pixel[rowbase[iy] + ix];
            net.X[p] = (ix + 0.5 * (double)(iy & 1)) * d.a;
            net.X[n + p] = iy * h;
            if (d.mass_tab) net.mass[p] = d.mass_tab[ph - 1];
            if (ix == 0 || ix == C - 1) {
                net.grip[p] = ix == 0 ? 1 : 2;
                net.fixm[p] = d.grip_mode == 1 ? 3 : 1;
            }
            // same row, then row iy + 1 at x - a/2 and x + a/2
            const int64_t up = ix + ((iy & 1) ? 0 : -1);
            const int64_t tx[3] = {ix + 1, up, up + 1}, ty[3] = {iy, iy + 1, iy + 1};
            for (int t = 0; t < 3; t++) {
                if (ty[t] >= R || tx[t] < 0 || tx[t] >= rowbase[ty[t] + 1] - rowbase[ty[t]]) continue;
                const int64_t site = rowbase[ty[t]] + tx[t];
                const int64_t q = pid[site];
                if (q < 0) continue;
                const int pq = d.phase[pixel[site]];
                net.sdir.push_back((uint8_t)t);
                net.si.push_back((int32_t)p);
                net.sj.push_back((int32_t)q);
                net.stype.push_back((uint16_t)(((ph - 1) * np + (pq - 1)) * 2));
            }
        }
    }
    net.m = (int64_t)net.si.size();
    if (net.m >= ((int64_t)1 << 31)) { err = "more than 2^31 - 1 springs"; return false; }
    for (double m : net.mass)
        if (!(m > 0)) { err = "mass must be > 0"; return false; }
    net.dt = d.dt;
    net.damping = d.damping;
    net.xc = 0.5 * (nx - 1) * d.a;
    net.omega = (nx - 1) * d.a * (R * h);
    net.grip_area = R * h;
    net.cell = d.a * h;
    net.load_mode = d.load_mode;
    net.precision = d.precision;
    net.grip_mode = d.grip_mode;
    net.a = d.a;
    net.lattice = 1;
    net.nx = nx; net.ny = ny; net.nz = 1;
    net.nphase = np;
    net.phase.assign(d.phase, d.phase + (int64_t)nx * ny);
    return true;
}

bool net_from_image(const lsm_desc &d, HostNet &net, std::string &err)
{
    if (d.lattice != 0 && d.lattice != 1) { err = "lattice must be 0 (square/cubic) or 1 (triangular)"; return false; }
    if (d.lattice == 1 && d.dim != 2) { err = "the triangular packing is 2D"; return false; }
    if (d.dim != 2 && d.dim != 3) { err = "dim must be 2 or 3"; return false; }
    const int nx = d.nx, ny = d.ny, nz = d.dim == 2 ? 1 : d.nz;
    if (nx < 2 || ny < 1 || nz < 1) { err = "image needs nx >= 2, ny >= 1, nz >= 1"; return false; }
    if (!d.phase || !d.k_tab || !d.epsc_tab) { err = "phase, k_tab and epsc_tab are required"; return false; }
    if (d.nphase < 1 || d.nphase > 181) { err = "nphase must be in 1..181"; return false; }
    if (!(d.a > 0) || !(d.dt > 0) || !(d.damping >= 0)) { err = "need a > 0, dt > 0, damping >= 0"; return false; }
    if (d.grip_mode != 0 && d.grip_mode != 1) { err = "grip_mode must be 0 or 1"; return false; }
    if (d.load_mode != 0 && d.load_mode != 1) { err = "load_mode must be 0 or 1"; return false; }
    const int64_t nvox = (int64_t)nx * ny * nz;
    if (nvox > ((int64_t)1 << 31) - 1) { err = "image larger than 2^31 - 1 voxels"; return false; }
    if (d.lattice == 1) return net_from_image_tri(d, net, err);
    const int np = d.nphase;

    std::vector<int64_t> pid(nvox);
    int64_t n = 0;
    for (int64_t v = 0; v < nvox; v++) {
        uint8_t ph = d.phase[v];
        if (ph > np) { err = "phase value above nphase"; return false; }
        pid[v] = ph ? n++ : -1;
    }
    if (n == 0) { err = "image has no particles"; return false; }

    // spring types: (pi, pj, shell) -> dense id
    net.types.assign((size_t)np * np * 2, SpringType{});
    for (int pi = 0; pi < np; pi++)
        for (int pj = 0; pj < np; pj++)
            for (int sh = 1; sh <= 2; sh++) {
                double k = d.k_tab[pi * np + pj];
                double ec = d.epsc_tab[pi * np + pj];
                if (!(k >= 0) || !(ec > -1.0)) { err = "k_tab must be >= 0 and epsc_tab > -1"; return false; }
                double r0 = sh == 1 ? d.a : d.a * std::sqrt(2.0);
                if (sh == 2) k = k * d.k2_ratio;
                double rc = r0 * (1.0 + ec);
                SpringType &t = net.types[((size_t)pi * np + pj) * 2 + (sh - 1)];
                t.k = k;
                t.r0 = r0;
                t.rc2 = rc * rc;
                t.kr0 = k * r0;
            }

    const std::vector<Offset> offs = forward_offsets(d.dim, nx, ny);
    net.offv.clear();
    for (const Offset &o : offs) {
        net.offv.push_back(o.dx * d.a);
        net.offv.push_back(o.dy * d.a);
        net.offv.push_back(o.dz * d.a);
    }
    net.sdir.clear();
    net.sdir.reserve((size_t)n * offs.size());
    net.dim = d.dim;
    net.n = n;
    net.X.assign((size_t)d.dim * n, 0.0);
    net.mass.assign(n, 1.0);
    net.fixm.assign(n, 0);
    net.grip.assign(n, 0);
    net.si.clear(); net.sj.clear(); net.stype.clear();
    net.si.reserve((size_t)n * offs.size());
    net.sj.reserve((size_t)n * offs.size());
    net.stype.reserve((size_t)n * offs.size());
    const uint8_t all = (uint8_t)((1u << d.dim) - 1u);
    for (int iz = 0; iz < nz; iz++)
        for (int iy = 0; iy < ny; iy++)
            for (int ix = 0; ix < nx; ix++) {
                const int64_t v = ix + (int64_t)nx * (iy + (int64_t)ny * iz);
                const int64_t p = pid[v];
                if (p < 0) continue;
                const int ph = d.phase[v];
                net.X[p] = ix * d.a;
                net.X[n + p] = iy * d.a;
                if (d.dim == 3) net.X[2 * n + p] = iz * d.a;
                if (d.mass_tab) net.mass[p] = d.mass_tab[ph - 1];
                if (ix == 0 || ix == nx - 1) {
                    net.grip[p] = ix == 0 ? 1 : 2;
                    net.fixm[p] = d.grip_mode == 1 ? all : 1;
                }
                for (size_t oi = 0; oi < offs.size(); oi++) {
                    const Offset &o = offs[oi];
                    const int jx = ix + o.dx, jy = iy + o.dy, jz = iz + o.dz;
                    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                    const int64_t q = pid[v + o.lin];
                    if (q < 0) continue;
                    const int pq = d.phase[v + o.lin];
                    net.sdir.push_back((uint8_t)oi);
                    net.si.push_back((int32_t)p);
                    net.sj.push_back((int32_t)q);
                    net.stype.push_back((uint16_t)((((ph - 1) * np) + (pq - 1)) * 2 + (o.shell - 1)));
                }
            }
    net.m = (int64_t)net.si.size();
    if (net.m >= ((int64_t)1 << 31)) { err = "more than 2^31 - 1 springs"; return false; }
    for (double m : net.mass)
        if (!(m > 0)) { err = "mass must be > 0"; return false; }
    net.dt = d.dt;
    net.damping = d.damping;
    net.xc = 0.5 * (nx - 1) * d.a;
    net.omega = (nx - 1) * d.a * (ny * d.a);
    net.grip_area = ny * d.a;
    if (d.dim == 3) {
        net.omega = net.omega * (nz * d.a);
        net.grip_area = net.grip_area * (nz * d.a);
    }
    net.cell = std::pow(d.a, (double)d.dim);
    net.load_mode = d.load_mode;
    net.precision = d.precision;
    net.grip_mode = d.grip_mode;
    net.a = d.a;
    net.lattice = 0;
    net.nx = nx; net.ny = ny; net.nz = nz;
    net.nphase = np;
    net.phase.assign(d.phase, d.phase + nvox);
    net.pix.resize(n);
    for (int64_t v = 0; v < nvox; v++)
        if (pid[v] >= 0) net.pix[pid[v]] = v;
    return true;
}

bool net_from_desc(const lsm_net_desc &d, HostNet &net, std::string &err)
{
    if (d.dim != 2 && d.dim != 3) { err = "dim must be 2 or 3"; return false; }
    if (d.n < 1 || d.m < 0 || d.n > ((int64_t)1 << 31) - 1 || d.m > ((int64_t)1 << 31) - 1) {
        err = "need 1 <= n < 2^31 and 0 <= m < 2^31"; return false;
    }
    if (!d.X || (d.m > 0 && (!d.si || !d.sj || !d.k || !d.r0 || !d.rc2))) {
        err = "X and the spring arrays are required"; return false;
    }
    if (!(d.dt > 0) || !(d.damping >= 0) || !(d.omega > 0) || !(d.grip_area > 0)) {
        err = "need dt > 0, damping >= 0, omega > 0, grip_area > 0"; return false;
    }
    net.dim = d.dim;
    net.n = d.n;
    net.m = d.m;
    net.X.assign(d.X, d.X + (size_t)d.dim * d.n);
    net.mass.assign(d.n, 1.0);
    if (d.mass) net.mass.assign(d.mass, d.mass + d.n);
    for (double m : net.mass)
        if (!(m > 0)) { err = "mass must be > 0"; return false; }
    net.fixm.assign(d.n, 0);
    if (d.fix)
        for (int c = 0; c < d.dim; c++)
            for (int64_t p = 0; p < d.n; p++)
                if (d.fix[c * d.n + p]) net.fixm[p] |= (uint8_t)(1u << c);
    net.grip.assign(d.n, 0);
    if (d.grip) {
        for (int64_t p = 0; p < d.n; p++) {
            if (d.grip[p] > 2) { err = "grip codes are 0, 1, 2"; return false; }
            net.grip[p] = d.grip[p];
        }
    }
    net.si.assign(d.si, d.si + d.m);
    net.sj.assign(d.sj, d.sj + d.m);
    std::map<std::tuple<double, double, double>, uint16_t> ids;
    net.types.clear();
    net.stype.resize(d.m);
    for (int64_t s = 0; s < d.m; s++) {
        if (d.si[s] < 0 || d.sj[s] >= d.n || d.si[s] >= d.sj[s]) {
            err = "spring endpoints must satisfy 0 <= si < sj < n"; return false;
        }
        if (s > 0 && (d.si[s] < d.si[s - 1] || (d.si[s] == d.si[s - 1] && d.sj[s] <= d.sj[s - 1]))) {
            err = "springs must be sorted by (si, sj) without duplicates"; return false;
        }
        if (!(d.k[s] >= 0) || !(d.r0[s] > 0) || !(d.rc2[s] >= 0)) {
            err = "need k >= 0, r0 > 0, rc2 >= 0"; return false;
        }
        auto key = std::make_tuple(d.k[s], d.r0[s], d.rc2[s]);
        auto it = ids.find(key);
        if (it == ids.end()) {
            if (net.types.size() >= 65536) { err = "more than 65536 distinct spring parameter triples"; return false; }
            uint16_t id = (uint16_t)net.types.size();
            net.types.push_back(SpringType{d.k[s], d.r0[s], d.rc2[s], d.k[s] * d.r0[s]});
            it = ids.emplace(key, id).first;
        }
        net.stype[s] = it->second;
    }
    if (net.types.empty()) net.types.push_back(SpringType{0, 1, 0, 0});
    net.dt = d.dt;
    net.damping = d.damping;
    net.xc = d.xc;
    net.omega = d.omega;
    net.grip_area = d.grip_area;
    net.load_mode = d.load_mode;
    net.precision = d.precision;
    return true;
}

}  // namespace lsm
