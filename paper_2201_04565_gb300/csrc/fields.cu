// fields.cu -- per-particle virial stress and Lagrangian strain (Section 3.2,
// Eqs. 7-8) of the current state, for stress and strain maps.
//
// One thread per particle walks the particle's springs in ascending spring
// order (the CSR incidence list) and
//   - adds 1/2 c d_a d_b for every intact spring, d = x_j - x_i and
//     c = k (r - r0)/r, which is (x_l - x_k)_a f_b seen from either endpoint
//     (the force on i is c d, on j it is -c d);
//   - forms A = sum X X^T and B = sum d X^T over its first-neighbour shell
//     (springs with the particle's smallest rest length), X the reference
//     bond vectors, so that J = B A^-1 is the least-squares affine map and
//     (J^T J - I)/2 the Lagrangian strain.
// All arithmetic is correctly rounded FP64 (no contraction); the kernel is
// post-processing, off the time-step path.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "lsm_internal.h"

namespace lsm {

namespace {

constexpr int FB = 128;

__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }

// component pairs of a symmetric tensor: 2D xx, yy, xy; 3D xx, yy, zz, xy, xz, yz
__device__ __forceinline__ void comp_pair(int dim, int q, int &a, int &b)
{
    if (dim == 2) {
        a = q == 1 ? 1 : 0;
        b = q == 0 ? 0 : 1;
    } else {
        const int ta[6] = {0, 1, 2, 0, 0, 1}, tb[6] = {0, 1, 2, 1, 2, 2};
        a = ta[q];
        b = tb[q];
    }
}

template <int DIM>
__global__ void __launch_bounds__(FB)
k_fields(int64_t n, const int64_t *__restrict__ row, const uint32_t *__restrict__ inc,
         const int32_t *__restrict__ si, const int32_t *__restrict__ sj, const uint16_t *__restrict__ stype,
         const SpringType *__restrict__ types, const uint8_t *__restrict__ state, const double *__restrict__ x,
         const double *__restrict__ v, const double *__restrict__ X, const double *__restrict__ mass, double cell,
         double *__restrict__ stress, double *__restrict__ strain)
{
    constexpr int NQ = DIM == 3 ? 6 : 3;
    const int64_t p = (int64_t)blockIdx.x * FB + threadIdx.x;
    if (p >= n) return;
    const int64_t e0 = row[p], e1 = row[p + 1];
    if (stress) {
        double S[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) S[q] = 0.0;
        for (int64_t e = e0; e < e1; e++) {
            const int64_t s = inc[e] >> 1;
            if (state[s]) continue;
            const int64_t i = si[s], j = sj[s];
            const SpringType t = types[stype[s]];
            double d[DIM];
#pragma unroll
            for (int c = 0; c < DIM; c++) d[c] = sub_(x[c * n + j], x[c * n + i]);
            double r2 = add_(mul_(d[0], d[0]), mul_(d[1], d[1]));
            if (DIM == 3) r2 = add_(r2, mul_(d[DIM - 1], d[DIM - 1]));
            const double r = __dsqrt_rn(r2);
            const double cs = div_(mul_(t.k, sub_(r, t.r0)), r);
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                int a, b;
                comp_pair(DIM, q, a, b);
                S[q] = add_(S[q], mul_(0.5, mul_(d[a], mul_(cs, d[b]))));
            }
        }
        const double mp = mass[p];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            int a, b;
            comp_pair(DIM, q, a, b);
            const double vv = mul_(mul_(mp, v[a * n + p]), v[b * n + p]);
            stress[q * n + p] = div_(sub_(S[q], vv), cell);
        }
    }
    if (strain) {
        double rmin = INFINITY;
        for (int64_t e = e0; e < e1; e++) rmin = fmin(rmin, types[stype[inc[e] >> 1]].r0);
        const double rlim = mul_(rmin, 1.0 + 1e-12);
        double A[DIM][DIM], B[DIM][DIM];
#pragma unroll
        for (int a = 0; a < DIM; a++)
#pragma unroll
            for (int b = 0; b < DIM; b++) A[a][b] = B[a][b] = 0.0;
        for (int64_t e = e0; e < e1; e++) {
            const int64_t s = inc[e] >> 1;
            if (types[stype[s]].r0 > rlim) continue;
            const int64_t i = si[s], j = sj[s];
            double Xd[DIM], d[DIM];
#pragma unroll
            for (int c = 0; c < DIM; c++) {
                Xd[c] = sub_(X[c * n + j], X[c * n + i]);
                d[c] = sub_(x[c * n + j], x[c * n + i]);
            }
#pragma unroll
            for (int a = 0; a < DIM; a++)
#pragma unroll
                for (int b = 0; b < DIM; b++) {
                    A[a][b] = add_(A[a][b], mul_(Xd[a], Xd[b]));
                    B[a][b] = add_(B[a][b], mul_(d[a], Xd[b]));
                }
        }
        // inverse of the symmetric A by cofactors
        double inv[DIM][DIM], det, scale;
        if constexpr (DIM == 2) {
            det = sub_(mul_(A[0][0], A[1][1]), mul_(A[0][1], A[1][0]));
            scale = mul_(mul_(0.5, add_(A[0][0], A[1][1])), mul_(0.5, add_(A[0][0], A[1][1])));
            inv[0][0] = div_(A[1][1], det);
            inv[0][1] = div_(-A[0][1], det);
            inv[1][0] = div_(-A[1][0], det);
            inv[1][1] = div_(A[0][0], det);
        } else {
            double cof[3][3];
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
                    cof[a][b] = sub_(mul_(A[a1][b1], A[a2][b2]), mul_(A[a1][b2], A[a2][b1]));
                }
            det = add_(add_(mul_(A[0][0], cof[0][0]), mul_(A[0][1], cof[0][1])), mul_(A[0][2], cof[0][2]));
            const double tr = div_(add_(add_(A[0][0], A[1][1]), A[2][2]), 3.0);
            scale = mul_(mul_(tr, tr), tr);
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) inv[a][b] = div_(cof[b][a], det);
        }
        if (!(fabs(det) > mul_(1e-12, scale))) {
#pragma unroll
            for (int q = 0; q < NQ; q++) strain[q * n + p] = NAN;
            return;
        }
        double J[DIM][DIM];  // J = B A^-1
#pragma unroll
        for (int a = 0; a < DIM; a++)
#pragma unroll
            for (int b = 0; b < DIM; b++) {
                double t = 0.0;
#pragma unroll
                for (int c = 0; c < DIM; c++) t = add_(t, mul_(B[a][c], inv[c][b]));
                J[a][b] = t;
            }
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            int a, b;
            comp_pair(DIM, q, a, b);
            double t = 0.0;
#pragma unroll
            for (int c = 0; c < DIM; c++) t = add_(t, mul_(J[c][a], J[c][b]));
            strain[q * n + p] = mul_(0.5, sub_(t, a == b ? 1.0 : 0.0));
        }
    }
}

// pixel/voxel-grid state of the tile paths -> compact particle order
__global__ void k_fields_compact(int64_t n, int64_t np, int dim, const int64_t *__restrict__ pix,
                                 const double *__restrict__ gx, const double *__restrict__ gv, double *__restrict__ x,
                                 double *__restrict__ v)
{
    const int64_t p = (int64_t)blockIdx.x * FB + threadIdx.x;
    if (p >= n) return;
    const int64_t g = pix[p];
    for (int c = 0; c < dim; c++) {
        x[c * n + p] = gx[c * np + g];
        v[c * n + p] = gv[c * np + g];
    }
}

template <typename T>
cudaError_t up(T **dst, const T *src, size_t count, cudaStream_t st)
{
    cudaError_t e = lsm::dev_malloc((void **)dst, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess || !count) return e;
    return cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
}

}  // namespace

void fields_free(Ctx &c)
{
    void *ptrs[] = {c.fX, c.fx, c.fv, c.fout, c.frow, c.finc, c.fsi, c.fsj, c.fstype, c.fmass, c.fpix};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    c.fX = c.fx = c.fv = c.fout = c.fmass = nullptr;
    c.frow = c.fpix = nullptr;
    c.finc = nullptr;
    c.fsi = c.fsj = nullptr;
    c.fstype = nullptr;
}

cudaError_t fields_compute(Ctx &c, double cell)
{
    const HostNet &h = c.h;
    const int64_t n = c.n, m = c.m;
    const int nq = h.dim == 3 ? 6 : 3;
    cudaStream_t st = c.stream;
    cudaError_t e;
    if (!c.fout) {
        if ((e = lsm::dev_malloc((void **)&c.fout, (size_t)2 * nq * (n ? n : 1) * sizeof(double))) != cudaSuccess) return e;
        if ((e = up(&c.fX, h.X.data(), (size_t)h.dim * n, st)) != cudaSuccess) return e;
        if (c.tile) {
            // spring lists and the incidence CSR, built here once
            std::vector<int64_t> row(n + 1, 0);
            for (int64_t s = 0; s < m; s++) {
                row[h.si[s] + 1]++;
                row[h.sj[s] + 1]++;
            }
            for (int64_t p = 0; p < n; p++) row[p + 1] += row[p];
            std::vector<uint32_t> inc(2 * m);
            std::vector<int64_t> fill(row.begin(), row.end() - 1);
            for (int64_t s = 0; s < m; s++) {
                inc[fill[h.si[s]]++] = (uint32_t)(s << 1);
                inc[fill[h.sj[s]]++] = (uint32_t)((s << 1) | 1);
            }
            if ((e = up(&c.frow, row.data(), row.size(), st)) != cudaSuccess) return e;
            if ((e = up(&c.finc, inc.data(), inc.size(), st)) != cudaSuccess) return e;
            if ((e = up(&c.fsi, h.si.data(), h.si.size(), st)) != cudaSuccess) return e;
            if ((e = up(&c.fsj, h.sj.data(), h.sj.size(), st)) != cudaSuccess) return e;
            if ((e = up(&c.fstype, h.stype.data(), h.stype.size(), st)) != cudaSuccess) return e;
            if ((e = up(&c.fmass, h.mass.data(), h.mass.size(), st)) != cudaSuccess) return e;
            if (c.dim == 2) {  // grid index of each particle (pixel, or site of the packing)
                if ((e = up(&c.fpix, c.tgidx.data(), c.tgidx.size(), st)) != cudaSuccess) return e;
            } else if ((e = up(&c.fpix, h.pix.data(), h.pix.size(), st)) != cudaSuccess) {
                return e;
            }
            if ((e = lsm::dev_malloc((void **)&c.fx, (size_t)h.dim * (n ? n : 1) * sizeof(double))) != cudaSuccess) return e;
            if ((e = lsm::dev_malloc((void **)&c.fv, (size_t)h.dim * (n ? n : 1) * sizeof(double))) != cudaSuccess) return e;
            // the host vectors above must outlive their copies
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        }
    }
    if (n == 0) return cudaSuccess;
    const unsigned g = (unsigned)((n + FB - 1) / FB);
    const double *x = c.x, *v = c.v, *mass = c.mass;
    const int64_t *row = c.row;
    const uint32_t *inc = c.inc;
    const int32_t *si = c.si, *sj = c.sj;
    const uint16_t *stype = c.stype;
    const uint8_t *state = c.state;
    if (c.tile) {
        k_fields_compact<<<g, FB, 0, st>>>(n, c.tnp, h.dim, c.fpix, c.tx[c.tcur], c.tvobs, c.fx, c.fv);
        if ((e = tile_export(c, false)) != cudaSuccess) return e;  // canonical broken flags -> texport
        x = c.fx;
        v = c.fv;
        mass = c.fmass;
        row = c.frow;
        inc = c.finc;
        si = c.fsi;
        sj = c.fsj;
        stype = c.fstype;
        state = m ? c.texport : nullptr;
        if (!m) state = (const uint8_t *)c.fout;  // never read: no springs
    }
    double *stress = c.fout, *strain = c.fout + (size_t)nq * n;
    if (h.dim == 3)
        k_fields<3><<<g, FB, 0, st>>>(n, row, inc, si, sj, stype, c.types, state, x, v, c.fX, mass, cell, stress,
                                      strain);
    else
        k_fields<2><<<g, FB, 0, st>>>(n, row, inc, si, sj, stype, c.types, state, x, v, c.fX, mass, cell, stress,
                                      strain);
    return cudaGetLastError();
}

}  // namespace lsm
