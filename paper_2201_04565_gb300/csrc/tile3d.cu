// tile3d.cu -- one launch per time step for 3D voxel lattices (first and
// second neighbours, 18 springs per interior particle) in the fixed-point
// modes (F32, DF).
//
// A CTA (512 threads) owns a 32 x 8 x 8 block of voxels. Per time step it
//   1. loads the block plus a one-voxel halo (phase, broken flags, positions
//      drifted by dt vh, Eq. 3) into shared memory as 64-bit fixed point;
//   2. compacts the block's particles into a list in raster order (porous
//      volumes leave most voxels void; the list keeps every warp busy);
//   3. for each listed particle evaluates all 18 of its springs, incoming springs by
//      ascending source, then outgoing springs by ascending target (the
//      canonical order of the sequential sum), accumulating the force in
//      registers. Every spring is evaluated by both endpoints from the same
//      data (d = x_upper - x_lower, the upper endpoint negates the force), so
//      both see the same break decision and equal and opposite forces; the
//      lower endpoint records breaks. No shared-memory force exchange and one
//      barrier per step: in 3D that exchange (9 slots x 3 components per
//      source voxel) would cost more shared memory than the recomputation
//      costs arithmetic in these modes;
//      and integrates (Eqs. 4-5) in FP64, writing x(t+dt), vh(t+3dt/2).
// The FP64 modes keep the spring-list kernels for 3D: recomputing every
// spring twice would double their FP64-pipe work.
//
// Broken flags: 9 bits per voxel (its forward springs in slot order, the
// canonical order of the targets), written only by the owning thread; break
// steps [9][nv].
#include "tile_body.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace lsm {

namespace {

constexpr int T3X = 32, T3Y = 8, T3Z = 8, T3V = T3X * T3Y * T3Z;  // voxels per block
constexpr int T3N = 512;                                             // threads per CTA
constexpr int R3X = T3X + 2, R3Y = T3Y + 2, R3Z = T3Z + 2, R3N = R3X * R3Y * R3Z;

// shared memory of one CTA (dynamic)
struct Smem3 {
    long long xf[3][R3N];     // fixed-point drifted positions of the region
    uint16_t mk[R3N];         // broken flags
    uint16_t list[T3V];       // region indices of the block's particles (compacted)
    uint8_t ph[R3N];          // phase (0 = void)
};

struct Tile3Args {
    int nx, ny, nz, nphase;
    int64_t nv;
    const double *x_in, *vh_in;
    double *x_out, *vh_out, *v_obs;
    const uint8_t *phase;
    uint16_t *mask;
    long long *brk;  // [9][nv]
    const TypeDF *tdf;
    const double *mass;
    const Coef4 *coef;
    int S;
    long long a_fix;
    float p24, p0;
    double dt, a, xc;
    int grip_mode;
    int rate_on;  // constant strain rate: grips at rate_eps0 + (s - rate_step0) rate_dt
    double rate_eps0, rate_dt;
    long long rate_step0;
    const long long *d_step;
    int64_t t_off;
    unsigned long long *first_break, *nbroken;
    int *status;
    double *part_s, *part_p;
    int64_t ntiles;
    int sd[9][3];   // forward offsets in canonical (ascending raster) order
    int ssh[9];     // their shells (1: face, 2: edge diagonal)
    float oo2[2];   // |o|^2 per shell as floats (F32 mode)
    float fa;       // lattice spacing as a float (F32 mode)
};

// x of a grip at the strain of the step being computed (constant strain
// rate); the kernel evaluates it for the two grip columns once per thread
__device__ __forceinline__ double rate_grip_x(const Tile3Args &A, int gx)
{
    const long long s = *A.d_step + A.t_off + 1 - A.rate_step0;
    const double eps = __dadd_rn(A.rate_eps0, __dmul_rn((double)s, A.rate_dt));
    const double X = __dmul_rn((double)gx, A.a);
    return __dadd_rn(X, __dmul_rn(eps, __dsub_rn(X, A.xc)));
}

// rate_l, rate_r: the grips' x under the constant strain rate (RATE)
template <int MODE, bool RATE>
__device__ __forceinline__ void load_voxel(const Tile3Args &A, int x0, int y0, int z0, int rx, int ry, int rz,
                                           Smem3 &S, bool &over, double rate_l, double rate_r)
{
    const int gx = x0 - 1 + rx, gy = y0 - 1 + ry, gz = z0 - 1 + rz;
    const int e = rx + R3X * (ry + R3Y * rz);
    uint8_t ph = 0;
    uint16_t mk = 0;
    double px[3] = {0.0, 0.0, 0.0};
    if (gx >= 0 && gx < A.nx && gy >= 0 && gy < A.ny && gz >= 0 && gz < A.nz) {
        const int64_t g = gx + (int64_t)A.nx * (gy + (int64_t)A.ny * gz);
        ph = A.phase[g];
        if (ph) {
            mk = A.mask[g];
            const bool grip = gx == 0 || gx == A.nx - 1;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                px[c] = A.x_in[c * A.nv + g];
                const bool fixed = grip && (c == 0 || A.grip_mode == 1);
                if (MODE == T_STEP && !fixed) px[c] = fma(A.dt, A.vh_in[c * A.nv + g], px[c]);
            }
            if (RATE && MODE == T_STEP && grip) px[0] = gx == 0 ? rate_l : rate_r;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) S.xf[c][e] = dbl_to_fix(px[c], A.S, over);
    S.ph[e] = ph;
    S.mk[e] = mk;
}

// Force of the spring lower -> upper on the lower endpoint (d = x_upper -
// x_lower); false if the spring breaks now (r^2 > rc^2).
template <int PREC, bool TEST>
__device__ __forceinline__ bool spring3(const Tile3Args &A, const long long *dl, const long long *du, int s,
                                        const TypeDF &t, ff *f, ff &w, ff &u, bool sample)
{
    if constexpr (PREC == LSM_PREC_DF) {
        ff d[3];
#pragma unroll
        for (int c = 0; c < 3; c++) d[c] = fix_to_ff_i2f2(du[c] - dl[c], A.p24, A.p0);
        const ff r2 = ff_norm3_un(d[0], d[1], d[2]);
        if (TEST && ff_gt_un(r2, t.rc2)) return false;
        ff y;
        const ff g = ff_spring_g(r2, t.r0, sample ? &y : nullptr);
        const ff cc = ff_mul_un(t.k, g);  // unnormalised: only multiplied or summed further
#pragma unroll
        for (int c = 0; c < 3; c++) f[c] = ff_mul_un(cc, d[c]);
        if (sample) {  // double-float sums: no FP64 pipe work per spring
            const ff st = ff_mul(ff_mul(r2, y), g);  // r - r0
            u = ff_add_sloppy(u, ff_mul(ff_mul_f(t.k, 0.5f), ff_sqr(st)));
            w = ff_add_sloppy(w, ff_mul(d[0], f[0]));
        }
    } else {  // F32: e = d - o exact, (2 o + e).e carries no cancellation
        float e[3], dd[3], num = t.cor.hi;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const long long ef = du[c] - dl[c] - (long long)A.sd[s][c] * A.a_fix;
            e[c] = fix_to_float_i2f(ef, A.p24, A.p0);
            const float o = A.sd[s][c] == 0 ? 0.0f : (A.sd[s][c] > 0 ? A.fa : -A.fa);
            dd[c] = o + e[c];
            num = fmaf(2.0f * o + e[c], e[c], num);
        }
        const float r2f = A.oo2[A.ssh[s] - 1] + num;
        if (TEST && r2f > t.rc2.hi) return false;
        const float ir = rsqrtf(r2f);
        const float st = __fdividef(num, fmaf(r2f, ir, t.r0.hi));  // r - r0
        const float cc = t.k.hi * st * ir;
#pragma unroll
        for (int c = 0; c < 3; c++) f[c] = ff{cc * dd[c], 0.0f};
        if (sample) {
            u = ff_add_f(u, 0.5f * t.k.hi * st * st);
            w = ff_add_f(w, dd[0] * f[0].hi);
        }
    }
    return true;
}

// RATE: constant strain-rate loading (a separate instance, so that the
// ordinary step carries none of its code)
template <int PREC, int MODE, bool SAMPLE, bool RATE>
__global__ void __launch_bounds__(T3N)
k_tile3d(Tile3Args A)
{
    extern __shared__ __align__(16) unsigned char smem3[];
    Smem3 &S = *reinterpret_cast<Smem3 *>(smem3);
    __shared__ TypeDF sdf[128];
    __shared__ Coef4 scoef[8];
    __shared__ float smassf[8];
    __shared__ int soff[9];
    __shared__ int wcount[T3V / 32];  // particles per 32-voxel row, then the rows' offsets
    __shared__ int ntotal;
    __shared__ double sred[T3N / 32];

    const int tid = threadIdx.x, lane = tid & 31;
    const int x0 = blockIdx.x * T3X, y0 = blockIdx.y * T3Y, z0 = blockIdx.z * T3Z;
    const int64_t tile_id = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    const int nt = 2 * A.nphase * A.nphase;
    for (int q = tid; q < nt; q += T3N) sdf[q] = A.tdf[q];
    if (tid < A.nphase) {
        smassf[tid] = (float)A.mass[tid];
        scoef[tid] = A.coef[tid];
    }
    if (tid < 9) soff[tid] = A.sd[tid][0] + R3X * (A.sd[tid][1] + R3Y * A.sd[tid][2]);
    const long long step_now = MODE == T_STEP ? *A.d_step + A.t_off : 0;

    // 1. region (block + one-voxel halo) into shared memory
    bool over = false;
    double rate_l = 0.0, rate_r = 0.0;  // grips' x under the constant strain rate
    if constexpr (RATE && MODE == T_STEP) {
        rate_l = rate_grip_x(A, 0);
        rate_r = rate_grip_x(A, A.nx - 1);
    }
    for (int e = tid; e < R3N; e += T3N) {
        const int rx = e % R3X, ry = (e / R3X) % R3Y, rz = e / (R3X * R3Y);
        load_voxel<MODE, RATE>(A, x0, y0, z0, rx, ry, rz, S, over, rate_l, rate_r);
    }
    if (over) atomicOr(A.status, 2);
    __syncthreads();

    // 2. compact the block's particles (rows of 32 voxels; deterministic order:
    // raster order of the block) so that every warp works on particles
    for (int r = tid >> 5; r < T3V / 32; r += T3N / 32) {
        const int ly = r % T3Y, lz = r / T3Y;
        const int ep = (lane + 1) + R3X * ((ly + 1) + R3Y * (lz + 1));
        const bool live = x0 + lane < A.nx && y0 + ly < A.ny && z0 + lz < A.nz && S.ph[ep];
        const unsigned b = __ballot_sync(0xffffffffu, live);
        if (lane == 0) wcount[r] = __popc(b);
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int r = 0; r < T3V / 32; r++) {
            const int cnt = wcount[r];
            wcount[r] = acc;
            acc += cnt;
        }
        ntotal = acc;
    }
    __syncthreads();
    for (int r = tid >> 5; r < T3V / 32; r += T3N / 32) {
        const int ly = r % T3Y, lz = r / T3Y;
        const int ep = (lane + 1) + R3X * ((ly + 1) + R3Y * (lz + 1));
        const bool live = x0 + lane < A.nx && y0 + ly < A.ny && z0 + lz < A.nz && S.ph[ep];
        const unsigned b = __ballot_sync(0xffffffffu, live);
        if (live) S.list[wcount[r] + __popc(b & ((1u << lane) - 1u))] = (uint16_t)ep;
    }
    __syncthreads();

    // 3. each particle's 18 springs in canonical order, then the integration
    ff w_acc{0.0f, 0.0f}, u_acc{0.0f, 0.0f};
    float mvx2f = 0.0f, kef = 0.0f, resf = 0.0f;
    ff reactf{0.0f, 0.0f};
    bool bad = false;
    const int count = ntotal;
    for (int i = tid; i < count; i += T3N) {
        const int ep = S.list[i];
        const int rx = ep % R3X, ry = (ep / R3X) % R3Y, rz = ep / (R3X * R3Y);
        const int gx = x0 + rx - 1, gy = y0 + ry - 1, gz = z0 + rz - 1;
        const int64_t g = gx + (int64_t)A.nx * (gy + (int64_t)A.ny * gz);
        const int pp = S.ph[ep];
        const uint16_t mk = S.mk[ep];
        const long long xp[3] = {S.xf[0][ep], S.xf[1][ep], S.xf[2][ep]};
        float hs[3] = {0.0f, 0.0f, 0.0f}, el[3] = {0.0f, 0.0f, 0.0f};
        // time steps without a sample issue the integration's global loads
        // here, so their latency hides behind the springs (the sample
        // instance keeps them late: it has no registers to spare)
        constexpr bool PRE = MODE == T_STEP && !SAMPLE;
        double xpre[3], vpre[3];
        if constexpr (PRE) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                xpre[c] = A.x_in[c * A.nv + g];
                vpre[c] = A.vh_in[c * A.nv + g];
            }
        }
        // incoming: source p - o_s, ascending source = descending slot
#pragma unroll 1
        for (int s = 8; s >= 0; s--) {
            const int eq = ep - soff[s];
            const int pq = S.ph[eq];
            if (!pq || ((S.mk[eq] >> s) & 1)) continue;
            const long long xq[3] = {S.xf[0][eq], S.xf[1][eq], S.xf[2][eq]};
            const TypeDF t = sdf[(((pq - 1) * A.nphase) + (pp - 1)) * 2 + (A.ssh[s] - 1)];
            ff f[3], wd{0.0f, 0.0f}, ud{0.0f, 0.0f};
            if (!spring3<PREC, MODE == T_STEP>(A, xq, xp, s, t, f, wd, ud, false)) continue;
#pragma unroll
            for (int c = 0; c < 3; c++) {  // F -= f (cascaded sum)
                const ff tt = two_sum(hs[c], -f[c].hi);
                hs[c] = tt.hi;
                el[c] = __fadd_rn(el[c], __fsub_rn(tt.lo, f[c].lo));
            }
        }
        // outgoing: target p + o_s, ascending slot
        uint16_t newb = 0;
#pragma unroll 1
        for (int s = 0; s < 9; s++) {
            const int eq = ep + soff[s];
            const int pq = S.ph[eq];
            if (!pq || ((mk >> s) & 1)) continue;
            const long long xq[3] = {S.xf[0][eq], S.xf[1][eq], S.xf[2][eq]};
            const TypeDF t = sdf[(((pp - 1) * A.nphase) + (pq - 1)) * 2 + (A.ssh[s] - 1)];
            ff f[3];
            if (!spring3<PREC, MODE == T_STEP>(A, xp, xq, s, t, f, w_acc, u_acc, SAMPLE)) {
                newb |= (uint16_t)(1u << s);
                A.brk[(int64_t)s * A.nv + g] = step_now;
                atomicMin(A.first_break, (unsigned long long)step_now);
                atomicAdd(A.nbroken, 1ull);
                continue;
            }
#pragma unroll
            for (int c = 0; c < 3; c++) {  // F += f
                const ff tt = two_sum(hs[c], f[c].hi);
                hs[c] = tt.hi;
                el[c] = __fadd_rn(el[c], __fadd_rn(tt.lo, f[c].lo));
            }
        }
        if (MODE == T_STEP && newb) A.mask[g] = (uint16_t)(mk | newb);

        // integration (Eqs. 4-5), FP64; the drift is recomputed exactly as in
        // the region load (same operations on the same inputs)
        const bool grip = gx == 0 || gx == A.nx - 1;
        const int ph = pp - 1;
        if (SAMPLE && gx == A.nx - 1) reactf = ff_add_sloppy(reactf, ff{-hs[0], -el[0]});
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const bool fixed = grip && (c == 0 || A.grip_mode == 1);
            const int64_t q = c * A.nv + g;
            const double F = f2d_force(hs[c]) + f2d_force(el[c]);
            const float Ff = __fadd_rn(hs[c], el[c]);
            double xr;
            double vh;
            if constexpr (PRE) {
                xr = xpre[c];
                vh = vpre[c];
            } else {
                xr = A.x_in[q];
                vh = MODE == T_INIT ? A.v_obs[q] : A.vh_in[q];
            }
            if (MODE == T_STEP && !fixed) xr = fma(A.dt, vh, xr);
            if (RATE && MODE == T_STEP && c == 0 && grip) xr = gx == 0 ? rate_l : rate_r;
            if (MODE == T_STEP) A.x_out[q] = xr;
            if (fixed) {
                if (MODE == T_STEP) A.vh_out[q] = 0.0;
                if (MODE == T_STEP && SAMPLE) A.v_obs[q] = 0.0;
                continue;
            }
            if (MODE == T_OBSERVE) {
                if (SAMPLE) {
                    const float vf = d2f_bits(A.v_obs[q]);
                    resf = fmaxf(resf, fmaxf(fabsf(Ff), fabsf(vf)));
                    kef = fmaf(0.5f * smassf[ph] * vf, vf, kef);
                    if (c == 0) mvx2f = fmaf(smassf[ph] * vf, vf, mvx2f);
                }
                continue;
            }
            const Coef4 k4 = scoef[ph];
            const double vn = fma(k4.c2h, F, k4.c1h * vh);
            if (MODE == T_INIT) {
                A.vh_out[q] = vn;
                continue;
            }
            A.vh_out[q] = fma(k4.c2, F, k4.c1 * vh);
            if (SAMPLE) {
                A.v_obs[q] = vn;
                const float vf = d2f_bits(vn);
                resf = fmaxf(resf, fmaxf(fabsf(Ff), fabsf(vf)));
                kef = fmaf(0.5f * smassf[ph] * vf, vf, kef);
                if (c == 0) mvx2f = fmaf(smassf[ph] * vf, vf, mvx2f);
                bad |= !dbl_finite_bits(vn) || !dbl_finite_bits(xr);
            }
        }
    }
    if (SAMPLE) {
        if (bad) atomicOr(A.status, 1);
        const double t0 = bsum_ff<T3N / 32>(w_acc, sred);
        const double t1 = bsum_ff<T3N / 32>(u_acc, sred);
        const double t2 = bsum_ff<T3N / 32>(ff{mvx2f, 0.0f}, sred);
        const double t3 = bsum_ff<T3N / 32>(ff{kef, 0.0f}, sred);
        const double t4 = bsum_ff<T3N / 32>(reactf, sred);
        const double t5 = bmax_f<T3N / 32>(resf, sred);
        if (tid == 0) {
            A.part_s[tile_id] = t0;
            A.part_s[A.ntiles + tile_id] = t1;
            A.part_p[tile_id] = t2;
            A.part_p[A.ntiles + tile_id] = t3;
            A.part_p[2 * A.ntiles + tile_id] = t4;
            A.part_p[3 * A.ntiles + tile_id] = t5;
        }
    }
}

// voxel-grid broken flags / break steps -> canonical spring order
__global__ void k_tile3_export(int nx, int ny, int nz, int64_t nv, Tile3Args A, const uint8_t *__restrict__ phase,
                               const uint16_t *__restrict__ mask, const long long *__restrict__ brk,
                               const int64_t *__restrict__ sbase, uint8_t *__restrict__ out_mask,
                               long long *__restrict__ out_brk)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nv || !phase[g]) return;
    const int gx = (int)(g % nx), gy = (int)((g / nx) % ny), gz = (int)(g / ((int64_t)nx * ny));
    int64_t b = sbase[g];
    const uint16_t mk = mask[g];
    for (int s = 0; s < 9; s++) {
        const int qx = gx + A.sd[s][0], qy = gy + A.sd[s][1], qz = gz + A.sd[s][2];
        if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || qz < 0 || qz >= nz) continue;
        if (!phase[qx + (int64_t)nx * (qy + (int64_t)ny * qz)]) continue;
        if (out_mask) out_mask[b] = (mk >> s) & 1u;
        if (out_brk) out_brk[b] = brk[(int64_t)s * nv + g];
        b++;
    }
}

Tile3Args tile3_args(Ctx &c)
{
    Tile3Args A{};
    A.nx = c.h.nx;
    A.ny = c.h.ny;
    A.nz = c.h.nz;
    A.nphase = c.tile_nphase;
    A.nv = c.tnp;
    A.x_in = c.tx[c.tcur];
    A.vh_in = c.tvh[c.tcur];
    A.x_out = c.tx[c.tcur ^ 1];
    A.vh_out = c.tvh[c.tcur ^ 1];
    A.v_obs = c.tvobs;
    A.phase = c.tph;
    A.mask = c.tmask3;
    A.brk = c.tbrk;
    A.tdf = c.tdf;
    A.mass = c.tmass;
    A.coef = (const Coef4 *)c.tinvm;
    A.S = c.fix_S;
    A.a_fix = c.a_fix;
    A.p24 = ldexpf(1.0f, 24 - c.fix_S);
    A.p0 = ldexpf(1.0f, -c.fix_S);
    A.dt = c.h.dt;
    A.a = c.h.a;
    A.xc = c.h.xc;
    A.grip_mode = c.h.grip_mode;
    A.rate_on = c.rate_on;
    A.rate_eps0 = c.rate_eps0;
    A.rate_dt = c.rate_dt;
    A.rate_step0 = c.rate_step0;
    A.d_step = c.d_step;
    A.first_break = c.d_first_break;
    A.nbroken = c.d_nbroken;
    A.status = c.d_status;
    A.part_s = c.part_s;
    A.part_p = c.part_p;
    A.ntiles = c.ntiles;
    const double aa = std::ldexp((double)c.a_fix, -c.fix_S);
    for (int s = 0; s < 9; s++) {
        int l2 = 0;
        for (int k = 0; k < 3; k++) {
            A.sd[s][k] = (int)std::lround(c.h.offv[3 * s + k] / c.h.a);
            l2 += A.sd[s][k] * A.sd[s][k];
        }
        A.ssh[s] = l2;
    }
    A.fa = (float)aa;
    A.oo2[0] = (float)(aa * aa);
    A.oo2[1] = (float)(2.0 * aa * aa);
    return A;
}

template <int PREC, int MODE, bool SAMPLE, bool RATE>
cudaError_t launch3(Ctx &c, Tile3Args A)
{
    auto kern = k_tile3d<PREC, MODE, SAMPLE, RATE>;
    static bool configured = false;  // per template instance
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem3));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const dim3 grid((c.h.nx + T3X - 1) / T3X, (c.h.ny + T3Y - 1) / T3Y, (c.h.nz + T3Z - 1) / T3Z);
    kern<<<grid, T3N, sizeof(Smem3), c.stream>>>(A);
    return cudaSuccess;
}

template <int MODE, bool SAMPLE>
cudaError_t launch3_prec(Ctx &c, Tile3Args A)
{
    if constexpr (MODE == T_STEP) {
        if (c.rate_on) {
            if (c.h.precision == LSM_PREC_F32) return launch3<LSM_PREC_F32, MODE, SAMPLE, true>(c, A);
            return launch3<LSM_PREC_DF, MODE, SAMPLE, true>(c, A);
        }
    }
    if (c.h.precision == LSM_PREC_F32) return launch3<LSM_PREC_F32, MODE, SAMPLE, false>(c, A);
    return launch3<LSM_PREC_DF, MODE, SAMPLE, false>(c, A);
}

ff split_ff3(double v)
{
    const float hi = (float)v;
    return ff{hi, (float)(v - (double)hi)};
}

template <typename T>
cudaError_t dal(T **p, size_t count)
{
    return lsm::dev_malloc((void **)p, (count ? count : 1) * sizeof(T));
}

}  // namespace

int64_t tile3_count(const Ctx &c)
{
    return (int64_t)((c.h.nx + T3X - 1) / T3X) * ((c.h.ny + T3Y - 1) / T3Y) * ((c.h.nz + T3Z - 1) / T3Z);
}

cudaError_t tile3_upload(Ctx &c)
{
    const HostNet &h = c.h;
    const int64_t nv = (int64_t)h.nx * h.ny * h.nz;
    c.tnp = nv;
    c.tile_nphase = h.nphase;
    c.ntiles = tile3_count(c);
    c.tgidx.assign(h.pix.begin(), h.pix.end());  // grid index of each particle: its voxel
    c.tgnx = h.nx;                                // rows of nx voxels, x fastest (the load
    c.tgny = h.ny * h.nz;                         // increment's kernel works per row)
    std::vector<double> X(3 * nv);
    for (int64_t g = 0; g < nv; g++) {
        X[g] = (g % h.nx) * h.a;
        X[nv + g] = ((g / h.nx) % h.ny) * h.a;
        X[2 * nv + g] = (g / ((int64_t)h.nx * h.ny)) * h.a;
    }
    std::vector<double> mtab(h.nphase, 1.0), itab(4 * h.nphase, 0.0);
    for (int64_t p = 0; p < h.n; p++) mtab[h.phase[h.pix[p]] - 1] = h.mass[p];
    for (int q = 0; q < h.nphase; q++) {
        const double dt = h.dt, hdt = 0.5 * h.dt, gm = h.damping, m = mtab[q];
        itab[4 * q + 0] = 1.0 - dt * gm / m;
        itab[4 * q + 1] = dt / m;
        itab[4 * q + 2] = 1.0 - hdt * gm / m;
        itab[4 * q + 3] = hdt / m;
    }
    const int maxext = std::max(h.nx, std::max(h.ny, h.nz));
    c.fix_S = 61 - (int)std::ceil(std::log2(4.0 * maxext * h.a + 16.0));
    c.fix_S = std::min(c.fix_S, 47 - (int)std::ceil(std::log2(h.a * std::sqrt(2.0))));
    c.fix_S = std::min(c.fix_S, 47 - (int)std::floor(std::log2(max_critical_length(h.types))));
    c.a_fix = std::llround(std::ldexp(h.a, c.fix_S));
    const double aa = std::ldexp((double)c.a_fix, -c.fix_S);
    std::vector<TypeDF> tdf(h.types.size());
    for (size_t q = 0; q < h.types.size(); q++) {
        const SpringType &t = h.types[q];
        const double shell = (q & 1) ? 2.0 : 1.0;
        const double p = t.r0 * t.r0, pe = std::fma(t.r0, t.r0, -p);
        const double o2 = shell * aa * aa, o2e = shell * std::fma(aa, aa, -(aa * aa));
        tdf[q].k = split_ff3(t.k);
        tdf[q].r0 = split_ff3(t.r0);
        tdf[q].rc2 = split_ff3(t.rc2);
        tdf[q].cor = split_ff3((o2 - p) + (o2e - pe));
    }
    std::vector<int64_t> sbase(nv, 0);
    for (int64_t s = h.m - 1; s >= 0; s--) sbase[h.pix[h.si[s]]] = s;
    cudaError_t e;
#define T3_TRY(x)                             \
    do {                                      \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    for (int b = 0; b < 2; b++) {
        T3_TRY(dal(&c.tx[b], 3 * nv));
        T3_TRY(dal(&c.tvh[b], 3 * nv));
    }
    T3_TRY(dal(&c.tvobs, 3 * nv));
    T3_TRY(dal(&c.tph, nv));
    T3_TRY(dal(&c.tmask3, nv));
    T3_TRY(dal(&c.tbrk, 9 * nv));
    T3_TRY(dal(&c.tmass, h.nphase));
    T3_TRY(dal(&c.tinvm, 4 * h.nphase));
    T3_TRY(dal(&c.tdf, tdf.size()));
    T3_TRY(dal(&c.tsbase, nv));
    T3_TRY(dal(&c.part_s, 2 * c.ntiles));
    T3_TRY(dal(&c.part_p, 4 * c.ntiles));
    cudaStream_t st = c.stream;
    for (int b = 0; b < 2; b++) {
        T3_TRY(cudaMemcpyAsync(c.tx[b], X.data(), 3 * nv * sizeof(double), cudaMemcpyHostToDevice, st));
        T3_TRY(cudaMemsetAsync(c.tvh[b], 0, 3 * nv * sizeof(double), st));
    }
    T3_TRY(cudaMemsetAsync(c.tvobs, 0, 3 * nv * sizeof(double), st));
    T3_TRY(cudaMemcpyAsync(c.tph, h.phase.data(), nv, cudaMemcpyHostToDevice, st));
    T3_TRY(cudaMemsetAsync(c.tmask3, 0, nv * sizeof(uint16_t), st));
    T3_TRY(cudaMemsetAsync(c.tbrk, 0xff, 9 * nv * sizeof(long long), st));
    T3_TRY(cudaMemcpyAsync(c.tmass, mtab.data(), h.nphase * sizeof(double), cudaMemcpyHostToDevice, st));
    T3_TRY(cudaMemcpyAsync(c.tinvm, itab.data(), 4 * h.nphase * sizeof(double), cudaMemcpyHostToDevice, st));
    T3_TRY(cudaMemcpyAsync(c.tdf, tdf.data(), tdf.size() * sizeof(TypeDF), cudaMemcpyHostToDevice, st));
    T3_TRY(cudaMemcpyAsync(c.tsbase, sbase.data(), nv * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    c.tcur = 0;
    T3_TRY(cudaStreamSynchronize(st));
#undef T3_TRY
    return cudaSuccess;
}

cudaError_t tile3_enqueue_steps(Ctx &c, int64_t nsteps, int start_buf)
{
    int cur = start_buf;
    for (int64_t t = 0; t < nsteps; t++) {
        Tile3Args A = tile3_args(c);
        A.t_off = t;
        A.x_in = c.tx[cur];
        A.vh_in = c.tvh[cur];
        A.x_out = c.tx[cur ^ 1];
        A.vh_out = c.tvh[cur ^ 1];
        cudaError_t e = t == nsteps - 1 ? launch3_prec<T_STEP, true>(c, A) : launch3_prec<T_STEP, false>(c, A);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    return cudaGetLastError();
}

cudaError_t tile3_init_accel(Ctx &c)
{
    Tile3Args A = tile3_args(c);
    A.vh_out = c.tvh[c.tcur];
    cudaError_t e = launch3_prec<T_INIT, false>(c, A);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t tile3_observe(Ctx &c)
{
    cudaError_t e = launch3_prec<T_OBSERVE, true>(c, tile3_args(c));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t tile3_export(Ctx &c, bool steps)
{
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
    k_tile3_export<<<g, 256, 0, c.stream>>>(c.h.nx, c.h.ny, c.h.nz, c.tnp, tile3_args(c), c.tph, c.tmask3, c.tbrk,
                                            c.tsbase, steps ? nullptr : c.texport,
                                            steps ? c.texport_brk : nullptr);
    return cudaGetLastError();
}

}  // namespace lsm
