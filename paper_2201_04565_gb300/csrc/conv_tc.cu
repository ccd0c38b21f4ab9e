// conv_tc.cu -- the U-Net's convolutions on the 5th-generation tensor cores.
//
// Both kernels are implicit GEMMs with BF16 operands staged by the tensor
// memory accelerator (TMA) into swizzled shared memory and FP32 accumulators
// in tensor memory (TMEM):
//
//   forward   D[pixel][co] = sum over (tap, ci) of in[pixel shifted by tap][ci]
//             W[co][tap][ci]; M = 128 pixels (a bx x by patch of one image),
//             N = BN output channels, K = taps x Cin in chunks of KC = 64
//             (or 32) channels of one tap. Both operands K-major: the input
//             patch is one 4D TMA box (channels, x, y, image) at the tap's
//             shifted origin, whose out-of-image part the TMA fills with
//             zeros (the convolution's zero padding), and the weights one 2D
//             box. Persistent CTAs walk a static list of tiles; warp 0 issues
//             the copies into an S-stage ring, warp 1 the MMAs, and warps
//             2-5 drain the accumulator (bias, ReLU, BF16 stores), which is
//             double-buffered in TMEM so that the next tile's MMAs overlap
//             the epilogue.
//   wgrad     D[tap, ci][co] = sum over pixels p of in[p shifted by tap][ci]
//             grad[p][co]; M = 128 rows of (tap, ci), N = BN output channels,
//             K = pixels in patches of 64. Both operands MN-major (channels
//             contiguous), copied by TMA boxes of KC channels x 64 pixels;
//             the pixel patches are split over CTAs and each split's tile
//             stored as a partial, folded afterwards in a fixed order (so the
//             result does not depend on timing).
//
// Every mbarrier wait is bounded (g_conv_wait_limit polls): a role that gives
// up raises g_conv_timeout and a flag in shared memory that the CTA's other
// roles see in their own waits; the CTA then waits (bounded again, with the
// default limit) for the copies and MMAs it has issued, frees its TMEM and
// returns, and the host reports the convolution as timed out. (Grids are
// about one wave, so CTAs do not consult each other: each one runs into its
// own bounded waits.)
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "nn_internal.h"

namespace lsm {
namespace nn {

__device__ int g_conv_timeout;

constexpr int TC_WAIT = 1 << 20;
__device__ int g_conv_wait_limit = TC_WAIT;

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned cv_smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of the given parity, at most `limit` polls; gives up
// early once another role of the CTA has given up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int limit, const volatile int *abort)
{
    for (int it = 0; it < limit; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 31) == 31 && *abort) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// TMA tile loads into this CTA's shared memory, completing on an mbarrier
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap *map, unsigned bar, int c0, int c1,
                                            int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, unsigned bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void tma_prefetch(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}
// TMA tile store from this CTA's shared memory (bulk async-group completion);
// the part of the box outside the tensor is not written
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, unsigned src, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                     (uint64_t)map),
                 "r"(src), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one of this thread's bulk groups still reading shared memory
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// every bulk group of this thread complete (writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// this thread's shared-memory writes made visible to the TMA (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// barrier 1 over the 128 epilogue threads (barrier 0 is __syncthreads)
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), descriptor version 1 (bit 46), swizzle mode in
// bits 61-63 (2: 128-byte, 4: 64-byte). K-major swizzled tiles: rows of one
// swizzle width, 8-row groups SBO apart (LBO unused). MN-major swizzled
// tiles: K rows of one swizzle width holding consecutive M (or N) elements,
// 8-row groups SBO apart along K, blocks of one swizzle width LBO apart
// along M (or N).
__device__ __forceinline__ uint64_t sdesc_sw(unsigned addr, unsigned lbo, unsigned sbo, unsigned mode)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46) | ((uint64_t)mode << 61);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), A / B MN-major (bits 15 / 16), N / 8 (bits
// 17-22), M / 16 (bits 24-28).
__host__ __device__ constexpr unsigned idesc_bf16(int m, int n, bool mn_major)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (mn_major ? (1u << 15) | (1u << 16) : 0u) |
           ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem, uint64_t ad, uint64_t bd, unsigned id, unsigned accum)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(accum));
}
__device__ __forceinline__ void mma_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 16 columns of FP32 from TMEM (this warp's lane quarter), not
// waited for (tmem_wait_ld before the registers are read)
__device__ __forceinline__ void tmem_ld16_nw(unsigned addr, unsigned *v)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 16 columns of FP32 from TMEM (this warp's lane quarter)
__device__ __forceinline__ void tmem_ld16(unsigned addr, unsigned *v)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(unsigned *slot, int cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cv_smem_u32(slot)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(unsigned tmem, int cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// a role gives up: the CTA's flag and the device-wide one the host reads
__device__ __forceinline__ void give_up(volatile int *abort)
{
    *abort = 1;
    atomicOr(&g_conv_timeout, 1);
}

// the wait variant for draining after a give-up: never cut short
__device__ __forceinline__ bool mbar_wait_plain(unsigned bar, unsigned parity, int limit)
{
    for (int it = 0; it < limit; it++)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// patch mt of the image grid: image b, top-left (x0, y0) of a bx x by patch
__device__ __forceinline__ void patch_of(int mt, int ntx, int nty, int bx, int by, int &b, int &y0, int &x0)
{
    const int per = ntx * nty;
    b = mt / per;
    const int r = mt - b * per, ty = r / ntx;
    y0 = ty * by;
    x0 = (r - ty * ntx) * bx;
}

// ---------------------------------------------------------- conv forward

constexpr int FW_THREADS = 192;  // warp 0 copies, warp 1 MMAs, warps 2-5 epilogue

// stages of MT input boxes (128 pixels x KC channels each) and one weight
// box (BN x KC) in a ring of at most 192 KB, at most 8
__host__ __device__ constexpr int fwd_stages(int BN, int KC, int MT)
{
    return (196608 / ((128 * MT + BN) * KC * 2)) < 8 ? (196608 / ((128 * MT + BN) * KC * 2)) : 8;
}

// Output staging of the epilogue: blocks of SB = min(BN, 64) channels of the
// tile's 128 pixels, in two alternating shared-memory buffers, each stored
// by one TMA copy (box SB channels x bx x by).
__host__ __device__ constexpr int out_block(int BN) { return BN < 64 ? BN : 64; }
__host__ __device__ constexpr unsigned out_staging(int BN) { return 2u * 128u * (unsigned)out_block(BN) * 2u; }

template <int BN, int KC, int MT>
struct FwdCfg {
    static constexpr int S = fwd_stages(BN, KC, MT);
    static constexpr unsigned ROW = KC * 2;  // bytes per operand row: one swizzle width
    static constexpr unsigned A_BYTES = 128 * ROW, B_BYTES = BN * ROW, STAGE = MT * A_BYTES + B_BYTES;
    // ring, output staging, + slack to align the ring to 1024 bytes
    static constexpr unsigned SMEM = S * STAGE + out_staging(BN) + 1024;
    static constexpr unsigned SW = KC == 64 ? 2u : 4u;  // 128- or 64-byte swizzle
};

// Epilogue of one tile, run by the 128 epilogue threads; this thread holds
// pixel m of the tile (TMEM lane m, taddr: its lane quarter's first
// accumulator column). Per block of SB channels: the accumulator columns
// (all loads issued, one wait), bias and ReLU, BF16 into a staging buffer
// in the TMA's swizzled layout (16-byte chunk j of row m at chunk j ^ (m & 7)
// for 128-byte rows, j ^ ((m >> 1) & 3) for 64-byte rows), then thread 0 of
// the group stores the block with one TMA copy at (n0 + block, x0, y0, b),
// which leaves out the pixels outside the image. The two staging buffers
// alternate (`blk` counts the blocks this thread has staged); before one is
// rewritten, the copy that read it two blocks earlier must have finished
// reading (wait_group.read 1).
template <int BN>
__device__ __forceinline__ void fwd_epilogue(unsigned taddr, unsigned stage, const CUtensorMap *tm_out, int n0,
                                             const float *__restrict__ bias, int relu, int b, int x0, int y0, int m,
                                             bool leader, int &blk)
{
    constexpr int SB = out_block(BN), CH = SB / 8;  // channels per block, 16-byte chunks per row
    constexpr unsigned RB = SB * 2, BUF = 128u * RB;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += SB, blk++) {
        unsigned r[SB];
#pragma unroll
        for (int c = 0; c < SB; c += 16) tmem_ld16_nw(taddr + (unsigned)(c0 + c), r + c);
        float4 bv[SB / 4];
#pragma unroll
        for (int k = 0; k < SB / 4; k++)
            bv[k] = bias ? __ldg((const float4 *)(bias + n0 + c0) + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        tmem_wait_ld();
        if (leader) bulk_wait_read1();
        epi_bar();  // the buffer of this block is free
        const unsigned buf = stage + (unsigned)(blk & 1) * BUF + (unsigned)m * RB;
#pragma unroll
        for (int j = 0; j < CH; j++) {
            const float *bj = reinterpret_cast<const float *>(bv) + 8 * j;
            unsigned w[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                float v0 = __uint_as_float(r[8 * j + 2 * e]) + bj[2 * e];
                float v1 = __uint_as_float(r[8 * j + 2 * e + 1]) + bj[2 * e + 1];
                if (relu) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                w[e] = *reinterpret_cast<const unsigned *>(&h);
            }
            const unsigned sw = SB == 64 ? (unsigned)(m & 7) : (unsigned)((m >> 1) & 3);
            const unsigned a = buf + (((unsigned)j ^ sw) << 4);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                         "r"(w[3])
                         : "memory");
        }
        fence_proxy_async();
        epi_bar();  // the block is staged
        if (leader) {
            tma_store_4d(tm_out, stage + (unsigned)(blk & 1) * BUF, n0 + c0, x0, y0, b);
            bulk_commit();
        }
    }
}

// out[b, y, x, out_c0 + co] = act(bias[co] + sum over taps, ci of
// in[b, y + dy, x + dx, ci] W[co][tap][ci]), zero outside the image.
// A work item is MT consecutive pixel patches (M tiles) of one output-channel
// tile: each stage holds the MT input boxes and one weight box, which the MT
// accumulators share, so MT = 2 reads the weights once per two patches. A
// patch past the last one (odd count) is read as zeros (its boxes lie
// outside the tensor) and not stored.
template <int BN, int KC, int MT>
__global__ void __launch_bounds__(FW_THREADS, 1)
k_conv_fwd_tc(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_w,
              const __grid_constant__ CUtensorMap tm_out, const float *__restrict__ bias, bf16 *__restrict__ out, int out_cs, int out_c0, int Cout, int Cin,
              int B, int H, int Wd, int taps, int relu, int bx, int by, int ntx, int nty)
{
    using C = FwdCfg<BN, KC, MT>;
    constexpr int S = C::S;
    constexpr int ACC = MT * BN;  // TMEM columns of one work item's accumulators
    extern __shared__ unsigned char fw_smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S], tfull[2], tempty[2], drain;
    __shared__ unsigned tbase;
    __shared__ int s_abort, s_eok;
    volatile int *abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_abort = 0;
    const unsigned ring = (cv_smem_u32(fw_smem) + 1023u) & ~1023u;
    if (warp == 0) tmem_alloc(&tbase, 2 * ACC);
    if (tid == 32) {
        for (int s = 0; s < S; s++) {
            mbar_init(cv_smem_u32(&full[s]), 1);
            mbar_init(cv_smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(cv_smem_u32(&tfull[a]), 1);
            mbar_init(cv_smem_u32(&tempty[a]), 4);  // one arrival per epilogue warp
        }
        mbar_init(cv_smem_u32(&drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tbase;
    const unsigned ostage = ring + (unsigned)S * C::STAGE;  // output staging (1024-byte aligned)
    const int kch = Cin / KC, KT = taps * kch;
    const int nmt = ntx * nty * B, nmi = (nmt + MT - 1) / MT;  // patches, work items per channel tile
    const int nnt = Cout / BN, ntiles = nmi * nnt;
    const int limit = g_conv_wait_limit;
    int issued = 0;  // warp 0, lane 0: stage fills issued

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch(&tm_in);
            tma_prefetch(&tm_w);
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int mi = t / nnt, n0 = (t - mi * nnt) * BN;
                int b[MT], y0[MT], x0[MT];
#pragma unroll
                for (int j = 0; j < MT; j++) patch_of(mi * MT + j, ntx, nty, bx, by, b[j], y0[j], x0[j]);
                for (int tap = 0; tap < taps && ok; tap++) {
                    const int dy = taps == 9 ? tap / 3 - 1 : 0, dx = taps == 9 ? tap % 3 - 1 : 0;
                    for (int ci0 = 0; ci0 < Cin; ci0 += KC) {
                        const int s = issued % S, u = issued / S;
                        if (u > 0 && !mbar_wait(cv_smem_u32(&empty[s]), (unsigned)((u - 1) & 1), limit, abort)) {
                            ok = false;
                            break;
                        }
                        const unsigned fb = cv_smem_u32(&full[s]), a = ring + (unsigned)s * C::STAGE;
                        mbar_expect_tx(fb, C::STAGE);
#pragma unroll
                        for (int j = 0; j < MT; j++)
                            tma_load_4d(a + (unsigned)j * C::A_BYTES, &tm_in, fb, ci0, x0[j] + dx, y0[j] + dy, b[j]);
                        tma_load_2d(a + MT * C::A_BYTES, &tm_w, fb, tap * Cin + ci0, n0);
                        issued++;
                    }
                }
            }
            if (!ok) give_up(abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const unsigned id = idesc_bf16(128, BN, false);
            const uint64_t desc0 = sdesc_sw(ring, 16, 8 * C::ROW, C::SW);
            bool ok = true;
            int it = 0, tc = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, tc++) {
                const int acc = tc & 1, ua = tc >> 1;
                if (ua > 0 && !mbar_wait(cv_smem_u32(&tempty[acc]), (unsigned)((ua - 1) & 1), limit, abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned d = tmem + (unsigned)(acc * ACC);
                for (int kt = 0; kt < KT; kt++, it++) {
                    const int s = it % S, u = it / S;
                    if (!mbar_wait(cv_smem_u32(&full[s]), (unsigned)(u & 1), limit, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = desc0 + (uint64_t)(((unsigned)s * C::STAGE) >> 4);
                    const uint64_t bd = ad + ((MT * C::A_BYTES) >> 4);
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ks++)
#pragma unroll
                        for (int j = 0; j < MT; j++)
                            mma_bf16(d + (unsigned)(j * BN), ad + ((j * C::A_BYTES) >> 4) + 2 * ks, bd + 2 * ks, id,
                                     (kt > 0 || ks > 0) ? 1u : 0u);
                    mma_commit(cv_smem_u32(&empty[s]));  // the stage is free once these MMAs are done
                }
                if (!ok) break;
                mma_commit(cv_smem_u32(&tfull[acc]));  // the tile's accumulator is complete
            }
            if (!ok) give_up(abort);
        }
    } else {
        // warps 2-5: TMEM lane quarter warp % 4 holds tile rows 32 (warp % 4) + lane
        const int q = warp & 3, m = 32 * q + lane;
        const bool leader = warp == 2 && lane == 0;  // issues the group's TMA stores
        int tc = 0, blk = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, tc++) {
            const int acc = tc & 1, ua = tc >> 1;
            // one wait for the four warps, so that all of them take the same
            // branch (the epilogue's named barriers need all 128 threads)
            if (leader) s_eok = mbar_wait(cv_smem_u32(&tfull[acc]), (unsigned)(ua & 1), limit, abort) ? 1 : 0;
            epi_bar();
            if (!*(volatile int *)&s_eok) {
                if (leader) give_up(abort);
                break;
            }
            tc_fence_after();
            const int mi = t / nnt, n0 = (t - mi * nnt) * BN;
#pragma unroll 1
            for (int j = 0; j < MT && mi * MT + j < nmt; j++) {  // uniform over the 128 threads
                int b, y0, x0;
                patch_of(mi * MT + j, ntx, nty, bx, by, b, y0, x0);
                fwd_epilogue<BN>(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(acc * ACC + j * BN), ostage, &tm_out,
                                 n0, bias, relu, b, x0, y0, m, leader, blk);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(cv_smem_u32(&tempty[acc]));  // the accumulator may be overwritten
        }
        if (leader) bulk_wait_all();  // the output stores are done before the CTA ends
    }
    __syncthreads();
    if (s_abort) {
        // gave up: no copy into shared memory and no MMA into tensor memory
        // may still be running when the CTA frees them
        if (tid == 0)
            for (int j = issued > S ? issued - S : 0; j < issued; j++)
                mbar_wait_plain(cv_smem_u32(&full[j % S]), (unsigned)((j / S) & 1), TC_WAIT);
        if (tid == 32) {
            mma_commit(cv_smem_u32(&drain));  // arrives once every MMA issued so far is done
            mbar_wait_plain(cv_smem_u32(&drain), 0u, TC_WAIT);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tmem_free(tmem, 2 * ACC);
    }
}

// -------------------------------------------- conv forward, halo variant
//
// For 3x3 convolutions whose weight block (BN output channels x 9 taps x
// Cin) fits in shared memory beside the ring: the CTA loads it once and
// keeps it; per K chunk of KC input channels a stage holds the tile's input
// with its halo as three copies, one per horizontal tap offset dx, each
// bx x (by + 2) pixels from (x0 + dx, y0 - 1). The MMAs of tap (dy, dx) read
// the copy dx from row (dy + 1) bx on: pixel (c, r) of the tile is then row
// (r + dy + 1) bx + c, and as bx is a multiple of 8 every operand starts on
// a swizzle-pattern boundary. A stage is 3 bx (by + 2) rows instead of the
// 9 x 128 rows of one copy per tap. CTA i serves output-channel tile
// i % nnt and every (grid / nnt)-th pixel patch.

constexpr int HL_MAXST = 4;

template <int BN, int KC>
__global__ void __launch_bounds__(FW_THREADS, 1)
k_conv_fwd_halo(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_w,
                const __grid_constant__ CUtensorMap tm_out, const float *__restrict__ bias, bf16 *__restrict__ out, int out_cs, int out_c0, int Cout, int Cin,
                int B, int H, int Wd, int relu, int bx, int by, int ntx, int nty, int S)
{
    constexpr unsigned ROW = KC * 2, SW = KC == 64 ? 2u : 4u, WBLK = BN * ROW;
    extern __shared__ unsigned char hl_smem[];
    __shared__ __align__(8) uint64_t full[HL_MAXST], empty[HL_MAXST], tfull[2], tempty[2], wfull, drain;
    __shared__ unsigned tbase;
    __shared__ int s_abort, s_eok;
    volatile int *abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_abort = 0;
    const int nch = Cin / KC;
    const unsigned wres = (cv_smem_u32(hl_smem) + 1023u) & ~1023u;  // resident weights
    const unsigned dxbuf = (unsigned)(bx * (by + 2)) * ROW, abytes = 3 * dxbuf;
    const unsigned ring = wres + 9u * (unsigned)nch * WBLK;
    const unsigned ostage = ring + (unsigned)S * abytes;  // output staging (1024-byte aligned)
    if (warp == 0) tmem_alloc(&tbase, 2 * BN);
    if (tid == 32) {
        for (int q = 0; q < S; q++) {
            mbar_init(cv_smem_u32(&full[q]), 1);
            mbar_init(cv_smem_u32(&empty[q]), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(cv_smem_u32(&tfull[a]), 1);
            mbar_init(cv_smem_u32(&tempty[a]), 4);
        }
        mbar_init(cv_smem_u32(&wfull), 1);
        mbar_init(cv_smem_u32(&drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tbase;
    const int nnt = Cout / BN, n0 = (blockIdx.x % nnt) * BN;
    const int mt0 = blockIdx.x / nnt, mstep = gridDim.x / nnt, nmt = ntx * nty * B;
    const int limit = g_conv_wait_limit;
    int issued = 0;

    if (warp == 0) {
        if (lane == 0) {
            tma_prefetch(&tm_in);
            tma_prefetch(&tm_w);
            const unsigned wb = cv_smem_u32(&wfull);
            mbar_expect_tx(wb, 9u * (unsigned)nch * WBLK);
            for (int tap = 0; tap < 9; tap++)
                for (int ch = 0; ch < nch; ch++)
                    tma_load_2d(wres + (unsigned)(tap * nch + ch) * WBLK, &tm_w, wb, tap * Cin + ch * KC, n0);
            bool ok = true;
            for (int mt = mt0; mt < nmt && ok; mt += mstep) {
                int b, y0, x0;
                patch_of(mt, ntx, nty, bx, by, b, y0, x0);
                for (int ch = 0; ch < nch; ch++) {
                    const int s = issued % S, u = issued / S;
                    if (u > 0 && !mbar_wait(cv_smem_u32(&empty[s]), (unsigned)((u - 1) & 1), limit, abort)) {
                        ok = false;
                        break;
                    }
                    const unsigned fb = cv_smem_u32(&full[s]), a = ring + (unsigned)s * abytes;
                    mbar_expect_tx(fb, abytes);
#pragma unroll
                    for (int dx = -1; dx <= 1; dx++)
                        tma_load_4d(a + (unsigned)(dx + 1) * dxbuf, &tm_in, fb, ch * KC, x0 + dx, y0 - 1, b);
                    issued++;
                }
            }
            if (!ok) give_up(abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const unsigned id = idesc_bf16(128, BN, false);
            const uint64_t adesc0 = sdesc_sw(ring, 16, 8 * ROW, SW), wdesc0 = sdesc_sw(wres, 16, 8 * ROW, SW);
            const unsigned dxq = dxbuf >> 4, rq = ((unsigned)bx * ROW) >> 4;  // tap offsets, 16-byte units
            const unsigned wq = WBLK >> 4, tq = (unsigned)nch * wq;
            bool ok = mbar_wait(cv_smem_u32(&wfull), 0u, limit, abort);
            int it = 0, tc = 0;
            for (int mt = mt0; mt < nmt && ok; mt += mstep, tc++) {
                const int acc = tc & 1, ua = tc >> 1;
                if (ua > 0 && !mbar_wait(cv_smem_u32(&tempty[acc]), (unsigned)((ua - 1) & 1), limit, abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned d = tmem + (unsigned)(acc * BN);
                for (int ch = 0; ch < nch; ch++, it++) {
                    const int s = it % S, u = it / S;
                    if (!mbar_wait(cv_smem_u32(&full[s]), (unsigned)(u & 1), limit, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // descriptors as 64-bit values; offsets add to the address
                    // field (16-byte units, addresses below 256 KB)
                    const uint64_t ad = adesc0 + (uint64_t)(((unsigned)s * abytes) >> 4);
                    const uint64_t bd = wdesc0 + (uint64_t)(ch * wq);
#pragma unroll
                    for (int tap = 0; tap < 9; tap++) {  // tap = (dy + 1) * 3 + dx + 1
                        const uint64_t at = ad + (uint64_t)((tap % 3) * dxq + (tap / 3) * rq);
                        const uint64_t bt = bd + (uint64_t)(tap * tq);
#pragma unroll
                        for (int ks = 0; ks < KC / 16; ks++)
                            mma_bf16(d, at + 2 * ks, bt + 2 * ks, id, (tap > 0 || ks > 0 || ch > 0) ? 1u : 0u);
                    }
                    mma_commit(cv_smem_u32(&empty[s]));
                }
                if (!ok) break;
                mma_commit(cv_smem_u32(&tfull[acc]));
            }
            if (!ok) give_up(abort);
        }
    } else {
        const int q = warp & 3, m = 32 * q + lane;
        const bool leader = warp == 2 && lane == 0;  // issues the group's TMA stores
        int tc = 0, blk = 0;
        for (int mt = mt0; mt < nmt; mt += mstep, tc++) {
            const int acc = tc & 1, ua = tc >> 1;
            // one wait for the four warps, so that all of them take the same
            // branch (the epilogue's named barriers need all 128 threads)
            if (leader) s_eok = mbar_wait(cv_smem_u32(&tfull[acc]), (unsigned)(ua & 1), limit, abort) ? 1 : 0;
            epi_bar();
            if (!*(volatile int *)&s_eok) {
                if (leader) give_up(abort);
                break;
            }
            tc_fence_after();
            int b, y0, x0;
            patch_of(mt, ntx, nty, bx, by, b, y0, x0);
            fwd_epilogue<BN>(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(acc * BN), ostage, &tm_out, n0, bias,
                             relu, b, x0, y0, m, leader, blk);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(cv_smem_u32(&tempty[acc]));
        }
        if (leader) bulk_wait_all();  // the output stores are done before the CTA ends
    }
    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            mbar_wait_plain(cv_smem_u32(&wfull), 0u, TC_WAIT);
            for (int j = issued > S ? issued - S : 0; j < issued; j++)
                mbar_wait_plain(cv_smem_u32(&full[j % S]), (unsigned)((j / S) & 1), TC_WAIT);
        }
        if (tid == 32) {
            mma_commit(cv_smem_u32(&drain));
            mbar_wait_plain(cv_smem_u32(&drain), 0u, TC_WAIT);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tmem_free(tmem, 2 * BN);
    }
}

// ------------------------------------------------------------ conv wgrad

constexpr int WG_THREADS = 128;  // warp 0 copies, warp 1 MMAs, all four the epilogue
constexpr int WG_STAGES = 4;
constexpr int WG_PIX = 64;  // pixels (K) per stage

template <int BN, int KCA, int KCB>
struct WgdCfg {
    static constexpr unsigned A_ROW = KCA * 2, B_ROW = KCB * 2;                // bytes per pixel row of a box
    static constexpr unsigned A_BOX = WG_PIX * A_ROW, B_BOX = WG_PIX * B_ROW;  // one TMA box
    static constexpr unsigned A_BYTES = 128 * WG_PIX * 2, B_BYTES = BN * WG_PIX * 2;
    static constexpr unsigned STAGE = A_BYTES + B_BYTES;
    static constexpr unsigned SMEM = WG_STAGES * STAGE + 1024;
    static constexpr unsigned A_SW = KCA == 64 ? 2u : 4u, B_SW = KCB == 64 ? 2u : 4u;
};

// part[split][co][tap * Cin + ci] = sum over the split's pixel patches of
// in[p shifted by tap][ci] grad[p][co] (zero outside the image). Tile: 128
// rows (tap, ci) from blockIdx.x, BN output channels from blockIdx.y; the
// split's patches from blockIdx.z.
template <int BN, int KCA, int KCB>
__global__ void __launch_bounds__(WG_THREADS, 1)
k_conv_wgrad_tc(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_g, int Cout,
                int Cin, int taps, int bx, int by, int ntx, int nty, int npatch, int per_split,
                float *__restrict__ part)
{
    using C = WgdCfg<BN, KCA, KCB>;
    constexpr int S = WG_STAGES;
    extern __shared__ unsigned char wg_smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S], done, drain;
    __shared__ unsigned tbase;
    __shared__ int s_abort;
    volatile int *abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_abort = 0;
    const unsigned ring = (cv_smem_u32(wg_smem) + 1023u) & ~1023u;
    const int K = taps * Cin, kk0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int p0 = blockIdx.z * per_split, p1 = min(npatch, p0 + per_split), KT = p1 > p0 ? p1 - p0 : 0;
    const int nA = min(128, K - kk0) / KCA;  // boxes holding rows of this tile (KCA divides Cin)
    if (warp == 0) tmem_alloc(&tbase, BN);
    if (tid == 32) {
        for (int s = 0; s < S; s++) {
            mbar_init(cv_smem_u32(&full[s]), 1);
            mbar_init(cv_smem_u32(&empty[s]), 1);
        }
        mbar_init(cv_smem_u32(&done), 1);
        mbar_init(cv_smem_u32(&drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tbase;
    const int limit = g_conv_wait_limit;
    int issued = 0;

    if (tid == 0) {
        tma_prefetch(&tm_in);
        tma_prefetch(&tm_g);
        const unsigned bytes = (unsigned)nA * C::A_BOX + C::B_BYTES;
        // the tile's A boxes: input channel chunk and tap shift, the same for
        // every patch (at most 128 / KCA of them)
        int bci[128 / KCA], bdx[128 / KCA], bdy[128 / KCA];
#pragma unroll
        for (int r = 0; r < 128 / KCA; r++) {
            const int kk = kk0 + r * KCA, tap = kk / Cin;
            bci[r] = kk - tap * Cin;
            bdy[r] = taps == 9 ? tap / 3 - 1 : 0;
            bdx[r] = taps == 9 ? tap % 3 - 1 : 0;
        }
        int b, y0, x0;  // the current patch, advanced in patch order
        patch_of(p0, ntx, nty, bx, by, b, y0, x0);
        const int xe = ntx * bx, ye = nty * by;
        for (int kt = 0; kt < KT; kt++) {
            const int s = kt % S, u = kt / S;
            if (u > 0 && !mbar_wait(cv_smem_u32(&empty[s]), (unsigned)((u - 1) & 1), limit, abort)) {
                give_up(abort);
                break;
            }
            const unsigned fb = cv_smem_u32(&full[s]), a = ring + (unsigned)s * C::STAGE;
            mbar_expect_tx(fb, bytes);
#pragma unroll
            for (int r = 0; r < 128 / KCA; r++)
                if (r < nA) tma_load_4d(a + (unsigned)r * C::A_BOX, &tm_in, fb, bci[r], x0 + bdx[r], y0 + bdy[r], b);
#pragma unroll
            for (int j = 0; j < BN / KCB; j++)
                tma_load_4d(a + C::A_BYTES + (unsigned)j * C::B_BOX, &tm_g, fb, n0 + j * KCB, x0, y0, b);
            issued++;
            x0 += bx;
            if (x0 >= xe) {
                x0 = 0;
                y0 += by;
                if (y0 >= ye) {
                    y0 = 0;
                    b++;
                }
            }
        }
    } else if (tid == 32) {
        const unsigned id = idesc_bf16(128, BN, true);
        const uint64_t adesc0 = sdesc_sw(ring, C::A_BOX, 8 * C::A_ROW, C::A_SW);
        const uint64_t bdesc0 = sdesc_sw(ring + C::A_BYTES, C::B_BOX, 8 * C::B_ROW, C::B_SW);
        bool ok = true;
        for (int kt = 0; kt < KT; kt++) {
            const int s = kt % S, u = kt / S;
            if (!mbar_wait(cv_smem_u32(&full[s]), (unsigned)(u & 1), limit, abort)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint64_t ad = adesc0 + (uint64_t)(((unsigned)s * C::STAGE) >> 4);
            const uint64_t bd = bdesc0 + (uint64_t)(((unsigned)s * C::STAGE) >> 4);
#pragma unroll
            for (int ks = 0; ks < WG_PIX / 16; ks++)  // 16 pixels = two 8-row groups per MMA
                mma_bf16(tmem, ad + ks * (C::A_ROW), bd + ks * (C::B_ROW), id, (kt > 0 || ks > 0) ? 1u : 0u);
            mma_commit(cv_smem_u32(&empty[s]));
        }
        if (ok) mma_commit(cv_smem_u32(&done));
        else give_up(abort);
    }
    __syncwarp();
    // epilogue: warp w holds rows 32 w + lane of the tile
    int ok = 1;
    if (lane == 0) {
        ok = !s_abort;
        if (ok && KT > 0) {
            ok = mbar_wait(cv_smem_u32(&done), 0u, limit, abort);
            if (!ok) give_up(abort);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
        const int kk = kk0 + 32 * warp + lane;
        float *dst = part + ((int64_t)blockIdx.z * Cout + n0) * K + kk;
        if (KT == 0) {  // an empty split contributes zeros
            if (kk < K)
                for (int c = 0; c < BN; c++) dst[(int64_t)c * K] = 0.0f;
        } else {
            tc_fence_after();
            for (int c0 = 0; c0 < BN; c0 += 16) {
                unsigned r[16];
                tmem_ld16(tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0, r);
                if (kk < K)
#pragma unroll
                    for (int j = 0; j < 16; j++) dst[(int64_t)(c0 + j) * K] = __uint_as_float(r[j]);
            }
        }
    }
    __syncthreads();
    if (s_abort) {
        if (tid == 0)
            for (int j = issued > S ? issued - S : 0; j < issued; j++)
                mbar_wait_plain(cv_smem_u32(&full[j % S]), (unsigned)((j / S) & 1), TC_WAIT);
        if (tid == 32) {
            mma_commit(cv_smem_u32(&drain));
            mbar_wait_plain(cv_smem_u32(&drain), 0u, TC_WAIT);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tmem_free(tmem, BN);
    }
}

// out[i] = sum over splits s (in order) of part[s][i]; eight loads in
// flight, added in split order
__global__ void k_conv_fold(const float *__restrict__ part, int64_t n, int splits, float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    int q = 0;
    for (; q + 8 <= splits; q += 8) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; j++) v[j] = part[(int64_t)(q + j) * n + i];
#pragma unroll
        for (int j = 0; j < 8; j++) s += v[j];
    }
    for (; q < splits; q++) s += part[(int64_t)q * n + i];
    out[i] = s;
}

// Per-split column sums of grad (the bias gradient): part[split][c]. The
// block's 256 threads take channel c = t % C and every (256 / C)-th pixel
// of the split from t / C on; the partial sums are added in that order.
__global__ void __launch_bounds__(256) k_conv_bias_part(const bf16 *__restrict__ grad, int g_cs, int C, int M,
                                                        int pix_per_split, float *__restrict__ part)
{
    __shared__ float red[256];
    const int p0 = blockIdx.x * pix_per_split, p1 = min(M, p0 + pix_per_split);
    const int t = threadIdx.x;
    const int lanes = C < 256 ? 256 / C : 1;  // threads per channel
    for (int cb = 0; cb < C; cb += 256 / lanes) {
        const int c = cb + t % (256 / lanes), sub = t / (256 / lanes);
        float s = 0.0f;
        if (c < C)
            for (int p = p0 + sub; p < p1; p += lanes) s += __bfloat162float(grad[(int64_t)p * g_cs + c]);
        red[t] = s;
        __syncthreads();
        if (sub == 0 && c < C) {
            float r = red[t];
            for (int j = 1; j < lanes; j++) r += red[t + j * (256 / lanes)];
            part[(int64_t)blockIdx.x * C + c] = r;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host

static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// NHWC activation (C channels of cs-wide pixel rows starting at base) as a
// 4D map (channel, x, y, image); box (kc channels, bx, by, 1), swizzled to
// the box's row width, zeros outside the tensor.
static cudaError_t act_map(CUtensorMap *m, const bf16 *base, int C, int cs, int B, int H, int W, int kc, int bx,
                           int by)
{
    auto enc = tmap_encoder();
    if (!enc) return cudaErrorNotSupported;
    if ((uintptr_t)base % 16) return cudaErrorMisalignedAddress;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {(cuuint64_t)cs * 2, (cuuint64_t)W * cs * 2, (cuuint64_t)H * W * cs * 2};
    const cuuint32_t box[4] = {(cuuint32_t)kc, (cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)base, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE,
                           kc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// weights [Cout][K] (K = taps x Cin, K-major rows) as a 2D map; box (kc, bn)
static cudaError_t weight_map(CUtensorMap *m, const bf16 *W, int K, int Cout, int kc, int bn)
{
    auto enc = tmap_encoder();
    if (!enc) return cudaErrorNotSupported;
    if ((uintptr_t)W % 16) return cudaErrorMisalignedAddress;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)Cout};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kc, (cuuint32_t)bn};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)W, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE,
                           kc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int sm_count()
{
    static int n = 0;
    if (!n) {
        int d = 0;
        if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) !=
                                                    cudaSuccess || n <= 0)
            n = 1;
    }
    return n;
}

// patch of `pix` pixels (a power of two): bx = the smallest power of two
// >= W (at most pix), by = pix / bx
static void patch_shape(int W, int pix, int &bx, int &by)
{
    bx = 1;
    while (bx < W && bx < pix) bx *= 2;
    by = pix / bx;
}

// largest of 256, 128, 64, 32 that divides c (c a multiple of 32)
static int tile_n(int c) { return c % 256 == 0 ? 256 : c % 128 == 0 ? 128 : c % 64 == 0 ? 64 : 32; }

template <typename Kern>
static cudaError_t smem_attr(Kern k, unsigned bytes, bool &done)
{
    if (done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done = true;
    return e;
}

template <int BN, int KC, int MT>
static cudaError_t launch_fwd_mt(const CUtensorMap &ti, const CUtensorMap &tw, const CUtensorMap &to,
                                 const float *bias, bf16 *out, int out_cs, int out_c0, int Cout, int Cin, int B, int H,
                                 int Wd, int taps, int relu, int bx, int by, int ntx, int nty, cudaStream_t st)
{
    using Cfg = FwdCfg<BN, KC, MT>;
    static bool attr = false;
    const cudaError_t e = smem_attr(k_conv_fwd_tc<BN, KC, MT>, Cfg::SMEM, attr);
    if (e != cudaSuccess) return e;
    const int64_t nmt = (int64_t)ntx * nty * B, items = (nmt + MT - 1) / MT * (Cout / BN);
    const int grid = (int)std::min<int64_t>(items, sm_count());
    k_conv_fwd_tc<BN, KC, MT><<<grid, FW_THREADS, Cfg::SMEM, st>>>(ti, tw, to, bias, out, out_cs, out_c0, Cout, Cin,
                                                                    B, H, Wd, taps, relu, bx, by, ntx, nty);
    return cudaGetLastError();
}

// Two patches per work item (the weight boxes shared) once there are more
// patches than SMs (output tiles up to 128 channels: two double-buffered
// accumulators fit in tensor memory); one below that, where halving the
// work items would idle SMs.
template <int BN, int KC>
static cudaError_t launch_fwd(const CUtensorMap &ti, const CUtensorMap &tw, const float *bias, bf16 *out, int out_cs,
                              int out_c0, int Cout, int Cin, int B, int H, int Wd, int taps, int relu, int bx, int by,
                              int ntx, int nty, cudaStream_t st)
{
    CUtensorMap to;  // output: blocks of out_block(BN) channels x the tile's patch
    const cudaError_t e = act_map(&to, out + out_c0, Cout, out_cs, B, H, Wd, out_block(BN), bx, by);
    if (e != cudaSuccess) return e;
    const int64_t nmt = (int64_t)ntx * nty * B;
    if constexpr (BN <= 128) {
        if (nmt * (Cout / BN) > sm_count())
            return launch_fwd_mt<BN, KC, 2>(ti, tw, to, bias, out, out_cs, out_c0, Cout, Cin, B, H, Wd, taps, relu, bx,
                                            by, ntx, nty, st);
    }
    return launch_fwd_mt<BN, KC, 1>(ti, tw, to, bias, out, out_cs, out_c0, Cout, Cin, B, H, Wd, taps, relu, bx, by,
                                    ntx, nty, st);
}

// Shared memory of the halo variant: resident weights + stages (0: does not
// fit with two stages).
static unsigned halo_smem(int Cin, int BN, int KC, int bx, int by, int &S)
{
    // less alignment slack, static barriers and the output staging
    const unsigned budget = 227u * 1024u - 1024u - 256u - out_staging(BN);
    const unsigned wbytes = 9u * (unsigned)(Cin / KC) * (unsigned)(BN * KC * 2);
    const unsigned abytes = 3u * (unsigned)(bx * (by + 2) * KC * 2);
    if (wbytes + 2 * abytes > budget) return 0;
    S = (int)std::min<unsigned>(HL_MAXST, (budget - wbytes) / abytes);
    return 1024u + wbytes + (unsigned)S * abytes + out_staging(BN);
}

template <int BN, int KC>
static cudaError_t launch_halo(const bf16 *in, int in_cs, int in_c0, int Cin, const bf16 *W, const float *bias,
                               bf16 *out, int out_cs, int out_c0, int Cout, int B, int H, int Wd, int relu, int bx,
                               int by, unsigned smem, int S, cudaStream_t st)
{
    static unsigned attr = 0;  // per instance: the largest dynamic shared memory configured
    if (smem > attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_conv_fwd_halo<BN, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    const int ntx = (Wd + bx - 1) / bx, nty = (H + by - 1) / by;
    const int64_t nmt = (int64_t)ntx * nty * B;
    const int nnt = Cout / BN;
    const int per = (int)std::min<int64_t>(nmt, std::max(1, sm_count() / nnt));
    CUtensorMap ti, tw, to;
    cudaError_t e = act_map(&ti, in + in_c0, Cin, in_cs, B, H, Wd, KC, bx, by + 2);
    if (e == cudaSuccess) e = weight_map(&tw, W, 9 * Cin, Cout, KC, BN);
    if (e == cudaSuccess) e = act_map(&to, out + out_c0, Cout, out_cs, B, H, Wd, out_block(BN), bx, by);
    if (e != cudaSuccess) return e;
    k_conv_fwd_halo<BN, KC><<<nnt * per, FW_THREADS, smem, st>>>(ti, tw, to, bias, out, out_cs, out_c0, Cout, Cin, B,
                                                                 H, Wd, relu, bx, by, ntx, nty, S);
    return cudaGetLastError();
}

cudaError_t conv_fwd(const bf16 *in, int in_cs, int in_c0, int Cin, const bf16 *W, const float *bias, bf16 *out,
                     int out_cs, int out_c0, int Cout, int B, int H, int Wd, int taps, bool relu, cudaStream_t st)
{
    if (Cin % 32 || Cout % 32 || (in_cs | in_c0 | out_cs | out_c0) % 8 || (taps != 1 && taps != 9))
        return cudaErrorInvalidValue;
    if ((uintptr_t)bias % 16) return cudaErrorInvalidValue;  // read as float4
    if ((int64_t)B * H * Wd == 0) return cudaSuccess;
    const int KC = Cin % 64 == 0 ? 64 : 32, BN = tile_n(Cout);
    if (taps == 9 && BN <= 64) {  // the halo variant where its weight block fits
        const int hbx = Wd > 8 ? 16 : 8, hby = 128 / hbx;
        int S = 0;
        const unsigned smem = halo_smem(Cin, BN, KC, hbx, hby, S);
        if (smem && (int64_t)((Wd + hbx - 1) / hbx) * ((H + hby - 1) / hby) * B <= INT32_MAX) {
            const int r = relu ? 1 : 0;
            if (BN == 64 && KC == 64)
                return launch_halo<64, 64>(in, in_cs, in_c0, Cin, W, bias, out, out_cs, out_c0, Cout, B, H, Wd, r, hbx,
                                           hby, smem, S, st);
            if (BN == 32 && KC == 64)
                return launch_halo<32, 64>(in, in_cs, in_c0, Cin, W, bias, out, out_cs, out_c0, Cout, B, H, Wd, r, hbx,
                                           hby, smem, S, st);
            if (BN == 64 && KC == 32)
                return launch_halo<64, 32>(in, in_cs, in_c0, Cin, W, bias, out, out_cs, out_c0, Cout, B, H, Wd, r, hbx,
                                           hby, smem, S, st);
            return launch_halo<32, 32>(in, in_cs, in_c0, Cin, W, bias, out, out_cs, out_c0, Cout, B, H, Wd, r, hbx,
                                       hby, smem, S, st);
        }
    }
    int bx, by;
    patch_shape(Wd, 128, bx, by);
    const int ntx = (Wd + bx - 1) / bx, nty = (H + by - 1) / by;
    if ((int64_t)ntx * nty * B * (Cout / BN) > INT32_MAX) return cudaErrorInvalidValue;
    CUtensorMap ti, tw;
    cudaError_t e = act_map(&ti, in + in_c0, Cin, in_cs, B, H, Wd, KC, bx, by);
    if (e == cudaSuccess) e = weight_map(&tw, W, taps * Cin, Cout, KC, BN);
    if (e != cudaSuccess) return e;
#define FWD_CASE(bn, kc)                                                                                         \
    if (BN == bn && KC == kc)                                                                                    \
        return launch_fwd<bn, kc>(ti, tw, bias, out, out_cs, out_c0, Cout, Cin, B, H, Wd, taps, relu ? 1 : 0, bx, \
                                  by, ntx, nty, st);
    FWD_CASE(256, 64)
    FWD_CASE(128, 64)
    FWD_CASE(64, 64)
    FWD_CASE(32, 64)
    FWD_CASE(256, 32)
    FWD_CASE(128, 32)
    FWD_CASE(64, 32)
    FWD_CASE(32, 32)
#undef FWD_CASE
    return cudaErrorInvalidValue;
}

template <int BN, int KCA, int KCB>
static cudaError_t launch_wgrad(dim3 grid, const CUtensorMap &ti, const CUtensorMap &tg, int Cout, int Cin, int taps,
                                int bx, int by, int ntx, int nty, int npatch, int per_split, float *part,
                                cudaStream_t st)
{
    static bool attr = false;
    cudaError_t e = smem_attr(k_conv_wgrad_tc<BN, KCA, KCB>, WgdCfg<BN, KCA, KCB>::SMEM, attr);
    if (e != cudaSuccess) return e;
    k_conv_wgrad_tc<BN, KCA, KCB><<<grid, WG_THREADS, WgdCfg<BN, KCA, KCB>::SMEM, st>>>(
        ti, tg, Cout, Cin, taps, bx, by, ntx, nty, npatch, per_split, part);
    return cudaGetLastError();
}

cudaError_t conv_wgrad(const bf16 *grad, int g_cs, int Cout, const bf16 *in, int in_cs, int in_c0, int Cin, int B,
                       int H, int Wd, int taps, float *dW, float *db, float *scratch, size_t scratch_floats,
                       cudaStream_t st)
{
    if (Cin % 32 || Cout % 32 || (g_cs | in_cs | in_c0) % 8 || (taps != 1 && taps != 9)) return cudaErrorInvalidValue;
    const int64_t M = (int64_t)B * H * Wd;
    const int64_t K = (int64_t)taps * Cin, per = (int64_t)Cout * K;
    if ((size_t)per > scratch_floats) return cudaErrorMemoryAllocation;
    if (M == 0) {
        cudaError_t e = cudaMemsetAsync(dW, 0, per * sizeof(float), st);
        if (e == cudaSuccess && db) e = cudaMemsetAsync(db, 0, Cout * sizeof(float), st);
        return e;
    }
    const int KCA = Cin % 64 == 0 ? 64 : 32, BN = tile_n(Cout), KCB = BN % 64 == 0 ? 64 : 32;
    int bx, by;
    patch_shape(Wd, WG_PIX, bx, by);
    const int ntx = (Wd + bx - 1) / bx, nty = (H + by - 1) / by;
    const int64_t npatch64 = (int64_t)ntx * nty * B;
    if (npatch64 > INT32_MAX) return cudaErrorInvalidValue;
    const int npatch = (int)npatch64;
    // pixel splits: enough CTAs to fill the SMs (two per SM where shared
    // memory allows), bounded by the scratch for the partial tiles
    const int mt = (int)((K + 127) / 128), nt = Cout / BN;
    const bool two = (BN == 32 ? WgdCfg<32, 64, 32>::SMEM : BN == 64 ? WgdCfg<64, 64, 64>::SMEM : 1u << 20) <= 113 * 1024;
    const int64_t target = (int64_t)sm_count() * (two ? 2 : 1);
    int64_t splits = std::max<int64_t>(1, (target + mt * nt - 1) / (mt * nt));
    splits = std::min<int64_t>(splits, npatch);
    while (splits > 1 && (size_t)(splits * per) > scratch_floats) splits = (splits + 1) / 2;
    if ((size_t)(splits * per) > scratch_floats) splits = 1;
    const int per_split = (int)((npatch + splits - 1) / splits);
    splits = (npatch + per_split - 1) / per_split;
    CUtensorMap ti, tg;
    cudaError_t e = act_map(&ti, in + in_c0, Cin, in_cs, B, H, Wd, KCA, bx, by);
    if (e == cudaSuccess) e = act_map(&tg, grad, Cout, g_cs, B, H, Wd, KCB, bx, by);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)mt, (unsigned)nt, (unsigned)splits);
#define WG_CASE(bn, kca, kcb)                                                                                       \
    if (BN == bn && KCA == kca && KCB == kcb)                                                                       \
        e = launch_wgrad<bn, kca, kcb>(grid, ti, tg, Cout, Cin, taps, bx, by, ntx, nty, npatch, per_split, scratch, \
                                       st);                                                                         \
    else
    WG_CASE(256, 64, 64)
    WG_CASE(128, 64, 64)
    WG_CASE(64, 64, 64)
    WG_CASE(32, 64, 32)
    WG_CASE(256, 32, 64)
    WG_CASE(128, 32, 64)
    WG_CASE(64, 32, 64)
    WG_CASE(32, 32, 32)
    e = cudaErrorInvalidValue;
#undef WG_CASE
    if (e != cudaSuccess) return e;
    k_conv_fold<<<(unsigned)((per + 255) / 256), 256, 0, st>>>(scratch, per, (int)splits, dW);
    if (db) {
        int64_t bs = (M + 1023) / 1024;
        if (bs > 1024) bs = 1024;
        const int bpp = (int)((M + bs - 1) / bs);
        k_conv_bias_part<<<(unsigned)bs, 256, 0, st>>>(grad, g_cs, Cout, (int)M, bpp, scratch);
        k_conv_fold<<<(unsigned)((Cout + 255) / 256), 256, 0, st>>>(scratch, Cout, (int)bs, db);
    }
    return cudaGetLastError();
}

cudaError_t conv_timeout(bool *flag, cudaStream_t st)
{
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_conv_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *flag = v != 0;
    if (e == cudaSuccess && v) {  // reported once; later convolutions run again
        const int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_conv_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e;
}

cudaError_t conv_set_wait_limit(int polls, cudaStream_t st)
{
    const int v = polls >= 0 ? polls : TC_WAIT;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_conv_wait_limit, &v, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace nn
}  // namespace lsm
