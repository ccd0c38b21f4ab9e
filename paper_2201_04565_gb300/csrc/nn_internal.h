// nn_internal.h -- BF16 tensor-core kernels of the warm-start U-Net.
//
// Layouts: activations NHWC bf16 with an explicit channel stride (so a
// kernel can read or write a channel slice of a concatenated tensor);
// 3x3 conv weights [Cout][tap][Cin] bf16 with tap = ky * 3 + kx (K-major per
// output channel); master weights and optimizer moments FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lsm {
namespace nn {

typedef __nv_bfloat16 bf16;

// out[m, oc0 + n] = act(bias[n] + sum_k A[m, k] W[n, k]) for the implicit-GEMM
// view of a 3x3 (taps = 9, pad 1) or 1x1 (taps = 1) convolution.
cudaError_t conv_fwd(const bf16 *in, int in_cs, int in_c0, int Cin, const bf16 *W, const float *bias, bf16 *out,
                     int out_cs, int out_c0, int Cout, int B, int H, int Wd, int taps, bool relu, cudaStream_t st);

// Whether a tensor-core convolution gave up a bounded wait since the last
// query (the affected outputs are incomplete); clears the flag. Synchronises
// the stream.
cudaError_t conv_timeout(bool *flag, cudaStream_t st);

// Polls of each bounded mbarrier wait in the tensor-core convolution
// (0: give up at once; < 0: the default, 2^20).
cudaError_t conv_set_wait_limit(int polls, cudaStream_t st);

// dW[n][tap][ci] (+= over pixel splits, then folded in a fixed order) and
// db[n] from grad_pre (gradient at the conv output before activation).
cudaError_t conv_wgrad(const bf16 *grad, int g_cs, int Cout, const bf16 *in, int in_cs, int in_c0, int Cin, int B,
                       int H, int Wd, int taps, float *dW, float *db, float *scratch, size_t scratch_floats,
                       cudaStream_t st);

// Rotate a 3x3 conv's weights by 180 degrees and swap in/out channels, so
// that conv_fwd with the result computes the gradient w.r.t. the input.
cudaError_t rotate_weights(const bf16 *W, bf16 *Wr, int Cout, int Cin, int taps, cudaStream_t st);

}  // namespace nn
}  // namespace lsm
