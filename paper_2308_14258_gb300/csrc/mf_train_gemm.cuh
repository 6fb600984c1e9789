// Internal interface of the training step's own dense products (mf_train_gemm.cu).
#pragma once
#include <cuda_runtime.h>

namespace mf {

// Bf[f][j] = sum_{k<128} W0[j][k] G[f][k]: the first layer's boundary term per function
// (Eq. 8). W0 is the packed first-layer matrix [H][130], G [F][128], Bf [F][H].
cudaError_t train_boundary_fwd(const float* W0, const float* G, int F, int H, float* Bf, cudaStream_t st);

// gW0[j][k] += sum_f S[f][j] G[f][k] (k < 128): the boundary block's gradient from the
// per-function sums S [F][H] of the first layer's g_z. gW0 is the packed [H][130] block.
cudaError_t train_boundary_grad(const float* S, const float* G, int F, int H, float* gW0, cudaStream_t st);

// out[r][n] = sum_k in[r][k] M[k][n] over `rows` rows of H values, with M = W^T (trans = 1)
// or M = W (trans = 0); W is row-major [H][H] (output unit, input unit). Operands FP32
// (bf16 = 0) or BF16 (bf16 = 1); out FP32.
cudaError_t train_row_gemm(int bf16, int H, const void* in, const void* W, int trans, long rows, float* out,
                           cudaStream_t st);

// gW[n][k] += sum_r gZ[r][n] X[r][k] over `rows` rows, through nblk per-block partials
// of H x H floats in `part` added in block order.
cudaError_t train_weight_grad(int bf16, int H, const void* gZ, const void* X, long rows, float* part, int nblk,
                              float* gW, cudaStream_t st);

// Blocks (and H x H partials) train_weight_grad is given on the current device.
int train_wgrad_blocks();

}  // namespace mf
