// Internal interface of the fused tensor-core training kernels (mf_train_tc.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mf {

constexpr int kTcMaxLayers = 8;  // hidden layers a batched column sum or a weight pack handles

// FP32 hidden weight matrices of one weight pack, layer by layer
struct TcPackLayers {
  const float* W[kTcMaxLayers];
};

// Forward of one hidden layer over all tiles: A_out = Taylor-mode tanh(W A_in^T + b).
// The collocation points' tiles (four Taylor channels) come first, then the data
// points' tiles (value channel); one launch covers both.
struct TcFwdParams {
  const uint8_t* A_in;   // tiles of A_{l-1} (BF16, swizzled operand layout)
  uint8_t* A_out;        // tiles of A_l
  const void* wimg;      // W_l image, K-major 128-byte swizzle, rows = output features
  const float* bias;     // b_l [128]
  int n_tiles4;          // collocation tiles (the first n_tiles4)
  int n_tiles;           // all tiles
  int* status;           // device status word (bounded waits)
};

// Forward of two consecutive hidden layers l, l+1: A_out1 = A_l, A_out2 = A_{l+1}; A_l is
// stored but not read back (layer l+1 reads it on chip).
struct TcFwd2Params {
  const uint8_t* A_in;   // tiles of A_{l-1}
  uint8_t* A_out1;       // tiles of A_l
  uint8_t* A_out2;       // tiles of A_{l+1}
  const void* wimg1;     // W_l image
  const void* wimg2;     // W_{l+1} image
  const float* bias1;    // b_l
  const float* bias2;    // b_{l+1}
  int n_tiles4;
  int n_tiles;
  int* status;
  // first = 1 (layers 1 and 2): A_{l-1} = A_0 is formed in the launch from the first
  // layer (Eq. 8) instead of loaded from A_in, and stored to A0_out for the backward pass
  int first;
  const float* Bf;       // [F][128] W1 g per function (b0 not included)
  const float* W0;       // [128][130] first-layer weights (W1 | W2)
  const float* b0;       // [128]
  const float* X[2];     // points of the collocation term [0] and the data term [1]
  int n[2];              // points per function of each term
  int R[2];              // points of each term
  uint8_t* A0_out;       // tiles of A_0
};

// One loss term of a backward launch: [0] the collocation points (four channels, the
// PDE residual), [1] the data points (value channel, u - y). Its tiles follow the other
// term's in the tile buffers (collocation first).
struct TcTerm {
  int n_tiles;           // tiles of the term
  int n_pts;             // its points (the data term's last tile may be padded)
  int n_per_fn;          // points per function
  const float* X;        // point coordinates [n_pts][2] (first layer's backward)
  const float* Y;        // data term: targets [n_pts]
  float gscale;          // top: 2 / (the term's points in the whole batch)
  double* loss_part;     // top: [CTAs][4] sums of squared residuals
  float* part32;         // first: [n_pts / 32][3][128] first-layer partial sums
};

// Backward of one hidden layer over all tiles (top = 1: the last hidden layer, with the
// output layer and the loss folded in; first = 1: layer 1 below the top, which also runs
// the first layer's backward in the epilogue, so that gA_0 is not written).
struct TcBwdParams {
  const uint8_t* A_in;   // tiles of A_{l-1}
  const uint8_t* gA_in;  // tiles of gA_l (unused at the top)
  uint8_t* gA_out;       // tiles of gA_{l-1} (unused with first = 1)
  const void* wimg;      // W_l image
  const void* wimgT;     // W_l^T image
  const float* bias;     // b_l
  float* gW_part;        // [CTAs][128][128] per-CTA g_W
  float* gb_part;        // [CTAs][4][128] per-CTA g_b (four point quarters)
  const float* wout;     // top: w_out [128]
  const float* bout;     // top: b_out (device scalar)
  float* gwout_part;     // top: [CTAs][4][128]
  float* gbout_part;     // top: [CTAs][4]
  TcTerm term[2];
  int top;
  int first;
  const float* Bf;       // first: W1 g per function [F][128]
  const float* W0;       // first: first-layer weights [128][130] (W1 | W2)
  const float* b0;       // first: [128]
  int* status;
};

size_t tc_tile_bytes();     // bytes of one 128 x 128 BF16 tile
int tc_tiles(int R, int C); // tiles of R points with C channels (the last one padded)
size_t tc_image_bytes();    // bytes of one 128 x 128 BF16 weight image
int tc_partial_ctas();      // most CTAs a backward launch uses (partial-buffer rows)
int tc_partial_groups();    // partial sums per CTA of g_b, g_wout, g_bout and the loss
// hidden weight matrices W_1..W_n (FP32 [128][128] each) -> n (W, W^T) image pairs,
// back to back from `images` (2 n tc_image_bytes()), in one launch
cudaError_t tc_pack_layers(const TcPackLayers& L, int n_layers, void* images, cudaStream_t st);
cudaError_t tc_first_fwd(const float* Bf, const float* W0, const float* b0, const float* X, int n, int R, int C,
                         void* A0, cudaStream_t st);
cudaError_t tc_first_bwd(const float* Bf, const float* W0, const float* b0, const float* X, int n, int R, int C,
                         const void* gA0, float* part, cudaStream_t st);
cudaError_t tc_layer_fwd(const TcFwdParams& p, cudaStream_t st);
cudaError_t tc_layer_fwd2(const TcFwd2Params& p, cudaStream_t st);
cudaError_t tc_layer_bwd(const TcBwdParams& p, int* grid_used, cudaStream_t st);
cudaError_t tc_colsum(const float* part, int nblk, int stride, int n, float* out, int accumulate, cudaStream_t st);
// out[off[l] + j] += sum over rows of layer l's nrows x ncols partials (at part + l
// layer_stride), for l < n_layers, in one launch
cudaError_t tc_colsum_layers(const float* part, int n_layers, size_t layer_stride, int nrows, int ncols, float* out,
                             const long long* out_off, cudaStream_t st);
// out (+)= column sums of a tall nrows x ncols matrix in two deterministic stages, with
// scratch (at least 64 x ncols floats) for the partial sums
cudaError_t tc_colsum_tall(const float* part, int nrows, int stride, int ncols, float* scratch, int scratch_floats,
                           float* out, int accumulate, cudaStream_t st);
cudaError_t tc_sum_double(const double* part, int n, double scale, double* out, cudaStream_t st);
cudaError_t tc_sum_float(const float* part, int n, float* out, cudaStream_t st);

}  // namespace mf
