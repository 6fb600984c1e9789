// K7-K9: one physics-informed SDNet training step (Eq. 3, Algorithm 1) on one GPU.
//
// Loss (Section 3.3): L = L_data + L_pde, L_data = mean over the data points of
// (N(x_b, g) - y_b)^2, L_pde = mean over the collocation points of (Delta_x N(x_c, g))^2.
// Algorithm 1: forward/backward of the data points, then of the collocation points,
// gradients summed; the allreduce of step 3 is the identity on one device.
//
// Instead of nested reverse-mode passes (three backward passes, Section 5.2) the
// Laplacian is carried forward in Taylor mode: every row holds four channels, the value
// h and its derivatives h_x, h_y and Delta h with respect to the query coordinate. For
// a linear layer each channel is multiplied by the same weights (the bias enters the
// value channel only), so the four channels are stacked as rows of one GEMM. For
// a = tanh(z), with s = 1 - a^2 and t = -2 a s:
//   a_x = s z_x,  a_y = s z_y,  Delta a = t (z_x^2 + z_y^2) + s Delta z.
// The first layer is input-split (Eq. 8): z = B[f] + W2 x with B[f] = W1 g_f + b0, so
// z_x = W2[:,0], z_y = W2[:,1] and Delta z = 0; the output u = w_out . h + b_out gives
// Delta u = w_out . Delta h.
// The backward pass is written out by hand (t' = dt/dz = -2 s^2 + 4 a^2 s):
//   g_z   = g_a s + (g_ax z_x + g_ay z_y) t + g_aL (t' (z_x^2 + z_y^2) + t Delta z)
//   g_zx  = g_ax s + 2 g_aL t z_x,  g_zy = g_ay s + 2 g_aL t z_y,  g_zL = g_aL s
// then for z = W h (+ b): g_W += sum over rows and channels of g_z h^T, g_b += sum of
// the value channel, g_h = W^T g_z per channel. In the first layer the boundary-weight
// gradient is input-split as well: sum g_z over each function's points, then one
// (H x F)(F x 128) product.
//
// Two engines run these formulas. The fused engine (BF16, width 128; mf_train_tc.cu)
// keeps each layer's GEMM and its Taylor-mode epilogue in one tensor-core kernel and
// moves only BF16 activation and gradient tiles through HBM. The GEMM engine (FP32 or
// BF16, any width) runs the layer products (stacked channels x H times H x H, and the
// H x H weight gradients) as separate FP32-accumulating kernels (mf_train_gemm.cu) and
// every other step in the kernels below. The first layer's boundary term and its
// gradient are the small products of mf_train_gemm.cu in both engines. Reductions use
// fixed-order block partials throughout, so results do not depend on timing.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mosaicflow.h"
#include "mf_internal.cuh"
#include "mf_train_gemm.cuh"
#include "mf_train_tc.cuh"

namespace mf {
void set_last_error(const std::string& msg);
}

namespace {

namespace cg = cooperative_groups;

constexpr int kRB = 64;        // rows per block in the row-tiled kernels
constexpr int kNB = 128;       // boundary values per function

// element type of GEMM operands
template <typename T> __device__ __forceinline__ T to_t(float x);
template <> __device__ __forceinline__ float to_t<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 to_t<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// First layer, Taylor mode: rows r = f*n + p, columns j (one thread per column);
// Bf[f][j] = (W1 g_f)_j comes from a GEMM.
template <typename T, int C>
__global__ void first_fwd_kernel(const float* __restrict__ Bf, const float* __restrict__ W0,
                                 const float* __restrict__ b0, const float* __restrict__ X, int n, int R, int H,
                                 T* __restrict__ A, float* __restrict__ a0) {
  const int j = threadIdx.x;
  const float w2x = W0[(size_t)j * (kNB + 2) + kNB], w2y = W0[(size_t)j * (kNB + 2) + kNB + 1];
  const float bj = b0[j];
  const int r1 = min(R, (blockIdx.x + 1) * kRB);
  for (int r = blockIdx.x * kRB; r < r1; ++r) {
    const int f = r / n;
    const float x = X[2 * (size_t)r], y = X[2 * (size_t)r + 1];
    const float a = tanhf(fmaf(w2y, y, fmaf(w2x, x, Bf[(size_t)f * H + j] + bj)));
    const size_t e = (size_t)r * H + j;
    a0[e] = a;
    A[e] = to_t<T>(a);
    if (C == 4) {
      const float s = 1.f - a * a, t = -2.f * a * s;
      const size_t cs = (size_t)R * H;
      A[cs + e] = to_t<T>(s * w2x);
      A[2 * cs + e] = to_t<T>(s * w2y);
      A[3 * cs + e] = to_t<T>(t * (w2x * w2x + w2y * w2y));
    }
  }
}

// Hidden layer activation, Taylor mode: Z (FP32, C channels) + bias -> A (GEMM type) and
// the value activation a (FP32, kept for the backward pass).
template <typename T, int C>
__global__ void act_fwd_kernel(const float* __restrict__ Z, const float* __restrict__ bias, int R, int H,
                               T* __restrict__ A, float* __restrict__ av) {
  const int j = threadIdx.x;
  const float b = bias[j];
  const size_t cs = (size_t)R * H;
  const int r1 = min(R, (blockIdx.x + 1) * kRB);
  for (int r = blockIdx.x * kRB; r < r1; ++r) {
    const size_t e = (size_t)r * H + j;
    const float a = tanhf(Z[e] + b);
    av[e] = a;
    A[e] = to_t<T>(a);
    if (C == 4) {
      const float s = 1.f - a * a, t = -2.f * a * s;
      const float zx = Z[cs + e], zy = Z[2 * cs + e], zl = Z[3 * cs + e];
      A[cs + e] = to_t<T>(s * zx);
      A[2 * cs + e] = to_t<T>(s * zy);
      A[3 * cs + e] = to_t<T>(fmaf(t, zx * zx + zy * zy, s * zl));
    }
  }
}

// Output layer and loss. One warp per row: u = w_out . a + b_out (data rows) or
// Delta u = w_out . Delta a (collocation rows, Delta a recomputed in FP32 from Z and a).
// Writes the loss partial of the block, the gradient w.r.t. the last activations, and
// block partials of the w_out / b_out gradients.
template <int C>
__global__ void out_kernel(const float* __restrict__ av, const float* __restrict__ Z,
                           const float* __restrict__ wout, const float* __restrict__ bout_p,
                           const float* __restrict__ Y, int R, int H,
                           float gscale, float* __restrict__ gA, double* __restrict__ loss_part,
                           float* __restrict__ gw_part, float* __restrict__ gbo_part) {
  __shared__ float sgw[8][128];
  __shared__ double sl[8];
  __shared__ float sgb[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t cs = (size_t)R * H;
  float gw[4] = {0.f, 0.f, 0.f, 0.f};
  double lsum = 0.0;
  float gbsum = 0.f;
  const float bout = *bout_p;
  const int r1 = min(R, (blockIdx.x + 1) * kRB);
  for (int r = blockIdx.x * kRB + warp; r < r1; r += 8) {
    float av4[4], al4[4];
    float dot = 0.f;
    for (int q = 0; q < H / 32; ++q) {
      const int j = lane + 32 * q;
      const size_t e = (size_t)r * H + j;
      const float a = av[e];
      av4[q] = a;
      if (C == 4) {
        const float s = 1.f - a * a, t = -2.f * a * s;
        const float zx = Z[cs + e], zy = Z[2 * cs + e], zl = Z[3 * cs + e];
        al4[q] = fmaf(t, zx * zx + zy * zy, s * zl);
        dot = fmaf(wout[j], al4[q], dot);
      } else {
        dot = fmaf(wout[j], a, dot);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    float gu = 0.f, gul = 0.f;
    if (C == 4) {
      gul = gscale * dot;  // d/dDelta u of mean (Delta u)^2
      lsum += (double)dot * (double)dot;
    } else {
      const float d = dot + bout - Y[r];
      gu = gscale * d;     // d/du of mean (u - y)^2
      lsum += (double)d * (double)d;
      gbsum += gu;
    }
    for (int q = 0; q < H / 32; ++q) {
      const int j = lane + 32 * q;
      const size_t e = (size_t)r * H + j;
      if (C == 4) {
        gA[e] = 0.f;
        gA[cs + e] = 0.f;
        gA[2 * cs + e] = 0.f;
        gA[3 * cs + e] = gul * wout[j];
        gw[q] = fmaf(gul, al4[q], gw[q]);
      } else {
        gA[e] = gu * wout[j];
        gw[q] = fmaf(gu, av4[q], gw[q]);
      }
    }
  }
  for (int q = 0; q < H / 32; ++q) sgw[warp][lane + 32 * q] = gw[q];
  if (lane == 0) { sl[warp] = lsum; sgb[warp] = gbsum; }
  __syncthreads();
  if (threadIdx.x < H) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += sgw[w][threadIdx.x];
    gw_part[(size_t)blockIdx.x * H + threadIdx.x] = s;
  }
  if (threadIdx.x == 0) {
    double l = 0.0;
    float b = 0.f;
    for (int w = 0; w < 8; ++w) { l += sl[w]; b += sgb[w]; }
    loss_part[blockIdx.x] = l;
    gbo_part[blockIdx.x] = b;
  }
}

// Hidden layer backward through the Taylor-mode tanh (see the file comment), plus the
// bias-gradient block partial (value channel).
template <typename T, int C>
__global__ void act_bwd_kernel(const float* __restrict__ gA, const float* __restrict__ Z, const float* __restrict__ av,
                               int R, int H, T* __restrict__ gZ, float* __restrict__ gb_part) {
  const int j = threadIdx.x;
  const size_t cs = (size_t)R * H;
  float gbs = 0.f;
  const int r1 = min(R, (blockIdx.x + 1) * kRB);
  for (int r = blockIdx.x * kRB; r < r1; ++r) {
    const size_t e = (size_t)r * H + j;
    const float a = av[e];
    const float s = 1.f - a * a, t = -2.f * a * s;
    const float ga = gA[e];
    float gz = ga * s;
    if (C == 4) {
      const float tp = -2.f * s * s + 4.f * a * a * s;
      const float gax = gA[cs + e], gay = gA[2 * cs + e], gal = gA[3 * cs + e];
      const float zx = Z[cs + e], zy = Z[2 * cs + e], zl = Z[3 * cs + e];
      gz += (gax * zx + gay * zy) * t + gal * fmaf(tp, zx * zx + zy * zy, t * zl);
      gZ[cs + e] = to_t<T>(fmaf(gax, s, 2.f * gal * t * zx));
      gZ[2 * cs + e] = to_t<T>(fmaf(gay, s, 2.f * gal * t * zy));
      gZ[3 * cs + e] = to_t<T>(gal * s);
    }
    gZ[e] = to_t<T>(gz);
    gbs += gz;
  }
  gb_part[(size_t)blockIdx.x * H + j] = gbs;
}

// First layer backward: g_z of the first layer (z_x = W2[:,0], z_y = W2[:,1], Delta z = 0)
// and its block partials: sum g_z (b0, and per function for W1 when a block's rows lie
// in one function), sum g_z x + g_zx and sum g_z y + g_zy (the two W2 columns).
template <int C>
__global__ void first_bwd_kernel(const float* __restrict__ gA, const float* __restrict__ a0,
                                 const float* __restrict__ W0, const float* __restrict__ X, int R, int H,
                                 float* __restrict__ part) {
  const int j = threadIdx.x;
  const float w2x = W0[(size_t)j * (kNB + 2) + kNB], w2y = W0[(size_t)j * (kNB + 2) + kNB + 1];
  const size_t cs = (size_t)R * H;
  float s0 = 0.f, sx = 0.f, sy = 0.f;
  const int r1 = min(R, (blockIdx.x + 1) * kRB);
  for (int r = blockIdx.x * kRB; r < r1; ++r) {
    const size_t e = (size_t)r * H + j;
    const float a = a0[e];
    const float s = 1.f - a * a, t = -2.f * a * s;
    const float ga = gA[e];
    float gz = ga * s, gzx = 0.f, gzy = 0.f;
    if (C == 4) {
      const float tp = -2.f * s * s + 4.f * a * a * s;
      const float gax = gA[cs + e], gay = gA[2 * cs + e], gal = gA[3 * cs + e];
      gz += (gax * w2x + gay * w2y) * t + gal * tp * (w2x * w2x + w2y * w2y);
      gzx = fmaf(gax, s, 2.f * gal * t * w2x);
      gzy = fmaf(gay, s, 2.f * gal * t * w2y);
    }
    const float x = X[2 * (size_t)r], y = X[2 * (size_t)r + 1];
    s0 += gz;
    sx += fmaf(gz, x, gzx);
    sy += fmaf(gz, y, gzy);
  }
  float* o = part + (size_t)blockIdx.x * 3 * H;
  o[j] = s0;
  o[H + j] = sx;
  o[2 * H + j] = sy;
}

// out[j] (+)= sum over b < nblk of part[b * stride + j]. Block (32 x 32): thread (ty, tx)
// sums blocks b = ty, ty + 32, ... of column 32 blockIdx.x + tx, then the 32 row sums
// are added in order of ty, so the result does not depend on timing.
__global__ void colsum_kernel(const float* __restrict__ part, int nblk, int stride, int H, float* __restrict__ out,
                              int accumulate) {
  __shared__ float sh[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + tx;
  float s = 0.f;
  if (j < H)
    for (int b = ty; b < nblk; b += 32) s += part[(size_t)b * stride + j];
  sh[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && j < H) {
    float t = 0.f;
    for (int k = 0; k < 32; ++k) t += sh[k][tx];
    out[j] = accumulate ? out[j] + t : t;
  }
}

// S[f][j] = sum of the first layer's g_z over function f's points, from the block
// partials (blocks_per_f = points per function / 64; a block never spans two functions).
__global__ void per_function_sum_kernel(const float* __restrict__ part, int blocks_per_f, int H,
                                        float* __restrict__ S, int accumulate) {
  const int f = blockIdx.x, j = threadIdx.x;
  float s = 0.f;
  for (int b = 0; b < blocks_per_f; ++b) s += part[(size_t)(f * blocks_per_f + b) * 3 * H + j];
  S[(size_t)f * H + j] = accumulate ? S[(size_t)f * H + j] + s : s;
}

__global__ void add_w2_b0_kernel(const float* __restrict__ sums3, int H, float* __restrict__ gW0, float* __restrict__ gb0) {
  // sums3: [3][H] = (sum g_z, sum g_z x + g_zx, sum g_z y + g_zy)
  const int j = threadIdx.x;
  if (j >= H) return;
  gb0[j] += sums3[j];
  gW0[(size_t)j * (kNB + 2) + kNB] += sums3[H + j];
  gW0[(size_t)j * (kNB + 2) + kNB + 1] += sums3[2 * H + j];
}

// *out += scale * sum of part[0..n) with 1024 threads: strided per-thread sums, then a
// shared-memory tree (fixed order, so the result does not depend on timing).
template <typename V>
__global__ void sum_all_kernel(const V* __restrict__ part, int n, V scale, V* __restrict__ out) {
  __shared__ V sh[1024];
  V s = 0;
  for (int i = threadIdx.x; i < n; i += 1024) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out += sh[0] * scale;
}

template <typename T>
__global__ void convert_kernel(const float* __restrict__ src, T* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = to_t<T>(src[i]);
}

// True when the gradient pass that precedes an update succeeded: no kernel wait gave up
// and both loss terms are finite. The update kernels read it on the device and do
// nothing otherwise, so a failed step leaves the weights and moments as they were.
__device__ __forceinline__ bool grad_pass_ok(const int* status, const double* loss) {
  return *status == mf::kDevErrNone && isfinite(loss[1]) && isfinite(loss[2]);
}

__global__ void sgd_kernel(float* __restrict__ w, const float* __restrict__ g, float lr, size_t n,
                           const int* __restrict__ status, const double* __restrict__ loss) {
  if (!grad_pass_ok(status, loss)) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    w[i] -= lr * g[i];
}

// LAMB (You et al., ICLR 2020): the moments and the raw update r of every element, then
// ||w|| and ||r|| of each parameter tensor (W0, b0, each W_l and b_l, w_out, b_out), then
// the trust-ratio step w -= lr (||w|| / ||r||) r, in one launch. A tensor is one
// thread-block cluster of kLambSplit CTAs; CTA c takes the c-th of kLambSplit equal
// slices and keeps its elements' w and r in registers (at most kLambPer per thread).
// Squares are summed in FP32 per thread and per warp (fixed shuffle tree), the warp sums
// in FP64 in warp order, and the CTAs' sums in rank order through distributed shared
// memory, so the norms do not depend on timing; FP64 arithmetic, slow on this part, is
// kept to the last few terms.
constexpr int kLambSplit = 8, kLambThreads = 256, kLambPer = 12;
constexpr size_t kLambMaxTensor = (size_t)kLambSplit * kLambThreads * kLambPer;
__global__ void __cluster_dims__(kLambSplit, 1, 1) __launch_bounds__(kLambThreads)
    lamb_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                const unsigned long long* __restrict__ ranges, float lr, float b1, float b2, float inv_c1,
                float inv_c2, float eps, float wd, const int* __restrict__ status, const double* __restrict__ loss) {
  // the same outcome for every CTA of the cluster, so none waits at the cluster barriers
  if (!grad_pass_ok(status, loss)) return;
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const int tensor = (int)(blockIdx.x / kLambSplit);
  const size_t b = ranges[2 * tensor], e = ranges[2 * tensor + 1];
  const size_t per = (e - b + kLambSplit - 1) / kLambSplit;
  const size_t cb = b + rank * per, ce = cb + per < e ? cb + per : e;
  float wr[kLambPer], rr[kLambPer];
  float aw = 0.f, ar = 0.f;
#pragma unroll
  for (int q = 0; q < kLambPer; ++q) {
    const size_t i = cb + threadIdx.x + (size_t)q * kLambThreads;
    wr[q] = rr[q] = 0.f;
    if (i < ce) {
      const float gi = g[i], wi = w[i];
      const float mi = b1 * m[i] + (1.f - b1) * gi;
      const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
      const float ri = (mi * inv_c1) / (sqrtf(vi * inv_c2) + eps) + wd * wi;
      m[i] = mi;
      v[i] = vi;
      wr[q] = wi;
      rr[q] = ri;
      aw = fmaf(wi, wi, aw);
      ar = fmaf(ri, ri, ar);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    aw += __shfl_down_sync(0xffffffffu, aw, o);
    ar += __shfl_down_sync(0xffffffffu, ar, o);
  }
  __shared__ float sw[kLambThreads / 32], sr[kLambThreads / 32];
  __shared__ double cta_w, cta_r;
  __shared__ float s_trust;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sw[warp] = aw; sr[warp] = ar; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double dw = 0.0, dr = 0.0;
    for (int k = 0; k < kLambThreads / 32; ++k) {
      dw += (double)sw[k];
      dr += (double)sr[k];
    }
    cta_w = dw;
    cta_r = dr;
  }
  cluster.sync();
  if (threadIdx.x == 0) {
    double tw = 0.0, tr = 0.0;
    for (unsigned c = 0; c < kLambSplit; ++c) {
      tw += *cluster.map_shared_rank(&cta_w, c);
      tr += *cluster.map_shared_rank(&cta_r, c);
    }
    const double wn = sqrt(tw), rn = sqrt(tr);
    s_trust = (wn > 0.0 && rn > 0.0) ? (float)(wn / rn) : 1.f;
  }
  cluster.sync();  // s_trust is set, and no CTA leaves while another reads its sums
  const float step = lr * s_trust;
#pragma unroll
  for (int q = 0; q < kLambPer; ++q) {
    const size_t i = cb + threadIdx.x + (size_t)q * kLambThreads;
    if (i < ce) w[i] = wr[q] - step * rr[q];
  }
}

}  // namespace

struct mf_trainer {
  int device = 0, H = 0, D = 0, NH = 0, precision = 0, optimizer = 0;
  float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-6f, wd = 0.f;
  int step = 0;
  int Fmax = 0, Nmax = 0;
  size_t Rmax = 0, n_params = 0;
  std::vector<size_t> offW, offb;  // hidden layer l = 1..NH
  size_t off_b0 = 0, off_wout = 0, off_bout = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  void* wq = nullptr;              // GEMM copies of the hidden weights [NH][H][H]
  std::vector<void*> A;            // [NH+1] GEMM-type [4][Rmax][H]
  std::vector<float*> Z;           // [NH+1] FP32 [4][Rmax][H] (index 0 unused)
  std::vector<float*> a;           // [NH+1] FP32 [Rmax][H]
  float* gA = nullptr;             // FP32 [4][Rmax][H]
  void* gZ = nullptr;              // GEMM-type [4][Rmax][H]
  float* Bf = nullptr;             // [Fmax][H] boundary term of the first layer
  float* S = nullptr;              // [Fmax][H] per-function sums of the first layer's g_z
  float* part = nullptr;           // block partials
  float* sums = nullptr;           // [3][H]
  double* lpart = nullptr;         // loss partials
  double* loss = nullptr;          // device [3]
  double* h_loss = nullptr;        // pinned [3]
  unsigned long long* ranges = nullptr;  // LAMB tensor ranges
  int n_groups = 0;
  float* wpart = nullptr;          // GEMM engine: per-block H x H weight-gradient partials
  int wblocks = 0;                 // their count
  // fused engine
  bool fused = false;
  void* timg = nullptr;            // [NH] x (W image, W^T image), BF16 swizzled
  float* tc_gw = nullptr;          // [NH][CTAs][H][H] per-layer, per-CTA g_W
  float* tc_gb = nullptr;          // [NH][CTAs][4][H] per-layer, per-CTA g_b
  float* tc_scratch = nullptr;     // [64][3 H] first stage of the first-layer sums
  float* tc_small = nullptr;       // per-CTA g_wout [CTAs][4][H], g_bout [CTAs][4]
  double* tc_loss = nullptr;       // [CTAs][2]
  int* status = nullptr;           // device status word of the fused kernels
  int* h_status = nullptr;         // pinned mirror
};

namespace {

mf_status tfail(mf_status code, const std::string& msg) {
  mf::set_last_error(msg);
  return code;
}
mf_status tcuda(cudaError_t e, const char* what) {
  return tfail(e == cudaErrorMemoryAllocation ? MF_ERR_OUT_OF_MEMORY : MF_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}
#define TR_CUDA(call, what)                          \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return tcuda(e_, what);   \
  } while (0)
#define TR_ON_DEVICE(dev, what)   \
  mf::DeviceGuard guard_((dev));  \
  if (guard_.err != cudaSuccess) return tcuda(guard_.err, what)

size_t esize(const mf_trainer* t) { return t->precision == MF_PREC_BF16 ? 2 : 4; }
int bf16(const mf_trainer* t) { return t->precision == MF_PREC_BF16 ? 1 : 0; }

// Row-major layer products of the GEMM engine (see the file comment):
// Z[rows][H] = X[rows][H] W^T   (W row-major [out][in])
cudaError_t gemm_fwd(mf_trainer* t, const void* W, const void* X, float* Zo, long rows, cudaStream_t st) {
  return mf::train_row_gemm(bf16(t), t->H, X, W, 1, rows, Zo, st);
}
// gX[rows][H] = gZ[rows][H] W
cudaError_t gemm_bwd_data(mf_trainer* t, const void* W, const void* gZ, float* gX, long rows, cudaStream_t st) {
  return mf::train_row_gemm(bf16(t), t->H, gZ, W, 0, rows, gX, st);
}
// gW[out][in] += gZ^T X over all rows
cudaError_t gemm_bwd_weight(mf_trainer* t, const void* X, const void* gZ, float* gW, long rows, cudaStream_t st) {
  return mf::train_weight_grad(bf16(t), t->H, gZ, X, rows, t->wpart, t->wblocks, gW, st);
}

// First layer, boundary block, FP32: Bf[f][j] = sum_k W0[j][k] G[f][k] (k < 128).
cudaError_t gemm_boundary(mf_trainer* t, const float* G, int F, cudaStream_t st) {
  return mf::train_boundary_fwd(t->w, G, F, t->H, t->Bf, st);
}
// First layer, boundary-block gradient, FP32: gW0[j][k] += sum_f S[f][j] G[f][k].
cudaError_t gemm_boundary_grad(mf_trainer* t, const float* G, int F, cudaStream_t st) {
  return mf::train_boundary_grad(t->S, G, F, t->H, t->g, st);
}

// One forward + backward pass over F functions with n points each (C = 1: data points,
// value channel only; C = 4: collocation points in Taylor mode). Gradients and the loss
// are added to t->g and *loss_slot; gscale = 2 / (points in the whole loss) and
// lscale = 1 / (points in the whole loss) make them the mean over every chunk.
template <typename T>
mf_status run_pass(mf_trainer* t, int C, int F, int n, const float* G, const float* X, const float* Y, float gscale,
                   double lscale, double* loss_slot, cudaStream_t st) {
  const int H = t->H, NH = t->NH;
  const int R = F * n;
  const int nblk = R / kRB;  // n is a multiple of kRB
  const int ncol = (H + 31) / 32;
  T* wq = static_cast<T*>(t->wq);
  // forward
  TR_CUDA(gemm_boundary(t, G, F, st), "train: boundary GEMM");
  if (C == 4)
    first_fwd_kernel<T, 4><<<nblk, H, 0, st>>>(t->Bf, t->w, t->w + t->off_b0, X, n, R, H, static_cast<T*>(t->A[0]),
                                               t->a[0]);
  else
    first_fwd_kernel<T, 1><<<nblk, H, 0, st>>>(t->Bf, t->w, t->w + t->off_b0, X, n, R, H, static_cast<T*>(t->A[0]),
                                               t->a[0]);
  TR_CUDA(cudaGetLastError(), "train: first layer");
  for (int l = 1; l <= NH; ++l) {
    TR_CUDA(gemm_fwd(t, wq + (size_t)(l - 1) * H * H, t->A[l - 1], t->Z[l], (long)C * R, st), "train: forward GEMM");
    const float* bl = t->w + t->offb[l];
    if (C == 4)
      act_fwd_kernel<T, 4><<<nblk, H, 0, st>>>(t->Z[l], bl, R, H, static_cast<T*>(t->A[l]), t->a[l]);
    else
      act_fwd_kernel<T, 1><<<nblk, H, 0, st>>>(t->Z[l], bl, R, H, static_cast<T*>(t->A[l]), t->a[l]);
    TR_CUDA(cudaGetLastError(), "train: activation");
  }
  // output, loss and the start of the backward pass
  float* gw_part = t->part;
  float* gbo_part = t->part + (size_t)nblk * H;
  if (C == 4)
    out_kernel<4><<<nblk, 256, 0, st>>>(t->a[NH], t->Z[NH], t->w + t->off_wout, t->w + t->off_bout, Y, R, H, gscale,
                                        t->gA, t->lpart, gw_part, gbo_part);
  else
    out_kernel<1><<<nblk, 256, 0, st>>>(t->a[NH], t->Z[NH], t->w + t->off_wout, t->w + t->off_bout, Y, R, H, gscale,
                                        t->gA, t->lpart, gw_part, gbo_part);
  TR_CUDA(cudaGetLastError(), "train: output");
  sum_all_kernel<double><<<1, 1024, 0, st>>>(t->lpart, nblk, lscale, loss_slot);
  colsum_kernel<<<ncol, 1024, 0, st>>>(gw_part, nblk, H, H, t->g + t->off_wout, 1);
  if (C == 1) sum_all_kernel<float><<<1, 1024, 0, st>>>(gbo_part, nblk, 1.f, t->g + t->off_bout);
  TR_CUDA(cudaGetLastError(), "train: output reductions");
  // hidden layers, top down
  for (int l = NH; l >= 1; --l) {
    if (C == 4)
      act_bwd_kernel<T, 4><<<nblk, H, 0, st>>>(t->gA, t->Z[l], t->a[l], R, H, static_cast<T*>(t->gZ), t->part);
    else
      act_bwd_kernel<T, 1><<<nblk, H, 0, st>>>(t->gA, t->Z[l], t->a[l], R, H, static_cast<T*>(t->gZ), t->part);
    TR_CUDA(cudaGetLastError(), "train: activation backward");
    colsum_kernel<<<ncol, 1024, 0, st>>>(t->part, nblk, H, H, t->g + t->offb[l], 1);
    TR_CUDA(gemm_bwd_weight(t, t->A[l - 1], t->gZ, t->g + t->offW[l], (long)C * R, st), "train: weight GEMM");
    TR_CUDA(gemm_bwd_data(t, wq + (size_t)(l - 1) * H * H, t->gZ, t->gA, (long)C * R, st), "train: data GEMM");
  }
  // first layer: W2 columns and b0 from all rows, W1 through per-function sums
  if (C == 4)
    first_bwd_kernel<4><<<nblk, H, 0, st>>>(t->gA, t->a[0], t->w, X, R, H, t->part);
  else
    first_bwd_kernel<1><<<nblk, H, 0, st>>>(t->gA, t->a[0], t->w, X, R, H, t->part);
  TR_CUDA(cudaGetLastError(), "train: first layer backward");
  for (int q = 0; q < 3; ++q) colsum_kernel<<<ncol, 1024, 0, st>>>(t->part + q * H, nblk, 3 * H, H, t->sums + q * H, 0);
  add_w2_b0_kernel<<<1, H, 0, st>>>(t->sums, H, t->g, t->g + t->off_b0);
  per_function_sum_kernel<<<F, H, 0, st>>>(t->part, n / kRB, H, t->S, 0);
  TR_CUDA(cudaGetLastError(), "train: first layer gradients");
  TR_CUDA(gemm_boundary_grad(t, G, F, st), "train: boundary gradient GEMM");
  return MF_OK;
}

// One chunk of functions on the fused engine, both loss terms at once: the first layer
// into A_0 tiles (collocation tiles first, then the data tiles), the forward kernels of
// hidden layers 1..NH-1, then the backward kernels from the top (which also forms the
// output layer and both losses) down; layer 1's kernel also runs the first layer's
// backward (with one hidden layer a separate kernel does, from the gA_0 tiles).
// term index 0: collocation points (four Taylor channels), 1: data points (value channel)
struct FusedTerm {
  int n;                 // points per function
  const float* X;        // coordinates of the chunk's points
  const float* Y;        // data targets (term 1)
  float gscale;          // 2 / (points of the term in the whole batch)
  double lscale;         // 1 / (points of the term in the whole batch)
  double* loss_slot;     // device accumulator of the term's loss
};

mf_status run_chunk_fused(mf_trainer* t, int F, const float* G, const FusedTerm (&term)[2], cudaStream_t st) {
  const int H = t->H, NH = t->NH;
  const int R[2] = {F * term[0].n, F * term[1].n};
  const int nt[2] = {mf::tc_tiles(R[0], 4), mf::tc_tiles(R[1], 1)};
  const size_t tile = mf::tc_tile_bytes();
  const size_t img = mf::tc_image_bytes();
  auto wimg = [&](int l) { return static_cast<const char*>(t->timg) + (size_t)(l - 1) * 2 * img; };
  const int ctas = mf::tc_partial_ctas(), pg = mf::tc_partial_groups();
  float* gwop = t->tc_small;
  float* gbop = gwop + (size_t)ctas * pg * H;
  const size_t gw_stride = (size_t)ctas * H * H, gb_stride = (size_t)ctas * pg * H;
  // per-32-point first-layer partial sums of each term, one after the other
  float* part32[2] = {t->part, t->part + (size_t)(R[0] / 32) * 3 * H};
  int grid_used = 0;
  TR_CUDA(gemm_boundary(t, G, F, st), "train: boundary GEMM");
  // with two or more hidden forward layers the first two-layer launch forms A_0 itself
  const bool first_in_fwd2 = NH >= 3;
  if (!first_in_fwd2)
    for (int k = 0; k < 2; ++k)
      TR_CUDA(mf::tc_first_fwd(t->Bf, t->w, t->w + t->off_b0, term[k].X, term[k].n, R[k], k == 0 ? 4 : 1,
                               static_cast<uint8_t*>(t->A[0]) + (k == 0 ? 0 : (size_t)nt[0] * tile), st),
              "train: first layer");
  // hidden layers 1..NH-1 forward, two per launch where two remain (layer l's output
  // stays on chip as layer l+1's input, besides being stored for the backward pass)
  for (int l = 1; l < NH;) {
    if (l + 1 < NH) {
      mf::TcFwd2Params fp{static_cast<const uint8_t*>(t->A[l - 1]), static_cast<uint8_t*>(t->A[l]),
                          static_cast<uint8_t*>(t->A[l + 1]), wimg(l), wimg(l + 1), t->w + t->offb[l],
                          t->w + t->offb[l + 1], nt[0], nt[0] + nt[1], t->status};
      if (l == 1 && first_in_fwd2) {
        fp.first = 1;
        fp.Bf = t->Bf;
        fp.W0 = t->w;
        fp.b0 = t->w + t->off_b0;
        for (int k = 0; k < 2; ++k) {
          fp.X[k] = term[k].X;
          fp.n[k] = term[k].n;
          fp.R[k] = R[k];
        }
        fp.A0_out = static_cast<uint8_t*>(t->A[0]);
      }
      TR_CUDA(mf::tc_layer_fwd2(fp, st), "train: fused two-layer forward");
      l += 2;
    } else {
      mf::TcFwdParams fp{static_cast<const uint8_t*>(t->A[l - 1]), static_cast<uint8_t*>(t->A[l]), wimg(l),
                         t->w + t->offb[l], nt[0], nt[0] + nt[1], t->status};
      TR_CUDA(mf::tc_layer_fwd(fp, st), "train: fused forward");
      l += 1;
    }
  }
  uint8_t* gbuf[2] = {static_cast<uint8_t*>(t->gZ), reinterpret_cast<uint8_t*>(t->gA)};
  int cur = 0;
  for (int l = NH; l >= 1; --l) {
    mf::TcBwdParams bp{};
    bp.A_in = static_cast<const uint8_t*>(t->A[l - 1]);
    bp.gA_in = l == NH ? nullptr : gbuf[cur];
    bp.gA_out = gbuf[cur ^ 1];
    bp.wimg = wimg(l);
    bp.wimgT = wimg(l) + img;
    bp.bias = t->w + t->offb[l];
    bp.gW_part = t->tc_gw + (size_t)(l - 1) * gw_stride;
    bp.gb_part = t->tc_gb + (size_t)(l - 1) * gb_stride;
    bp.wout = t->w + t->off_wout;
    bp.bout = t->w + t->off_bout;
    bp.gwout_part = gwop;
    bp.gbout_part = gbop;
    for (int k = 0; k < 2; ++k) {
      bp.term[k].n_tiles = nt[k];
      bp.term[k].n_pts = R[k];
      bp.term[k].n_per_fn = term[k].n;
      bp.term[k].X = term[k].X;
      bp.term[k].Y = term[k].Y;
      bp.term[k].gscale = term[k].gscale;
      bp.term[k].loss_part = t->tc_loss + (size_t)k * ctas * pg;
      bp.term[k].part32 = part32[k];
    }
    bp.top = l == NH ? 1 : 0;
    // layer 1 below the top also runs the first layer's backward (no gA_0 tiles)
    bp.first = (l == 1 && NH >= 2) ? 1 : 0;
    bp.Bf = t->Bf;
    bp.W0 = t->w;
    bp.b0 = t->w + t->off_b0;
    bp.status = t->status;
    int grid = 0;
    TR_CUDA(mf::tc_layer_bwd(bp, &grid, st), "train: fused backward");
    grid_used = grid;
    if (grid > 0 && l == NH) {
      TR_CUDA(mf::tc_colsum(gwop, pg * grid, H, H, t->g + t->off_wout, 1, st), "train: g_wout");
      TR_CUDA(mf::tc_sum_float(gbop, pg * grid, t->g + t->off_bout, st), "train: g_bout");
      for (int k = 0; k < 2; ++k)
        TR_CUDA(mf::tc_sum_double(t->tc_loss + (size_t)k * ctas * pg, pg * grid, term[k].lscale, term[k].loss_slot,
                                  st),
                "train: loss");
    }
    cur ^= 1;
  }
  // g_W and g_b of every hidden layer, from the per-layer partial sums, in two launches
  if (grid_used > 0) {
    long long offW[mf::kTcMaxLayers], offb[mf::kTcMaxLayers];
    for (int l = 1; l <= NH; ++l) {
      offW[l - 1] = (long long)t->offW[l];
      offb[l - 1] = (long long)t->offb[l];
    }
    TR_CUDA(mf::tc_colsum_layers(t->tc_gw, NH, gw_stride, grid_used, H * H, t->g, offW, st), "train: g_W");
    TR_CUDA(mf::tc_colsum_layers(t->tc_gb, NH, gb_stride, pg * grid_used, H, t->g, offb, st), "train: g_b");
  }
  // first layer, per term: W2 columns and b0 from all rows, W1 through per-function sums
  // (S of both terms added, then one GEMM). Partial sums per 32 points from the layer-1
  // kernel, or (one hidden layer) per 64 points from the first-layer kernel on gA_0.
  for (int k = 0; k < 2; ++k) {
    const int C = k == 0 ? 4 : 1;
    int group = 32;
    float* part = part32[k];
    if (NH == 1) {
      group = kRB;
      part = t->part;
      TR_CUDA(mf::tc_first_bwd(t->Bf, t->w, t->w + t->off_b0, term[k].X, term[k].n, R[k], C,
                               gbuf[cur] + (k == 0 ? 0 : (size_t)nt[0] * tile), part, st),
              "train: first layer backward");
    }
    TR_CUDA(mf::tc_colsum_tall(part, R[k] / group, 3 * H, 3 * H, t->tc_scratch, 64 * 3 * H, t->sums, 0, st),
            "train: first layer sums");
    add_w2_b0_kernel<<<1, H, 0, st>>>(t->sums, H, t->g, t->g + t->off_b0);
    per_function_sum_kernel<<<F, H, 0, st>>>(part, term[k].n / group, H, t->S, k);
  }
  TR_CUDA(cudaGetLastError(), "train: first layer gradients");
  TR_CUDA(gemm_boundary_grad(t, G, F, st), "train: boundary gradient GEMM");
  return MF_OK;
}

// Both loss terms on the fused engine, in chunks of at most max_functions functions.
mf_status run_terms_fused(mf_trainer* t, int F, int Nc, int Nb, const float* G, const float* Xc, const float* Xb,
                          const float* Yb, cudaStream_t st) {
  const double nc = (double)F * Nc, nb = (double)F * Nb;
  for (int f0 = 0; f0 < F; f0 += t->Fmax) {
    const int fc = F - f0 < t->Fmax ? F - f0 : t->Fmax;
    const FusedTerm term[2] = {
        {Nc, Xc + (size_t)f0 * Nc * 2, nullptr, (float)(2.0 / nc), 1.0 / nc, t->loss + 2},
        {Nb, Xb + (size_t)f0 * Nb * 2, Yb + (size_t)f0 * Nb, (float)(2.0 / nb), 1.0 / nb, t->loss + 1}};
    mf_status s = run_chunk_fused(t, fc, G + (size_t)f0 * kNB, term, st);
    if (s != MF_OK) return s;
  }
  return MF_OK;
}

// All functions of one loss term, in chunks of at most max_functions functions.
mf_status run_term(mf_trainer* t, int C, int F, int n, const float* G, const float* X, const float* Y,
                   double* loss_slot, cudaStream_t st) {
  const double npts = (double)F * n;
  for (int f0 = 0; f0 < F; f0 += t->Fmax) {
    const int fc = F - f0 < t->Fmax ? F - f0 : t->Fmax;
    const float* Gc = G + (size_t)f0 * kNB;
    const float* Xc = X + (size_t)f0 * n * 2;
    const float* Yc = Y ? Y + (size_t)f0 * n : nullptr;
    mf_status s = t->precision == MF_PREC_BF16
                      ? run_pass<__nv_bfloat16>(t, C, fc, n, Gc, Xc, Yc, (float)(2.0 / npts), 1.0 / npts, loss_slot, st)
                      : run_pass<float>(t, C, fc, n, Gc, Xc, Yc, (float)(2.0 / npts), 1.0 / npts, loss_slot, st);
    if (s != MF_OK) return s;
  }
  return MF_OK;
}

mf_status refresh_gemm_weights(mf_trainer* t, cudaStream_t st) {
  const size_t HH = (size_t)t->H * t->H;
  if (t->fused) {
    mf::TcPackLayers L{};
    for (int l = 1; l <= t->NH; ++l) L.W[l - 1] = t->w + t->offW[l];
    TR_CUDA(mf::tc_pack_layers(L, t->NH, t->timg, st), "train: weight images");
    return MF_OK;
  }
  for (int l = 1; l <= t->NH; ++l) {
    if (t->precision == MF_PREC_BF16)
      convert_kernel<__nv_bfloat16><<<64, 256, 0, st>>>(t->w + t->offW[l],
                                                        static_cast<__nv_bfloat16*>(t->wq) + (l - 1) * HH, HH);
    else
      convert_kernel<float><<<64, 256, 0, st>>>(t->w + t->offW[l], static_cast<float*>(t->wq) + (l - 1) * HH, HH);
  }
  TR_CUDA(cudaGetLastError(), "train: weight copy");
  return MF_OK;
}

// The gradient pass of one step, enqueued on st (Algorithm 1, steps 1-2: the data points'
// value channel, the collocation points' four Taylor channels): gradients into t->g, the
// loss into t->loss, and the loss and the device status word copied to pinned host
// memory. The caller synchronises st and then calls grad_outcome.
mf_status enqueue_grad(mf_trainer* t, int F, int Nc, int Nb, const float* G, const float* Xc, const float* Xb,
                       const float* Yb, cudaStream_t st) {
  TR_CUDA(cudaMemsetAsync(t->g, 0, t->n_params * 4, st), "train: zero grads");
  TR_CUDA(cudaMemsetAsync(t->loss, 0, 3 * sizeof(double), st), "train: zero loss");
  TR_CUDA(cudaMemsetAsync(t->status, 0, sizeof(int), st), "train: reset status");
  mf_status s;
  if (t->fused) {
    s = run_terms_fused(t, F, Nc, Nb, G, Xc, Xb, Yb, st);
  } else {
    s = run_term(t, 1, F, Nb, G, Xb, Yb, t->loss + 1, st);
    if (s == MF_OK) s = run_term(t, 4, F, Nc, G, Xc, nullptr, t->loss + 2, st);
  }
  if (s != MF_OK) return s;
  TR_CUDA(cudaMemcpyAsync(t->h_loss, t->loss, 3 * sizeof(double), cudaMemcpyDeviceToHost, st), "train: loss");
  TR_CUDA(cudaMemcpyAsync(t->h_status, t->status, sizeof(int), cudaMemcpyDeviceToHost, st), "train: status");
  return MF_OK;
}

// The outcome of a synchronised gradient pass: MF_ERR_TIMEOUT if a kernel wait gave up,
// MF_ERR_DIVERGED if a loss term is not finite; the loss (total, data, PDE) into loss3.
mf_status grad_outcome(mf_trainer* t, double* loss3, const char* who) {
  if (*t->h_status != mf::kDevErrNone) return tfail(MF_ERR_TIMEOUT, std::string(who) + ": a kernel wait timed out");
  if (loss3) {
    loss3[1] = t->h_loss[1];
    loss3[2] = t->h_loss[2];
    loss3[0] = loss3[1] + loss3[2];
  }
  if (!std::isfinite(t->h_loss[1]) || !std::isfinite(t->h_loss[2]))
    return tfail(MF_ERR_DIVERGED, std::string(who) + ": loss is not finite");
  return MF_OK;
}

mf_status validate_batch(const mf_trainer* t, int F, int Nc, int Nb, const void* G, const void* Xc, const void* Xb,
                         const void* Yb) {
  if (!G || !Xc || !Xb || !Yb) return tfail(MF_ERR_INVALID_ARG, "mf_train: null input");
  // the kernels read the inputs in 16-byte vectors and copies
  if ((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(Xc) | reinterpret_cast<uintptr_t>(Xb) |
       reinterpret_cast<uintptr_t>(Yb)) & 15u)
    return tfail(MF_ERR_INVALID_ARG, "mf_train: G, Xc, Xb and Yb must start on a 16-byte boundary");
  if (F < 1) return tfail(MF_ERR_INVALID_ARG, "mf_train: F must be >= 1");
  if (Nc < kRB || Nc > t->Nmax || Nc % kRB) return tfail(MF_ERR_INVALID_ARG, "mf_train: Nc must be a multiple of 64 up to max_points");
  if (Nb < kRB || Nb > t->Nmax || Nb % kRB) return tfail(MF_ERR_INVALID_ARG, "mf_train: Nb must be a multiple of 64 up to max_points");
  return MF_OK;
}

}  // namespace

extern "C" {

mf_status mf_destroy_trainer(mf_trainer* t) {
  if (!t) return MF_OK;
  mf::DeviceGuard guard(t->device);
  cudaFree(t->wpart);
  for (void* p : t->A) cudaFree(p);
  for (float* p : t->Z) cudaFree(p);
  for (float* p : t->a) cudaFree(p);
  cudaFree(t->w); cudaFree(t->g); cudaFree(t->m); cudaFree(t->v);
  cudaFree(t->wq); cudaFree(t->gA); cudaFree(t->gZ); cudaFree(t->Bf); cudaFree(t->S); cudaFree(t->part); cudaFree(t->sums);
  cudaFree(t->lpart); cudaFree(t->loss); cudaFree(t->ranges);
  cudaFree(t->timg); cudaFree(t->tc_gw); cudaFree(t->tc_gb); cudaFree(t->tc_scratch); cudaFree(t->tc_small);
  cudaFree(t->tc_loss); cudaFree(t->status);
  cudaFreeHost(t->h_loss); cudaFreeHost(t->h_status);
  delete t;
  return MF_OK;
}

mf_status mf_create_trainer(mf_ctx* ctx, const mf_train_desc* d, const float* weights, mf_trainer** out) {
  if (!d || !weights || !out) return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: null argument");
  *out = nullptr;
  if (d->width != 64 && d->width != 128) return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: width must be 64 or 128");
  if (d->depth < 2 || d->depth > 6) return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: depth must be in 2..6");
  if (d->max_functions < 1 || d->max_points < kRB || d->max_points % kRB)
    return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: need max_functions >= 1 and max_points a multiple of 64");
  if (4.0 * d->max_functions * d->max_points > 2147483647.0)
    return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: 4 * max_functions * max_points must fit in an int");
  if (d->precision != MF_PREC_FP32 && d->precision != MF_PREC_BF16)
    return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: precision must be MF_PREC_FP32 or MF_PREC_BF16");
  if (d->optimizer != MF_OPT_SGD && d->optimizer != MF_OPT_LAMB)
    return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: unknown optimizer");
  if (d->engine != MF_TRAIN_ENGINE_AUTO && d->engine != MF_TRAIN_ENGINE_GEMM)
    return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: unknown engine");
  {
    const size_t h = (size_t)d->width, n_params = h * (kNB + 2) + h + (size_t)(d->depth - 1) * (h * h + h) + h + 1;
    for (size_t i = 0; i < n_params; ++i)
      if (!std::isfinite(weights[i])) return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: non-finite weight");
  }
  if (!ctx) return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: null context");
  TR_ON_DEVICE(ctx->device, "mf_create_trainer: cudaSetDevice");
  mf_trainer* t = new mf_trainer();
  t->device = ctx->device;
  t->H = d->width;
  t->D = d->depth;
  t->NH = d->depth - 1;
  t->precision = d->precision;
  t->optimizer = d->optimizer;
  t->beta1 = d->beta1;
  t->beta2 = d->beta2;
  t->eps = d->eps;
  t->wd = d->weight_decay;
  t->Fmax = d->max_functions;
  t->Nmax = d->max_points;
  t->fused = d->engine == MF_TRAIN_ENGINE_AUTO && t->precision == MF_PREC_BF16 && t->H == 128;
  t->Rmax = (size_t)t->Fmax * t->Nmax;
  const size_t H = t->H, HH = H * H;
  t->off_b0 = H * (kNB + 2);
  t->offW.assign(t->NH + 1, 0);
  t->offb.assign(t->NH + 1, 0);
  for (int l = 1; l <= t->NH; ++l) {
    t->offW[l] = t->off_b0 + H + (size_t)(l - 1) * (HH + H);
    t->offb[l] = t->offW[l] + HH;
  }
  t->off_wout = t->off_b0 + H + (size_t)t->NH * (HH + H);
  t->off_bout = t->off_wout + H;
  t->n_params = t->off_bout + 1;
  const size_t es = esize(t), C4 = 4 * t->Rmax * H;
  // fused engine: a tile buffer holds a chunk's collocation tiles (4 channels, 32 points
  // each) followed by its data tiles (128 points each, the last one padded)
  const size_t fused_tile_bytes = (t->Rmax / 32 + t->Rmax / 128 + 2) * mf::tc_tile_bytes();
  const size_t nblk_max = (t->Rmax + kRB - 1) / kRB;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  alloc((void**)&t->w, t->n_params * 4);
  alloc((void**)&t->g, t->n_params * 4);
  alloc((void**)&t->m, t->n_params * 4);
  alloc((void**)&t->v, t->n_params * 4);
  alloc(&t->wq, (size_t)t->NH * HH * es);
  t->A.assign(t->NH + 1, nullptr);
  t->Z.assign(t->NH + 1, nullptr);
  t->a.assign(t->NH + 1, nullptr);
  for (int l = 0; l <= t->NH; ++l) {
    if (t->fused) {
      // activation tiles A_0..A_{NH-1} only: pre-activations are recomputed, never stored
      if (l < t->NH) alloc(&t->A[l], fused_tile_bytes);
      continue;
    }
    alloc(&t->A[l], C4 * es);
    alloc((void**)&t->a[l], t->Rmax * H * 4);
    if (l > 0) alloc((void**)&t->Z[l], C4 * 4);
  }
  if (t->fused) {
    const size_t ctas = (size_t)mf::tc_partial_ctas();
    alloc(&t->timg, (size_t)t->NH * 2 * mf::tc_image_bytes());
    alloc((void**)&t->tc_gw, (size_t)t->NH * ctas * HH * 4);
    alloc((void**)&t->tc_gb, (size_t)t->NH * ctas * mf::tc_partial_groups() * H * 4);
    alloc((void**)&t->tc_scratch, 64 * 3 * H * 4);
    const size_t pg = (size_t)mf::tc_partial_groups();
    alloc((void**)&t->tc_small, (ctas * pg * H + ctas * pg) * 4);
    alloc((void**)&t->tc_loss, 2 * ctas * pg * 8);
  }
  alloc((void**)&t->status, sizeof(int));
  alloc((void**)&t->gA, std::max(C4 * 4, fused_tile_bytes));
  alloc(&t->gZ, std::max(C4 * es, fused_tile_bytes));
  alloc((void**)&t->Bf, (size_t)t->Fmax * H * 4);
  alloc((void**)&t->S, (size_t)t->Fmax * H * 4);
  // row-block partials (64 rows) of the GEMM engine, or per-32-point first-layer partials
  // of the fused engine
  alloc((void**)&t->part, std::max(nblk_max * 3 * H * 4 + nblk_max * 4, (2 * t->Rmax / 32 + 2) * 3 * H * 4));
  alloc((void**)&t->sums, 3 * H * 4);
  alloc((void**)&t->lpart, nblk_max * 8);
  if (!t->fused) {
    t->wblocks = mf::train_wgrad_blocks();
    alloc((void**)&t->wpart, (size_t)t->wblocks * HH * 4);
  }
  alloc((void**)&t->loss, 4 * 8);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&t->h_loss, 4 * 8);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&t->h_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(t->status, 0, sizeof(int));
  // LAMB tensor ranges in packed order: W0, b0, {W_l, b_l}, w_out, b_out
  std::vector<unsigned long long> rg;
  rg.push_back(0); rg.push_back(t->off_b0);
  rg.push_back(t->off_b0); rg.push_back(t->off_b0 + H);
  for (int l = 1; l <= t->NH; ++l) {
    rg.push_back(t->offW[l]); rg.push_back(t->offW[l] + HH);
    rg.push_back(t->offb[l]); rg.push_back(t->offb[l] + H);
  }
  rg.push_back(t->off_wout); rg.push_back(t->off_wout + H);
  rg.push_back(t->off_bout); rg.push_back(t->off_bout + 1);
  t->n_groups = (int)rg.size() / 2;
  for (size_t k = 0; k < rg.size(); k += 2)
    if (rg[k + 1] - rg[k] > kLambMaxTensor) {
      mf_destroy_trainer(t);
      return tfail(MF_ERR_INVALID_ARG, "mf_create_trainer: a parameter tensor exceeds the optimiser's capacity");
    }
  alloc((void**)&t->ranges, rg.size() * 8);
  if (e == cudaSuccess) e = cudaMemcpy(t->ranges, rg.data(), rg.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t->w, weights, t->n_params * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(t->m, 0, t->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(t->v, 0, t->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(t->g, 0, t->n_params * 4);
  if (e != cudaSuccess) {
    mf_destroy_trainer(t);
    return tcuda(e, "mf_create_trainer");
  }
  mf_status s = refresh_gemm_weights(t, nullptr);
  if (s == MF_OK && cudaDeviceSynchronize() != cudaSuccess) s = tcuda(cudaGetLastError(), "mf_create_trainer");
  if (s != MF_OK) {
    mf_destroy_trainer(t);
    return s;
  }
  *out = t;
  return MF_OK;
}

mf_status mf_trainer_set_weights(mf_trainer* t, const float* src, int on_device, void* stream) {
  if (!t || !src) return tfail(MF_ERR_INVALID_ARG, "mf_trainer_set_weights: null argument");
  TR_ON_DEVICE(t->device, "mf_trainer_set_weights");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TR_CUDA(cudaMemcpyAsync(t->w, src, t->n_params * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
          "mf_trainer_set_weights");
  return refresh_gemm_weights(t, st);
}

mf_status mf_trainer_get_weights(const mf_trainer* t, float* dst, int on_device, void* stream) {
  if (!t || !dst) return tfail(MF_ERR_INVALID_ARG, "mf_trainer_get_weights: null argument");
  TR_ON_DEVICE(t->device, "mf_trainer_get_weights");
  TR_CUDA(cudaMemcpyAsync(dst, t->w, t->n_params * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          reinterpret_cast<cudaStream_t>(stream)),
          "mf_trainer_get_weights");
  return MF_OK;
}

mf_status mf_trainer_get_grads(const mf_trainer* t, float* dst, int on_device, void* stream) {
  if (!t || !dst) return tfail(MF_ERR_INVALID_ARG, "mf_trainer_get_grads: null argument");
  TR_ON_DEVICE(t->device, "mf_trainer_get_grads");
  TR_CUDA(cudaMemcpyAsync(dst, t->g, t->n_params * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          reinterpret_cast<cudaStream_t>(stream)),
          "mf_trainer_get_grads");
  return MF_OK;
}

mf_status mf_train_grad(mf_trainer* t, int F, int Nc, int Nb, const float* G, const float* Xc, const float* Xb,
                        const float* Yb, double* loss3, void* stream) {
  if (!t) return tfail(MF_ERR_INVALID_ARG, "mf_train_grad: null trainer");
  mf_status s = validate_batch(t, F, Nc, Nb, G, Xc, Xb, Yb);
  if (s != MF_OK) return s;
  TR_ON_DEVICE(t->device, "mf_train_grad");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = enqueue_grad(t, F, Nc, Nb, G, Xc, Xb, Yb, st);
  if (s != MF_OK) return s;
  TR_CUDA(cudaStreamSynchronize(st), "mf_train_grad: synchronize");
  return grad_outcome(t, loss3, "mf_train_grad");
}

mf_status mf_train_step(mf_trainer* t, int F, int Nc, int Nb, const float* G, const float* Xc, const float* Xb,
                        const float* Yb, float lr, double* loss3, void* stream) {
  if (!t) return tfail(MF_ERR_INVALID_ARG, "mf_train_step: null trainer");
  if (!std::isfinite(lr)) return tfail(MF_ERR_INVALID_ARG, "mf_train_step: lr must be finite");
  mf_status s = validate_batch(t, F, Nc, Nb, G, Xc, Xb, Yb);
  if (s != MF_OK) return s;
  TR_ON_DEVICE(t->device, "mf_train_step");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = enqueue_grad(t, F, Nc, Nb, G, Xc, Xb, Yb, st);
  if (s != MF_OK) return s;
  // the update follows the gradient pass on the stream without a host round trip: its
  // kernels read the pass's status word and loss on the device and skip the update if
  // the pass failed (the host reports the failure after the one synchronisation)
  const bool lamb = t->optimizer != MF_OPT_SGD;
  if (!lamb) {
    sgd_kernel<<<256, 256, 0, st>>>(t->w, t->g, lr, t->n_params, t->status, t->loss);
  } else {
    ++t->step;
    // bias corrections in double: 1 - beta^k cancels badly in FP32 for beta near 1
    const float inv_c1 = (float)(1.0 / (1.0 - pow((double)t->beta1, t->step)));
    const float inv_c2 = (float)(1.0 / (1.0 - pow((double)t->beta2, t->step)));
    lamb_kernel<<<t->n_groups * kLambSplit, kLambThreads, 0, st>>>(t->w, t->g, t->m, t->v, t->ranges, lr, t->beta1,
                                                                   t->beta2, inv_c1, inv_c2, t->eps, t->wd, t->status,
                                                                   t->loss);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) s = refresh_gemm_weights(t, st);
  const cudaError_t es = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess || s != MF_OK) {
    if (lamb) --t->step;
    return e != cudaSuccess ? tcuda(e, "mf_train_step: update") : s;
  }
  s = grad_outcome(t, loss3, "mf_train_step");
  if (s != MF_OK && lamb) --t->step;  // the update was skipped on the device
  return s;
}

}  // extern "C"
