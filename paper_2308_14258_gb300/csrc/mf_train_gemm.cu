// Dense products of the training step that are not layer kernels of the fused engine
// (Eq. 3, Algorithm 1; the input-split first layer of Eq. 7-8):
//
//  * the boundary term of the first layer, Bf[f][j] = sum_k W0[j][k] G[f][k] (k < 128),
//    one 128-wide matrix-vector product per function, and its gradient
//    gW0[j][k] += sum_f S[f][j] G[f][k], where S[f][j] is the first layer's g_z summed
//    over function f's points;
//  * the layer products of the GEMM engine (every channel of every row through the same
//    H x H matrix): Z = X W^T (forward), gX = gZ W (backward to the activations) and
//    gW += gZ^T X summed over all rows (backward to the weights).
//
// All run on the FP32 pipe: operands of type T (FP32 or BF16) are widened to FP32 in
// shared memory, products are accumulated in FP32, and every sum over rows or functions
// is taken in a fixed order (per-block partials added by one ordered column sum), so the
// results do not depend on timing.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mf_internal.cuh"
#include "mf_train_gemm.cuh"

namespace mf {
namespace {

namespace cg = cooperative_groups;

constexpr int kNB = 128;     // boundary values per function (columns of W1)
constexpr int kLd0 = kNB + 2;  // row length of W0 in the packed weights

template <typename T> __device__ __forceinline__ float widen(T x);
template <> __device__ __forceinline__ float widen<float>(float x) { return x; }
template <> __device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

// Bf[f][j] = sum_k W0[j][k] G[f][k]: a block takes kGF functions (their boundaries in
// shared memory), thread j one output column for each of them.
constexpr int kGF = 8;
__global__ void boundary_fwd_kernel(const float* __restrict__ W0, const float* __restrict__ G, int F, int H,
                                    float* __restrict__ Bf) {
  __shared__ float sg[kGF][kNB];
  const int f0 = blockIdx.x * kGF;
  for (int i = threadIdx.x; i < kGF * kNB; i += blockDim.x) {
    const int f = f0 + i / kNB;
    sg[i / kNB][i % kNB] = f < F ? G[(size_t)f * kNB + i % kNB] : 0.f;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= H) return;
  float acc[kGF];
#pragma unroll
  for (int q = 0; q < kGF; ++q) acc[q] = 0.f;
  const float* w = W0 + (size_t)j * kLd0;
  for (int k = 0; k < kNB; ++k) {
    const float wk = __ldg(w + k);
#pragma unroll
    for (int q = 0; q < kGF; ++q) acc[q] = fmaf(wk, sg[q][k], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < kGF; ++q)
    if (f0 + q < F) Bf[(size_t)(f0 + q) * H + j] = acc[q];
}

// gW0[j][k] += sum_f S[f][j] G[f][k] for k < 128: output tiles of 32 x 32. The functions
// are split into kGradSplit consecutive ranges, one CTA of a thread-block cluster each
// (the ranges streamed through shared memory 32 functions at a time, in order); the
// cluster's first CTA then adds the CTAs' partial tiles in rank order, read through
// distributed shared memory, so the sum does not depend on timing.
constexpr int kGradSplit = 8;
__global__ void __cluster_dims__(1, 1, kGradSplit) __launch_bounds__(256)
    boundary_grad_kernel(const float* __restrict__ S, const float* __restrict__ G, int F, int H,
                         float* __restrict__ gW0) {
  __shared__ float ss[32][33], sg[32][33];
  __shared__ float part[32 * 32];
  cg::cluster_group cluster = cg::this_cluster();
  const int tk = threadIdx.x & 31, tr = threadIdx.x >> 5;  // this thread: rows tr + 8 i, column tk
  const int j0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int per = ((F + kGradSplit - 1) / kGradSplit + 31) & ~31;
  const int fb = (int)cluster.block_rank() * per, fe = min(F, fb + per);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int f0 = fb; f0 < fe; f0 += 32) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = tr + 8 * i, f = f0 + r;
      ss[r][tk] = (f < fe && j0 + tk < H) ? S[(size_t)f * H + j0 + tk] : 0.f;
      sg[r][tk] = f < fe ? G[(size_t)f * kNB + k0 + tk] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
      const float gq = sg[q][tk];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fmaf(ss[q][tr + 8 * i], gq, acc[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) part[(tr + 8 * i) * 32 + tk] = acc[i];
  cluster.sync();
  if (cluster.block_rank() == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int jj = tr + 8 * i;
      float sum = 0.f;
      for (int c = 0; c < kGradSplit; ++c) sum += cluster.map_shared_rank(part, c)[jj * 32 + tk];
      if (j0 + jj < H) gW0[(size_t)(j0 + jj) * kLd0 + k0 + tk] += sum;
    }
  }
  cluster.sync();  // the partial tiles stay in place until the first CTA has read them
}

// Row products of the GEMM engine: out[r][n] = sum_k in[r][k] M[k][n], with M = W^T
// (forward, trans = 1: M[k][n] = W[n][k]) or M = W (backward to the activations,
// trans = 0). A block holds M (FP32, H x H) in shared memory and walks row tiles of
// kRowsT rows; 256 threads, each kRowsT/16 rows x H/16 columns of the tile.
constexpr int kRowsT = 64;
constexpr int kThreadsG = 256;

template <int H>
struct RowCfg {
  static constexpr int kPitch = H + 4;                 // padded row of the input tile
  static constexpr int kRowsPer = kRowsT / 16;         // rows per thread (4)
  static constexpr int kColsPer = H / 16;              // columns per thread (8 or 4)
  static constexpr size_t kSmem = (size_t)H * H * 4 + (size_t)kRowsT * kPitch * 4;
};

template <typename T, int H>
__global__ void __launch_bounds__(kThreadsG) row_gemm_kernel(const T* __restrict__ in, const T* __restrict__ W,
                                                             int trans, long rows, float* __restrict__ out) {
  using Cfg = RowCfg<H>;
  extern __shared__ __align__(16) float smem[];
  float* sM = smem;                 // [H k][H n]
  float* sX = smem + H * H;         // [kRowsT][kPitch]
  for (int i = threadIdx.x; i < H * H; i += kThreadsG) {
    const int k = i / H, n = i % H;
    sM[i] = widen<T>(trans ? W[(size_t)n * H + k] : W[(size_t)k * H + n]);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long tiles = (rows + kRowsT - 1) / kRowsT;
  for (long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const long r0 = t * kRowsT;
    __syncthreads();  // previous tile's reads of sX are done (and sM is written)
    for (int i = threadIdx.x; i < kRowsT * H; i += kThreadsG) {
      const int rr = i / H, k = i % H;
      const long r = r0 + rr;
      sX[rr * Cfg::kPitch + k] = r < rows ? widen<T>(in[(size_t)r * H + k]) : 0.f;
    }
    __syncthreads();
    float acc[Cfg::kRowsPer][Cfg::kColsPer];
#pragma unroll
    for (int i = 0; i < Cfg::kRowsPer; ++i)
#pragma unroll
      for (int c = 0; c < Cfg::kColsPer; ++c) acc[i][c] = 0.f;
    for (int k = 0; k < H; k += 4) {
      float a[Cfg::kRowsPer][4];
#pragma unroll
      for (int i = 0; i < Cfg::kRowsPer; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(sX + (ty * Cfg::kRowsPer + i) * Cfg::kPitch + k);
        a[i][0] = v.x; a[i][1] = v.y; a[i][2] = v.z; a[i][3] = v.w;
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        float b[Cfg::kColsPer];
#pragma unroll
        for (int c4 = 0; c4 < Cfg::kColsPer / 4; ++c4) {
          // columns tx*4 + 64*c4 .. +3: a warp reads 16 consecutive float4 (conflict-free)
          const float4 v = *reinterpret_cast<const float4*>(sM + (k + kk) * H + c4 * 64 + tx * 4);
          b[4 * c4] = v.x; b[4 * c4 + 1] = v.y; b[4 * c4 + 2] = v.z; b[4 * c4 + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < Cfg::kRowsPer; ++i)
#pragma unroll
          for (int c = 0; c < Cfg::kColsPer; ++c) acc[i][c] = fmaf(a[i][kk], b[c], acc[i][c]);
      }
    }
#pragma unroll
    for (int i = 0; i < Cfg::kRowsPer; ++i) {
      const long r = r0 + ty * Cfg::kRowsPer + i;
      if (r >= rows) continue;
#pragma unroll
      for (int c4 = 0; c4 < Cfg::kColsPer / 4; ++c4) {
        const float4 v = make_float4(acc[i][4 * c4], acc[i][4 * c4 + 1], acc[i][4 * c4 + 2], acc[i][4 * c4 + 3]);
        *reinterpret_cast<float4*>(out + (size_t)r * H + c4 * 64 + tx * 4) = v;
      }
    }
  }
}

// Weight gradient of the GEMM engine: part[b][n][k] = sum over the row tiles of block b
// (tiles b, b + gridDim.x, ...) of gZ[r][n] X[r][k]. Thread (tx, ty) owns outputs
// n = ty*4 + 64 c + {0..3}, k = tx*4 + 64 c' + {0..3} (H = 128: 8 x 8; H = 64: 4 x 4).
constexpr int kRowsW = 64;

template <int H>
struct WCfg {
  static constexpr int kPer = H / 16;  // outputs per thread along n and along k
  static constexpr size_t kSmem = (size_t)2 * kRowsW * H * 4;
};

template <typename T, int H>
__global__ void __launch_bounds__(kThreadsG) weight_grad_kernel(const T* __restrict__ gZ, const T* __restrict__ X,
                                                                long rows, float* __restrict__ part) {
  using Cfg = WCfg<H>;
  extern __shared__ __align__(16) float smem[];
  float* sZ = smem;                 // [kRowsW][H]
  float* sX = smem + kRowsW * H;    // [kRowsW][H]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[Cfg::kPer][Cfg::kPer];
#pragma unroll
  for (int i = 0; i < Cfg::kPer; ++i)
#pragma unroll
    for (int c = 0; c < Cfg::kPer; ++c) acc[i][c] = 0.f;
  const long tiles = (rows + kRowsW - 1) / kRowsW;
  for (long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const long r0 = t * kRowsW;
    __syncthreads();
    for (int i = threadIdx.x; i < kRowsW * H; i += kThreadsG) {
      const long r = r0 + i / H;
      const bool in = r < rows;
      sZ[i] = in ? widen<T>(gZ[(size_t)r0 * H + i]) : 0.f;
      sX[i] = in ? widen<T>(X[(size_t)r0 * H + i]) : 0.f;
    }
    __syncthreads();
    for (int rr = 0; rr < kRowsW; ++rr) {
      float a[Cfg::kPer], b[Cfg::kPer];
#pragma unroll
      for (int c4 = 0; c4 < Cfg::kPer / 4; ++c4) {
        const float4 va = *reinterpret_cast<const float4*>(sZ + rr * H + c4 * 64 + ty * 4);
        const float4 vb = *reinterpret_cast<const float4*>(sX + rr * H + c4 * 64 + tx * 4);
        a[4 * c4] = va.x; a[4 * c4 + 1] = va.y; a[4 * c4 + 2] = va.z; a[4 * c4 + 3] = va.w;
        b[4 * c4] = vb.x; b[4 * c4 + 1] = vb.y; b[4 * c4 + 2] = vb.z; b[4 * c4 + 3] = vb.w;
      }
#pragma unroll
      for (int i = 0; i < Cfg::kPer; ++i)
#pragma unroll
        for (int c = 0; c < Cfg::kPer; ++c) acc[i][c] = fmaf(a[i], b[c], acc[i][c]);
    }
  }
  float* p = part + (size_t)blockIdx.x * H * H;
#pragma unroll
  for (int i = 0; i < Cfg::kPer; ++i) {
    const int n = (i / 4) * 64 + ty * 4 + (i % 4);
#pragma unroll
    for (int c4 = 0; c4 < Cfg::kPer / 4; ++c4) {
      const float4 v = make_float4(acc[i][4 * c4], acc[i][4 * c4 + 1], acc[i][4 * c4 + 2], acc[i][4 * c4 + 3]);
      *reinterpret_cast<float4*>(p + (size_t)n * H + c4 * 64 + tx * 4) = v;
    }
  }
}

// out[i] += sum over b < nblk of part[b][i], for i < n, in the order of b.
__global__ void add_partials_kernel(const float* __restrict__ part, int nblk, size_t n, float* __restrict__ out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * n + i];
  out[i] += s;
}

template <typename T, int H>
cudaError_t launch_row(const void* in, const void* W, int trans, long rows, float* out, cudaStream_t st) {
  static PerDevice pd;
  int grid_cap = 0;
  cudaError_t e = per_device(pd, [](int dev, int* cap, size_t*) {
    cudaError_t e1 = cudaFuncSetAttribute(row_gemm_kernel<T, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)RowCfg<H>::kSmem);
    if (e1 != cudaSuccess) return e1;
    int sms = 0, per_sm = 0;
    e1 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e1 != cudaSuccess) return e1;
    e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, row_gemm_kernel<T, H>, kThreadsG, RowCfg<H>::kSmem);
    if (e1 != cudaSuccess) return e1;
    *cap = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
  }, &grid_cap);
  if (e != cudaSuccess) return e;
  const long tiles = (rows + kRowsT - 1) / kRowsT;
  if (tiles == 0) return cudaSuccess;
  const int grid = (int)(tiles < grid_cap ? tiles : grid_cap);
  row_gemm_kernel<T, H><<<grid, kThreadsG, RowCfg<H>::kSmem, st>>>(static_cast<const T*>(in),
                                                                   static_cast<const T*>(W), trans, rows, out);
  return cudaGetLastError();
}

template <typename T, int H>
cudaError_t launch_wgrad(const void* gZ, const void* X, long rows, float* part, int nblk, float* gW, cudaStream_t st) {
  static PerDevice pd;
  cudaError_t e = per_device(pd, [](int, int*, size_t*) {
    return cudaFuncSetAttribute(weight_grad_kernel<T, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)WCfg<H>::kSmem);
  });
  if (e != cudaSuccess) return e;
  if (rows <= 0) return cudaSuccess;
  weight_grad_kernel<T, H><<<nblk, kThreadsG, WCfg<H>::kSmem, st>>>(static_cast<const T*>(gZ),
                                                                    static_cast<const T*>(X), rows, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t n = (size_t)H * H;
  add_partials_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, nblk, n, gW);
  return cudaGetLastError();
}

}  // namespace

cudaError_t train_boundary_fwd(const float* W0, const float* G, int F, int H, float* Bf, cudaStream_t st) {
  if (F <= 0) return cudaSuccess;
  if (H != 64 && H != 128) return cudaErrorInvalidValue;
  boundary_fwd_kernel<<<(F + kGF - 1) / kGF, 128, 0, st>>>(W0, G, F, H, Bf);
  return cudaGetLastError();
}

cudaError_t train_boundary_grad(const float* S, const float* G, int F, int H, float* gW0, cudaStream_t st) {
  if (F <= 0) return cudaSuccess;
  if (H != 64 && H != 128) return cudaErrorInvalidValue;
  boundary_grad_kernel<<<dim3(H / 32, kNB / 32, kGradSplit), 256, 0, st>>>(S, G, F, H, gW0);
  return cudaGetLastError();
}

int train_wgrad_blocks() {
  int sms = 0;
  if (device_sms(&sms) != cudaSuccess || sms < 1) sms = 1;
  return 2 * sms;
}

cudaError_t train_row_gemm(int bf16, int H, const void* in, const void* W, int trans, long rows, float* out,
                           cudaStream_t st) {
  if (H == 128)
    return bf16 ? launch_row<__nv_bfloat16, 128>(in, W, trans, rows, out, st)
                : launch_row<float, 128>(in, W, trans, rows, out, st);
  if (H == 64)
    return bf16 ? launch_row<__nv_bfloat16, 64>(in, W, trans, rows, out, st)
                : launch_row<float, 64>(in, W, trans, rows, out, st);
  return cudaErrorInvalidValue;
}

cudaError_t train_weight_grad(int bf16, int H, const void* gZ, const void* X, long rows, float* part, int nblk,
                              float* gW, cudaStream_t st) {
  if (nblk < 1) return cudaErrorInvalidValue;
  if (H == 128)
    return bf16 ? launch_wgrad<__nv_bfloat16, 128>(gZ, X, rows, part, nblk, gW, st)
                : launch_wgrad<float, 128>(gZ, X, rows, part, nblk, gW, st);
  if (H == 64)
    return bf16 ? launch_wgrad<__nv_bfloat16, 64>(gZ, X, rows, part, nblk, gW, st)
                : launch_wgrad<float, 64>(gZ, X, rows, part, nblk, gW, st);
  return cudaErrorInvalidValue;
}

}  // namespace mf
