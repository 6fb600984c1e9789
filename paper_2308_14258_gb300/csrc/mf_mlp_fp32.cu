// K3f: FP32 SDNet over one colour, fused with the scatter into the grid.
//
// Rows r = (subdomain s, interior point p) of the colour are processed in tiles of 128.
// Per row the first layer is the input-split form of Eq. 8: tanh(B[s] + W2 x_p), with
// B[s] = W1 g_s + b0 from K1; then depth-1 hidden layers act(W h + b) and the linear
// output w_out . h + b_out (Section 3.1-3.2; act = tanh, or GELU for the variant). Activations stay in
// shared memory k-major (act[k][row]); each hidden layer is a 128 x H x H SIMT GEMM
// with an 8 x (H/16) register tile per thread, its weights streamed from L2 with
// cp.async into a double buffer while the previous layer computes. tanh is CUDA's
// accurate tanhf and GELU uses erff (no approximate hardware tanh), which keeps this
// path within 1e-5 of the FP64 oracle. The prediction of each row is written to its grid point (store for
// the multiplicative schedule, weighted add for the additive one).
#include "mf_internal.cuh"

namespace mf {

namespace {

constexpr int kThreads = 256;
constexpr int kTR = kTileRows;   // 128 rows per tile
constexpr int kLda = kTR + 4;    // act row stride (floats)

template <int H>
struct Fp32Cfg {
  static constexpr int kLdw = H + 4;                  // weight row stride (floats)
  static constexpr int kCG = H / 64 > 0 ? H / 64 : 1; // float4 column groups per thread
  static constexpr int kCols = H / 16;                // columns per thread
  static constexpr size_t kSmem = (size_t)(H * kLda + 2 * H * kLdw + 2 * kTR) * sizeof(float);
};

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Weights of hidden layer l, transposed (k-major, WhT[l][k][n]), into padded smem rows.
template <int H>
__device__ __forceinline__ void load_layer(float* dst, const float* __restrict__ WhT, int l) {
  const float* src = WhT + (size_t)l * H * H;
  constexpr int kChunks = H * H / 4;
  for (int c = threadIdx.x; c < kChunks; c += kThreads) {
    const int k = c / (H / 4), n4 = c % (H / 4);
    cp_async16(dst + k * Fp32Cfg<H>::kLdw + 4 * n4, src + (size_t)k * H + 4 * n4);
  }
}

template <int H, int ACT>
__global__ void __launch_bounds__(kThreads)
mlp_fp32_kernel(const float* __restrict__ B, ColourGeom g, int n_rows, const float* __restrict__ W2,
                const float* __restrict__ WhT, const float* __restrict__ bh, const float* __restrict__ wout,
                float bout, int n_hidden, float* __restrict__ u, int additive) {
  using C = Fp32Cfg<H>;
  extern __shared__ float4 smem4[];
  float* act = reinterpret_cast<float*>(smem4);  // [H][kLda]
  float* wbuf0 = act + H * kLda;                 // [H][kLdw]
  float* wbuf1 = wbuf0 + H * C::kLdw;
  float* red = wbuf1 + H * C::kLdw;              // [2][kTR]

  const int row0 = blockIdx.x * kTR;
  const int t = threadIdx.x;

  if (n_hidden > 0) load_layer<H>(wbuf0, WhT, 0);
  cp_async_commit();

  // First layer (Eq. 8): act[k][r] = tanh(B[s][k] + W2[k][0] x + W2[k][1] y).
  {
    const int r = t & (kTR - 1), half = t >> 7;
    const int row = min(row0 + r, n_rows - 1);
    const RowSite site = row_site(g, row);
    const float x = (float)(site.px + 1) * (1.0f / kPts), y = (float)(site.py + 1) * (1.0f / kPts);
    const float* Bs = B + (size_t)site.s * H;
    for (int k = half; k < H; k += 2) {
      const float2 w = __ldg(reinterpret_cast<const float2*>(W2) + k);
      act[k * kLda + r] = act_exact<ACT>(fmaf(w.y, y, fmaf(w.x, x, __ldg(Bs + k))));
    }
  }

  const int tn = t & 15, tr = t >> 4;
  for (int l = 0; l < n_hidden; ++l) {
    float* wcur = (l & 1) ? wbuf1 : wbuf0;
    if (l + 1 < n_hidden) load_layer<H>((l & 1) ? wbuf0 : wbuf1, WhT, l + 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    float acc[8][C::kCols];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < C::kCols; ++j) acc[i][j] = 0.f;

#pragma unroll 4
    for (int k = 0; k < H; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(act + k * kLda + 4 * tr);
      const float4 a1 = *reinterpret_cast<const float4*>(act + k * kLda + 64 + 4 * tr);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float w[C::kCols];
#pragma unroll
      for (int cg = 0; cg < C::kCG; ++cg) {
        const float4 wv = *reinterpret_cast<const float4*>(wcur + k * C::kLdw + 64 * cg + 4 * tn);
        w[4 * cg + 0] = wv.x; w[4 * cg + 1] = wv.y; w[4 * cg + 2] = wv.z; w[4 * cg + 3] = wv.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < C::kCols; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    __syncthreads();  // every thread has finished reading act

    const float* bl = bh + (size_t)l * H;
#pragma unroll
    for (int cg = 0; cg < C::kCG; ++cg)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = 64 * cg + 4 * tn + j;
        const float bn = __ldg(bl + n);
#pragma unroll
        for (int rg = 0; rg < 2; ++rg) {
          float4 v;
          v.x = act_exact<ACT>(acc[4 * rg + 0][4 * cg + j] + bn);
          v.y = act_exact<ACT>(acc[4 * rg + 1][4 * cg + j] + bn);
          v.z = act_exact<ACT>(acc[4 * rg + 2][4 * cg + j] + bn);
          v.w = act_exact<ACT>(acc[4 * rg + 3][4 * cg + j] + bn);
          *reinterpret_cast<float4*>(act + n * kLda + 64 * rg + 4 * tr) = v;
        }
      }
  }
  cp_async_wait<0>();
  __syncthreads();

  // Output layer: u = w_out . h + b_out, two half-sums per row folded in a fixed order.
  {
    const int r = t & (kTR - 1), half = t >> 7;
    float s = 0.f;
    for (int k = half * (H / 2); k < (half + 1) * (H / 2); ++k) s = fmaf(act[k * kLda + r], __ldg(wout + k), s);
    red[half * kTR + r] = s;
  }
  __syncthreads();
  if (t < kTR) {
    const int row = row0 + t;
    if (row < n_rows) {
      const float val = red[t] + red[kTR + t] + bout;
      const RowSite site = row_site(g, row);
      if (additive)
        u[site.idx] += cover_weight(g, site.ix, site.iy) * val;
      else
        u[site.idx] = val;
    }
  }
}

template <int H, int ACT>
cudaError_t launch_h(const float* B, const ColourGeom& g, const DevNet& net, float* u, int additive,
                     cudaStream_t st) {
  const int n_rows = g.n_c * g.rows_per_sub;
  const int tiles = (n_rows + kTR - 1) / kTR;
  const size_t smem = Fp32Cfg<H>::kSmem;
  static PerDevice pd;
  cudaError_t e = per_device(pd, [smem](int, int*, size_t*) {
    return cudaFuncSetAttribute(mlp_fp32_kernel<H, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  mlp_fp32_kernel<H, ACT><<<tiles, kThreads, smem, st>>>(B, g, n_rows, net.W2, net.WhT, net.bh, net.wout, net.bout,
                                                     net.n_hidden, u, additive);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mlp_fp32(const float* B, const ColourGeom& g, const DevNet& net, float* u, int additive,
                            cudaStream_t st) {
  if (g.n_c <= 0) return cudaSuccess;
  if (net.act == kActGelu)
    return net.width == 128 ? launch_h<128, kActGelu>(B, g, net, u, additive, st)
                            : launch_h<64, kActGelu>(B, g, net, u, additive, st);
  return net.width == 128 ? launch_h<128, kActTanh>(B, g, net, u, additive, st)
                          : launch_h<64, kActTanh>(B, g, net, u, additive, st);
}

}  // namespace mf
