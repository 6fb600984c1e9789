// K0 grid set-up and K1 boundary gather + per-subdomain first-layer term (with the
// conv1d boundary embedding of the SDNet variant when the network has one).
//
// K1 reads, for every subdomain of one colour, its 128 boundary values from the global
// grid (the in-device form of Algorithm 2's boundary exchange) and forms the left
// operand of the input-split first layer (Eq. 8): B[s][:] = W1 g_s + b0, with W1 the
// boundary block of the first-layer weights. The per-point coordinate term X W2^T is
// added later, per row, inside the MLP kernels, so the boundary GEMM runs once per
// subdomain instead of once per point (Section 3.2).
#include "mf_internal.cuh"

namespace mf {

namespace {

constexpr int kGatherThreads = 256;

// kSubPerBlock subdomains per block (4, 8 or 16; the default 16 has each warp gather
// two): fewer per block spread a small colour over more SMs, more per block share each
// weight load among more subdomains. W1 (128 x H FP32) is staged in shared memory with
// 16-byte loads issued all at once: read straight from L2 inside the product loop, a
// few loads in flight per thread left the kernel latency-bound.
template <int H, int kSubPerBlock>
__global__ void __launch_bounds__(kGatherThreads)
gather_boundary_kernel(const float* __restrict__ u, ColourGeom g, const float* __restrict__ W1t,
                       const float* __restrict__ b0, float* __restrict__ B) {
  __shared__ __align__(16) float gs[kSubPerBlock][kNbdry];
  extern __shared__ float4 w1s4[];  // [128][H / 4]
  const float* w1s = reinterpret_cast<const float*>(w1s4);
  const int s0 = blockIdx.x * kSubPerBlock;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    constexpr int kVec = kNbdry * H / 4;
    const float4* src = reinterpret_cast<const float4*>(W1t);
#pragma unroll
    for (int i = 0; i < kVec / kGatherThreads; ++i) w1s4[threadIdx.x + i * kGatherThreads] = __ldg(src + threadIdx.x + i * kGatherThreads);
  }

  // Gather: bottom and top strips are 32 consecutive floats (one 128-byte coalesced
  // request per warp); the left and right strips are one value per grid row.
  for (int i = warp; i < kSubPerBlock; i += kGatherThreads / 32) {
    const int s = s0 + i;
    if (s < g.n_c) {
      const size_t nx = sub_stride(g, s);
      const float* o = u + sub_point(g, s, 0, 0);
      gs[i][lane] = __ldg(o + lane);                                   // (lane, 0)
      gs[i][32 + lane] = __ldg(o + (size_t)lane * nx + kPts);          // (32, lane)
      gs[i][64 + lane] = __ldg(o + (size_t)kPts * nx + (kPts - lane)); // (32 - lane, 32)
      gs[i][96 + lane] = __ldg(o + (size_t)(kPts - lane) * nx);        // (0, 32 - lane)
    } else {
      gs[i][lane] = gs[i][32 + lane] = gs[i][64 + lane] = gs[i][96 + lane] = 0.f;
    }
  }
  __syncthreads();

  // B[s][j] = sum_k W1[j][k] g_s[k] + b0[j]; W1t is k-major so the weight reads of a
  // warp are one contiguous row segment.
  constexpr int kGroups = kGatherThreads / H;
  constexpr int kPer = kSubPerBlock / kGroups > 0 ? kSubPerBlock / kGroups : 1;
  const int j = threadIdx.x % H, grp = threadIdx.x / H;
  float acc[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) acc[i] = 0.f;
  // four boundary values of a subdomain per shared-memory read (the sum still runs over k
  // in order)
#pragma unroll 2
  for (int k = 0; k < kNbdry; k += 4) {
    const float w0 = w1s[k * H + j], w1 = w1s[(k + 1) * H + j];
    const float w2 = w1s[(k + 2) * H + j], w3 = w1s[(k + 3) * H + j];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int sl = grp + i * kGroups;
      if (sl < kSubPerBlock) {
        const float4 g4 = *reinterpret_cast<const float4*>(&gs[sl][k]);
        acc[i] = fmaf(w0, g4.x, acc[i]);
        acc[i] = fmaf(w1, g4.y, acc[i]);
        acc[i] = fmaf(w2, g4.z, acc[i]);
        acc[i] = fmaf(w3, g4.w, acc[i]);
      }
    }
  }
  const float bj = __ldg(b0 + j);
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int sl = grp + i * kGroups, s = s0 + sl;
    if (sl < kSubPerBlock && s < g.n_c) B[(size_t)s * H + j] = acc[i] + bj;
  }
}

// K1 for the SDNet variant with a boundary embedding (Section 3.1): the 128 boundary
// values of a subdomain, taken as a closed curve, pass through two circular conv1d
// layers (1 -> C channels at stride 1, then C -> C at stride 2, kernel K, each followed
// by the network's activation); the C x 64 outputs z, channel-major, give
// B[s][j] = sum_e W1[j][e] z[e] + b0[j]. Four subdomains per block; everything in FP32.
constexpr int kEmbedThreads = 256;
constexpr int kEmbedSubs = 4;

__host__ __device__ constexpr int embed_floats_per_sub(int C) { return kNbdry + C * kNbdry + C * (kNbdry / 2); }

template <int H, int ACT>
__global__ void __launch_bounds__(kEmbedThreads)
embed_boundary_kernel(const float* __restrict__ u, ColourGeom g, const float* __restrict__ cw1,
                      const float* __restrict__ cb1, const float* __restrict__ cw2, const float* __restrict__ cb2,
                      int C, int K, const float* __restrict__ W1t, const float* __restrict__ b0,
                      float* __restrict__ B) {
  extern __shared__ float sm[];  // per subdomain: g[128] | h1[C][128] | z = h2[C][64]
  const int per = embed_floats_per_sub(C);
  const int s0 = blockIdx.x * kEmbedSubs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < kEmbedSubs) {
    float* gs = sm + warp * per;
    const int s = s0 + warp;
    if (s < g.n_c) {
      const size_t nx = sub_stride(g, s);
      const float* o = u + sub_point(g, s, 0, 0);
      gs[lane] = __ldg(o + lane);
      gs[32 + lane] = __ldg(o + (size_t)lane * nx + kPts);
      gs[64 + lane] = __ldg(o + (size_t)kPts * nx + (kPts - lane));
      gs[96 + lane] = __ldg(o + (size_t)(kPts - lane) * nx);
    } else {
      gs[lane] = gs[32 + lane] = gs[64 + lane] = gs[96 + lane] = 0.f;
    }
  }
  __syncthreads();
  const int half = K / 2;
  // conv 1: h1[c][i] = act(cb1[c] + sum_t cw1[c][t] g[(i + t - K/2) mod 128])
  for (int idx = threadIdx.x; idx < kEmbedSubs * C * kNbdry; idx += kEmbedThreads) {
    const int i = idx & (kNbdry - 1), row = idx >> 7, c = row % C, sub = row / C;
    const float* gs = sm + sub * per;
    float acc = __ldg(cb1 + c);
    for (int t = 0; t < K; ++t) acc = fmaf(__ldg(cw1 + c * K + t), gs[(i + t - half + kNbdry) & (kNbdry - 1)], acc);
    sm[sub * per + kNbdry + c * kNbdry + i] = act_exact<ACT>(acc);
  }
  __syncthreads();
  // conv 2, stride 2: z[c][i] = act(cb2[c] + sum_{c',t} cw2[c][c'][t] h1[c'][(2i + t - K/2) mod 128])
  for (int idx = threadIdx.x; idx < kEmbedSubs * C * (kNbdry / 2); idx += kEmbedThreads) {
    const int i = idx & (kNbdry / 2 - 1), row = idx >> 6, c = row % C, sub = row / C;
    const float* h1 = sm + sub * per + kNbdry;
    float acc = __ldg(cb2 + c);
    for (int cp = 0; cp < C; ++cp) {
      const float* wr = cw2 + (size_t)(c * C + cp) * K;
      const float* hr = h1 + cp * kNbdry;
      for (int t = 0; t < K; ++t) acc = fmaf(__ldg(wr + t), hr[(2 * i + t - half + kNbdry) & (kNbdry - 1)], acc);
    }
    sm[sub * per + kNbdry + C * kNbdry + c * (kNbdry / 2) + i] = act_exact<ACT>(acc);
  }
  __syncthreads();
  // B[s][j] = sum_e W1t[e][j] z[e] + b0[j]
  constexpr int kGroups = kEmbedThreads / H;
  const int j = threadIdx.x % H, grp = threadIdx.x / H;
  const int n_in = C * (kNbdry / 2);
  for (int sub = grp; sub < kEmbedSubs; sub += kGroups) {
    const float* z = sm + sub * per + kNbdry + C * kNbdry;
    float acc = 0.f;
    for (int e = 0; e < n_in; ++e) acc = fmaf(__ldg(W1t + (size_t)e * H + j), z[e], acc);
    const int s = s0 + sub;
    if (s < g.n_c) B[(size_t)s * H + j] = acc + __ldg(b0 + j);
  }
}

template <int H, int ACT>
cudaError_t launch_embed(const float* u, const ColourGeom& g, const DevNet& net, float* B, cudaStream_t st) {
  const size_t smem = (size_t)kEmbedSubs * embed_floats_per_sub(net.embed_c) * sizeof(float);
  static PerDevice pd;
  cudaError_t e = per_device(pd, [](int, int*, size_t*) {
    const int max_smem = kEmbedSubs * embed_floats_per_sub(kMaxEmbedC) * (int)sizeof(float);
    return cudaFuncSetAttribute(embed_boundary_kernel<H, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  });
  if (e != cudaSuccess) return e;
  const int blocks = (g.n_c + kEmbedSubs - 1) / kEmbedSubs;
  embed_boundary_kernel<H, ACT><<<blocks, kEmbedThreads, smem, st>>>(u, g, net.cw1, net.cb1, net.cw2, net.cb2,
                                                                      net.embed_c, net.embed_k, net.W1t, net.b0, B);
  return cudaGetLastError();
}

// K0: boundary from the CCW Dirichlet list (rounded to FP32), interior zero.
__global__ void init_grid_kernel(float* __restrict__ u, int nx, int ny, const double* __restrict__ bc) {
  const size_t n = (size_t)nx * ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int iy = (int)(i / nx), ix = (int)(i % nx);
    float v = 0.f;
    if (iy == 0) {
      v = (float)bc[ix == nx - 1 ? (nx - 1) : ix];             // bottom, corner (nx-1,0) starts the right edge
    } else if (ix == nx - 1) {
      v = (float)bc[(nx - 1) + (iy == ny - 1 ? (ny - 1) : iy)]; // right, corner (nx-1,ny-1) starts the top
    } else if (iy == ny - 1) {
      v = (float)bc[(nx - 1) + (ny - 1) + (nx - 1 - ix)];       // top, ix = nx-1..1
    } else if (ix == 0) {
      v = (float)bc[2 * (nx - 1) + (ny - 1) + (ny - 1 - iy)];   // left, iy = ny-1..1
    }
    u[i] = v;
  }
}

__global__ void zero_interior_kernel(float* __restrict__ u, int nx, int ny) {
  const int mx = nx - 2;
  const size_t n = (size_t)mx * (ny - 2);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t iy = 1 + i / mx, ix = 1 + i % mx;
    u[iy * nx + ix] = 0.f;
  }
}

}  // namespace

template <int H>
cudaError_t launch_gather_h(const float* u, const ColourGeom& g, const DevNet& net, float* B, int subs,
                            cudaStream_t st) {
  constexpr size_t kW1Bytes = (size_t)kNbdry * H * sizeof(float);  // staged W1 (64 KB at H = 128)
  static PerDevice pd;
  cudaError_t e = per_device(pd, [](int, int*, size_t*) {
    cudaError_t e1 = cudaFuncSetAttribute(gather_boundary_kernel<H, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kW1Bytes);
    if (e1 == cudaSuccess)
      e1 = cudaFuncSetAttribute(gather_boundary_kernel<H, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kW1Bytes);
    if (e1 == cudaSuccess)
      e1 = cudaFuncSetAttribute(gather_boundary_kernel<H, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kW1Bytes);
    return e1;
  });
  if (e != cudaSuccess) return e;
  const int blocks = (g.n_c + subs - 1) / subs;
  switch (subs) {
    case 4: gather_boundary_kernel<H, 4><<<blocks, kGatherThreads, kW1Bytes, st>>>(u, g, net.W1t, net.b0, B); break;
    case 8: gather_boundary_kernel<H, 8><<<blocks, kGatherThreads, kW1Bytes, st>>>(u, g, net.W1t, net.b0, B); break;
    case 16:
      gather_boundary_kernel<H, 16><<<blocks, kGatherThreads, kW1Bytes, st>>>(u, g, net.W1t, net.b0, B);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_boundary(const float* u, const ColourGeom& g, const DevNet& net, float* B,
                                   cudaStream_t st, int subs_per_block) {
  if (g.n_c <= 0) return cudaSuccess;
  if (net.embed_c > 0) {
    if (net.width == 128)
      return net.act == kActGelu ? launch_embed<128, kActGelu>(u, g, net, B, st) : launch_embed<128, kActTanh>(u, g, net, B, st);
    return net.act == kActGelu ? launch_embed<64, kActGelu>(u, g, net, B, st) : launch_embed<64, kActTanh>(u, g, net, B, st);
  }
  return net.width == 128 ? launch_gather_h<128>(u, g, net, B, subs_per_block, st)
                          : launch_gather_h<64>(u, g, net, B, subs_per_block, st);
}

cudaError_t launch_init_grid(float* u, int nx, int ny, const double* bc, cudaStream_t st) {
  const size_t n = (size_t)nx * ny;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  init_grid_kernel<<<blocks, 256, 0, st>>>(u, nx, ny, bc);
  return cudaGetLastError();
}

cudaError_t launch_zero_interior(float* u, int nx, int ny, cudaStream_t st) {
  const size_t n = (size_t)(nx - 2) * (ny - 2);
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  zero_interior_kernel<<<blocks, 256, 0, st>>>(u, nx, ny);
  return cudaGetLastError();
}

}  // namespace mf
