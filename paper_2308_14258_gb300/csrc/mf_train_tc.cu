// K7-K8 on the tensor cores: fused Taylor-mode layer kernels of the physics-informed
// training step (Eq. 3, Algorithm 1), BF16 operands with FP32 accumulators, width 128.
//
// Orientation. A layer computes Z^T = W A^T with M = 128 output features (TMEM lanes)
// and N = 64 GEMM rows of a tile: the four Taylor channels (value, d/dx, d/dy, Delta) of
// 16 points, or 64 points of the value channel alone. Each epilogue thread then owns one
// feature and holds every channel of its points, which is what the chain rules of the
// Taylor-mode tanh need (see mf_train.cu for the formulas).
//
// Activations and their gradients travel between layers in HBM as BF16 tiles of 64
// GEMM rows x 128 features, 16 KB each, stored feature-major: feature k owns 128 bytes
// (its 64 rows, row r = channel x (points per tile) + point), 16-byte chunk c (rows
// 8c..8c+7) at chunk c ^ (k mod 8). This is byte for byte the 128-byte-swizzled operand
// layout, so one bulk copy loads a tile that the MMAs read directly: as an MN-major
// operand with N = rows and K = features (Z = W A^T, and gA^T = W^T g_Z^T), or as a
// K-major operand with N = features and K = rows (g_W = g_Z^T A). An epilogue thread owns
// one feature and so reads and writes its 128 bytes with 16-byte accesses.
//
// Forward kernel (hidden layers 1..NH-1): load tile A_{l-1}; MMA into TMEM; epilogue
// applies the Taylor-mode tanh and writes tile A_l. Pre-activations are never stored.
// Backward kernel (hidden layer l, top = l == NH): load A_{l-1} and (below the top) the
// incoming gradient tile gA_l; MMA 1 recomputes Z^T; epilogue 1 forms g_z for every
// channel (the top layer first folds the output layer and the loss in); MMA 2 gives
// gA_{l-1}^T = W^T g_Z^T and MMA 3 accumulates g_W += g_Z^T A_{l-1} in TMEM over all tiles
// of the CTA, both from the one g_Z^T tile the epilogue writes; epilogue 2 writes tile
// gA_{l-1}. The recompute MMA of the next tile is issued before MMAs 2 and 3 of the
// current one, so it runs while epilogue 1 works.
// Per-CTA partial sums of g_W, g_b (and of the output-layer gradient and the loss at the
// top) go to global memory and are added up in a fixed order afterwards, so results do
// not depend on timing.
//
// Roles per CTA (persistent, one CTA per SM, static tile schedule t = CTA + i x CTAs;
// the forward keeps four input tiles in flight, the backward two): warp 0 lane 0 issues
// the MMAs, warp 1 lane 0 issues the bulk loads, warps 2-9 are the epilogue (feature
// quadrant q = w mod 4, the TMEM lanes warp w may read; point half (w-2)/4). Every wait
// is bounded (mf_wait.cuh);
// after an abort the epilogue warps keep stepping through their loop without work, so
// that every named barrier is reached by every warp, and the CTA drains its MMAs and
// bulk copies before it frees TMEM and exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mf_internal.cuh"
#include "mf_tc.cuh"
#include "mf_train_tc.cuh"
#include "mf_wait.cuh"

namespace mf {

namespace {

constexpr int kW = 128;                        // width H on the fused path
constexpr int kTR = 64;                        // GEMM rows per tile
constexpr uint32_t kTile = kTR * kW * 2;       // 16 KB
constexpr uint32_t kWImg = kW * kW * 2;        // 32 KB
constexpr int kEpi = 8;                        // epilogue warps
constexpr int kThreadsTc = (2 + kEpi) * 32;    // MMA warp, load warp, epilogue
constexpr int kStagesF = 8;                    // input tiles in flight per CTA (forward)
constexpr uint32_t kIdescRows = idesc_bf16_bmn(128, kTR);  // B = tile, N = rows (MN-major)
constexpr uint32_t kIdescGW = idesc_bf16(128, kW);          // B = tile, N = features (K-major)

// Byte offset of the 16-byte chunk holding rows 8c..8c+7 of feature k in a tile.
__host__ __device__ __forceinline__ uint32_t tile_chunk(int k, int c) {
  return (uint32_t)k * 128u + ((uint32_t)(c ^ (k & 7)) << 4);
}
// K-step ks (features 16ks..16ks+15) of a tile read MN-major (N = 64 rows = one atom).
__device__ __forceinline__ uint64_t desc_rows(uint32_t tile, int ks) {
  return desc_sw128_mn(tile + (uint32_t)ks * 2048u, 8192u, 1024u);
}

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
               : "memory");
  return v;
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16);
}
// the 8 BF16 values of a chunk as floats
__device__ __forceinline__ void unpack8(uint4 v, float* f) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// a = tanh z and s = 1 - a^2 from e = exp(-2|z|): a = sign(z) (1 - e)/(1 + e) and
// s = 4 e / (1 + e)^2, which keeps s accurate relative to itself where |a| is near 1.
__device__ __forceinline__ void tanh_sech2(float z, float& a, float& s) {
  const float e = ex2_approx(-2.8853900817779268f * fabsf(z));  // 2 / ln 2
  const float r = rcp_approx(1.0f + e);
  a = copysignf((1.0f - e) * r, z);
  s = 4.0f * e * r * r;
}

// Columns [16 cq, 16 cq + 16) of this warp's 32 TMEM lanes <- K elements [32 cq, 32 cq + 32)
// of rows 32 q .. 32 q + 31 of a 128 x 128 BF16 image in the K-major 128-byte-swizzled
// layout (global memory): the A operand of tcgen05.mma held in tensor memory.
__device__ __forceinline__ void weights_to_tmem(const uint8_t* __restrict__ img, uint32_t tcol, int q, int lane,
                                                int cq) {
  const int row = 32 * q + lane;
  uint32_t v[16];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int chunk = (cq & 1) * 4 + c;
    const uint4 w = *reinterpret_cast<const uint4*>(img + (size_t)(cq >> 1) * 16384 + (size_t)row * 128 +
                                                    ((uint32_t)(chunk ^ (row & 7)) << 4));
    v[4 * c] = w.x; v[4 * c + 1] = w.y; v[4 * c + 2] = w.z; v[4 * c + 3] = w.w;
  }
  tmem_st16(tcol + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * cq), v);
}

// Points and GEMM rows of a tile for C channels.
__device__ __forceinline__ int pts_per_tile(int C) { return kTR / C; }

struct Smem {
  uint32_t base;
  __device__ uint32_t bar(int i) const { return base + 8u * (uint32_t)i; }
};

// ------------------------------------------------------------------ forward kernel

// barriers: 1+s in_full[s]; 9+s in_empty[s]; 17+b acc_full[b]; 19+b acc_empty[b]; 21 drain
constexpr int kFwdBars = 22;
enum { kFInF = 1, kFInE = 9, kFAccF = 17, kFAccE = 19, kFDrain = 21 };

__global__ void __launch_bounds__(kThreadsTc, 1) tc_fwd_kernel(const __grid_constant__ TcFwdParams P) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen = smem_raw + (base - raw);
  const uint32_t sIn = base;                             // kStagesF tiles
  const uint32_t sOut = sIn + kStagesF * kTile;          // 2 staging tiles
  const uint32_t sBar = sOut + 2 * kTile;
  Smem S{sBar};
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gen + (sBar - base) + 8 * kFwdBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gen + (sBar - base) + 8 * kFwdBars + 8);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = P.C, PT = pts_per_tile(C);
  const int n_it = P.n_tiles > (int)blockIdx.x ? (P.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesF; ++s) { mbar_init(S.bar(kFInF + s), 1); mbar_init(S.bar(kFInE + s), 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(S.bar(kFAccF + b), 1); mbar_init(S.bar(kFAccE + b), kEpi); }
    mbar_init(S.bar(kFDrain), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_addr(tmem_holder), 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  // TMEM columns: accumulators [0, 128) (two buffers of 64), W as the A operand [128, 192)
  const uint32_t Wt = tmem + 128;
  if (warp >= 2) {
    const int e = warp - 2;
    weights_to_tmem(static_cast<const uint8_t*>(P.wimg), Wt, warp & 3, lane, 2 * (e >> 2));
    weights_to_tmem(static_cast<const uint8_t*>(P.wimg), Wt, warp & 3, lane, 2 * (e >> 2) + 1);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      for (int it = 0; ok && it < n_it; ++it) {
        const int s = it % kStagesF, b = it & 1;
        ok = wait_spin(S.bar(kFInF + s), (uint32_t)((it / kStagesF) & 1), abort_flag, P.status);
        if (ok && it >= 2) ok = wait_spin(S.bar(kFAccE + b), (uint32_t)(((it >> 1) - 1) & 1), abort_flag, P.status);
        if (!ok) break;
        tc_fence_after();
        const uint32_t tin = sIn + (uint32_t)s * kTile;
        const uint32_t acc = tmem + (uint32_t)(b * kTR);
#pragma unroll
        for (int ks = 0; ks < kW / 16; ++ks) {
          if (ks == 0) mma_ts<0>(acc, Wt + (uint32_t)(8 * ks), desc_rows(tin, ks), kIdescRows);
          else mma_ts<1>(acc, Wt + (uint32_t)(8 * ks), desc_rows(tin, ks), kIdescRows);
        }
        mma_commit(S.bar(kFAccF + b));
        mma_commit(S.bar(kFInE + s));
      }
      mma_commit(S.bar(kFDrain));
      wait_bounded(S.bar(kFDrain), 0, abort_flag, P.status, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < n_it; ++it) {
        const int s = it % kStagesF;
        if (it >= kStagesF &&
            !wait_bounded(S.bar(kFInE + s), (uint32_t)(((it / kStagesF) - 1) & 1), abort_flag, P.status, true))
          break;
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        mbar_arrive_expect_tx(S.bar(kFInF + s), kTile);
        bulk_g2s(sIn + (uint32_t)s * kTile, P.A_in + (size_t)t * kTile, kTile, S.bar(kFInF + s));
        issued = it + 1;
      }
      // every load issued has landed before shared memory can go away
      for (int it = (issued > kStagesF ? issued - kStagesF : 0); it < issued; ++it)
        wait_bounded(S.bar(kFInF + it % kStagesF), (uint32_t)((it / kStagesF) & 1), abort_flag, P.status, false);
    }
    __syncwarp();
  } else {
    // a warp reads the TMEM lane quadrant (warp index mod 4): warps 2-5 and 6-9 each cover
    // all four quadrants, one point half each
    const int e = warp - 2, q = warp & 3, hh = e >> 2;
    const int j = 32 * q + lane;
    const float bj = P.bias[j];
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    bool ok = true;
    for (int it = 0; it < n_it; ++it) {
      const int b = it & 1;
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      if (ok) ok = wait_warp(S.bar(kFAccF + b), (uint32_t)((it >> 1) & 1), abort_flag, P.status);
      const uint32_t stage = sOut + (uint32_t)b * kTile;
      if (ok) {
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * kTR) + lane_off;
        if (C == 4) {
          uint32_t v[4][8];
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) tmem_ld8(acc + (uint32_t)(ch * 16 + 8 * hh), v[ch]);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(S.bar(kFAccE + b));
          float o[4][8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float z = __uint_as_float(v[0][i]) + bj;
            const float zx = __uint_as_float(v[1][i]), zy = __uint_as_float(v[2][i]), zl = __uint_as_float(v[3][i]);
            float a, sd;
            tanh_sech2(z, a, sd);
            const float td = -2.0f * a * sd;
            o[0][i] = a;
            o[1][i] = sd * zx;
            o[2][i] = sd * zy;
            o[3][i] = fmaf(td, zx * zx + zy * zy, sd * zl);
          }
          // rows ch * 16 + 8 hh .. + 7 of feature j: chunk 2 ch + hh
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
            st_shared_v4(stage + tile_chunk(j, 2 * ch + hh), pack2(o[ch][0], o[ch][1]), pack2(o[ch][2], o[ch][3]),
                         pack2(o[ch][4], o[ch][5]), pack2(o[ch][6], o[ch][7]));
        } else {
          uint32_t v[32];
          tmem_ld32(acc + (uint32_t)(32 * hh), *reinterpret_cast<uint32_t(*)[32]>(v));
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(S.bar(kFAccE + b));
          float o[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            float sd;
            tanh_sech2(__uint_as_float(v[i]) + bj, o[i], sd);
          }
          // rows 32 hh .. + 31: chunks 4 hh .. 4 hh + 3
#pragma unroll
          for (int c = 0; c < 4; ++c)
            st_shared_v4(stage + tile_chunk(j, 4 * hh + c), pack2(o[8 * c], o[8 * c + 1]), pack2(o[8 * c + 2], o[8 * c + 3]),
                         pack2(o[8 * c + 4], o[8 * c + 5]), pack2(o[8 * c + 6], o[8 * c + 7]));
        }
        fence_proxy_async_smem();
      }
      // one barrier per tile, reached by every epilogue warp, aborted or not: before it,
      // thread 0 waits until the store of tile it-1 has read the staging tile that tile
      // it+1 rewrites
      if (e == 0 && lane == 0) bulk_wait_read<0>();
      named_barrier_sync(1, kEpi * 32);
      if (e == 0 && lane == 0 && ok && !*abort_flag) {
        bulk_s2g(P.A_out + (size_t)t * kTile, stage, kTile);
        bulk_commit();
      }
    }
    if (e == 0 && lane == 0) bulk_wait_all<0>();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
  (void)PT;
}

// ------------------------------------------------------------------ backward kernel

// Backward kernel: 16 epilogue warps (feature quadrant q = w mod 4, point quarter
// pq = (w-2)/4), three input stages, two g_Z^T buffers so that epilogue 1 of tile t+1
// runs while MMAs 2 and 3 of tile t execute (epilogue order: 1(0), then per t: 1(t+1),
// 2(t)). W and W^T are the A operands of MMAs 1 and 2 from tensor memory, which halves
// the shared-memory operand traffic and leaves room for five input stages. Barriers:
// 1..5 in_full[s]; 6..10 in_empty[s] (16 epilogue + 1 MMA arrivals); 11 d1_full;
// 12 d1_empty; 13, 14 gz_full[buffer]; 15 d2_full; 16 d2_empty; 17 d3_done; 18 drain.
// Each barrier is waited on before it can complete again.
constexpr int kEpiB = 16;
constexpr int kThreadsB = (2 + kEpiB) * 32;
constexpr int kStagesB = 5;
constexpr int kBwdBars = 19;
enum { kBInF = 1, kBInE = 6, kBD1F = 11, kBD1E = 12, kBGZ = 13, kBD2F = 15, kBD2E = 16, kBD3 = 17, kBDrain = 18 };

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}
__device__ __forceinline__ uint2 ld_shared_v2(uint32_t addr) {
  uint2 v;
  asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

// Sum of v[0..N-1] (N = 4 or 16) over the 32 lanes of a warp: in the first log2 N
// shuffle rounds each lane sends the half of its values its partner keeps, then the
// remaining rounds finish the one value each lane is left with. Returns that sum; idx
// receives which value it is.
template <int N>
__device__ __forceinline__ float warp_sum_n(const float (&v)[N], int lane, int& idx) {
  float cur[N];
#pragma unroll
  for (int i = 0; i < N; ++i) cur[i] = v[i];
  idx = 0;
  int m = 16;
#pragma unroll
  for (int n = N; n > 1; n >>= 1) {
    const int half = n >> 1;
    const bool hi = (lane & m) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = hi ? cur[i] : cur[i + half];
      const float keep = hi ? cur[i + half] : cur[i];
      cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
    if (hi) idx += half;
    m >>= 1;
  }
  for (; m >= 1; m >>= 1) cur[0] += __shfl_xor_sync(0xffffffffu, cur[0], m);
  return cur[0];
}

template <int C>
__global__ void __launch_bounds__(kThreadsB, 1) tc_bwd_kernel(const __grid_constant__ TcBwdParams P) {
  constexpr int PT = kTR / C;     // points per tile
  constexpr int NP = PT / 4;      // points per epilogue warp: 4 (C = 4) or 16 (C = 1)
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen = smem_raw + (base - raw);
  const uint32_t sA = base;                              // kStagesB tiles of A_{l-1}
  const uint32_t sG = sA + kStagesB * kTile;             // kStagesB tiles of gA_l
  const uint32_t sGZT = sG + kStagesB * kTile;           // 2 g_Z^T tiles
  const uint32_t sOut = sGZT + 2 * kTile;                // 2 staging tiles of gA_{l-1}
  const uint32_t sBar = sOut + 2 * kTile;
  Smem S{sBar};
  uint8_t* genBar = gen + (sBar - base);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(genBar + 8 * kBwdBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(genBar + 8 * kBwdBars + 8);
  // top layer only (no gA tiles are loaded there): the reduction scratch of the output
  // layer, [2][4 quarters][4 quadrants][16 points], lives in the first gA stage
  float* red = reinterpret_cast<float*>(gen + (sG - base));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool top = P.top != 0;
  const int n_it = P.n_tiles > (int)blockIdx.x ? (P.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // TMEM columns: D1 = Z^T [0, 64), D2 = gA^T [64, 128), D3 = g_W [128, 256)
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesB; ++s) { mbar_init(S.bar(kBInF + s), 1); mbar_init(S.bar(kBInE + s), kEpiB + 1); }
    mbar_init(S.bar(kBD1F), 1);
    mbar_init(S.bar(kBD1E), kEpiB);
    mbar_init(S.bar(kBGZ), kEpiB);
    mbar_init(S.bar(kBGZ + 1), kEpiB);
    mbar_init(S.bar(kBD2F), 1);
    mbar_init(S.bar(kBD2E), kEpiB);
    mbar_init(S.bar(kBD3), 1);
    mbar_init(S.bar(kBDrain), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_addr(tmem_holder), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  // TMEM columns: D1 = Z^T [0, 64), D2 = gA^T [64, 128), D3 = g_W [128, 256),
  // W [256, 320) and W^T [320, 384) as A operands
  const uint32_t D1 = tmem, D2 = tmem + 64, D3 = tmem + 128, Wt = tmem + 256, WTt = tmem + 320;
  if (warp >= 2) {
    const int cq = (warp - 2) >> 2;
    weights_to_tmem(static_cast<const uint8_t*>(P.wimg), Wt, warp & 3, lane, cq);
    weights_to_tmem(static_cast<const uint8_t*>(P.wimgT), WTt, warp & 3, lane, cq);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      // MMA 1 (Z^T = W A^T) of tile `it`, once its tiles are in and D1 has been read out
      auto mma1 = [&](int it) -> bool {
        const int s = it % kStagesB;
        if (!wait_spin(S.bar(kBInF + s), (uint32_t)((it / kStagesB) & 1), abort_flag, P.status)) return false;
        if (it > 0 && !wait_spin(S.bar(kBD1E), (uint32_t)((it - 1) & 1), abort_flag, P.status)) return false;
        tc_fence_after();
        const uint32_t ta = sA + (uint32_t)s * kTile;
#pragma unroll
        for (int ks = 0; ks < kW / 16; ++ks) {
          if (ks == 0) mma_ts<0>(D1, Wt + (uint32_t)(8 * ks), desc_rows(ta, ks), kIdescRows);
          else mma_ts<1>(D1, Wt + (uint32_t)(8 * ks), desc_rows(ta, ks), kIdescRows);
        }
        mma_commit(S.bar(kBD1F));
        return true;
      };
      if (ok && n_it > 0) ok = mma1(0);
      for (int it = 0; ok && it < n_it; ++it) {
        const int s = it % kStagesB, zb = it & 1;
        const uint32_t ta = sA + (uint32_t)s * kTile;
        const uint32_t gz = sGZT + (uint32_t)zb * kTile;
        // the next tile's recompute runs while epilogue 1 of this tile works
        if (it + 1 < n_it && !mma1(it + 1)) { ok = false; break; }
        ok = wait_spin(S.bar(kBGZ + zb), (uint32_t)((it >> 1) & 1), abort_flag, P.status);
        if (ok && it > 0) ok = wait_spin(S.bar(kBD2E), (uint32_t)((it - 1) & 1), abort_flag, P.status);
        if (!ok) break;
        tc_fence_after();
        // MMA 2: gA^T = W^T g_Z^T (g_Z^T tile read MN-major: N = rows, K = features)
#pragma unroll
        for (int ks = 0; ks < kW / 16; ++ks) {
          if (ks == 0) mma_ts<0>(D2, WTt + (uint32_t)(8 * ks), desc_rows(gz, ks), kIdescRows);
          else mma_ts<1>(D2, WTt + (uint32_t)(8 * ks), desc_rows(gz, ks), kIdescRows);
        }
        // MMA 3: g_W += g_Z^T A (A tile read K-major: N = features, K = rows)
        const uint64_t gzd = desc_sw128(gz), tad = desc_sw128(ta);
#pragma unroll
        for (int ks = 0; ks < kTR / 16; ++ks) {
          const uint64_t a_op = desc_add(gzd, (uint32_t)ks * 32u);
          const uint64_t b_op = desc_add(tad, (uint32_t)ks * 32u);
          if (it == 0 && ks == 0) mma_ss<0>(D3, a_op, b_op, kIdescGW);
          else mma_ss<1>(D3, a_op, b_op, kIdescGW);
        }
        mma_commit(S.bar(kBD2F));
        mma_commit(S.bar(kBInE + s));
      }
      mma_commit(S.bar(kBD3));  // every MMA issued, including the last g_W accumulation, done
      mma_commit(S.bar(kBDrain));
      wait_bounded(S.bar(kBDrain), 0, abort_flag, P.status, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t bytes = top ? kTile : 2 * kTile;
      int issued = 0;
      for (int it = 0; it < n_it; ++it) {
        const int s = it % kStagesB;
        if (it >= kStagesB &&
            !wait_bounded(S.bar(kBInE + s), (uint32_t)(((it / kStagesB) - 1) & 1), abort_flag, P.status, true))
          break;
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        mbar_arrive_expect_tx(S.bar(kBInF + s), bytes);
        bulk_g2s(sA + (uint32_t)s * kTile, P.A_in + (size_t)t * kTile, kTile, S.bar(kBInF + s));
        if (!top) bulk_g2s(sG + (uint32_t)s * kTile, P.gA_in + (size_t)t * kTile, kTile, S.bar(kBInF + s));
        issued = it + 1;
      }
      for (int it = (issued > kStagesB ? issued - kStagesB : 0); it < issued; ++it)
        wait_bounded(S.bar(kBInF + it % kStagesB), (uint32_t)((it / kStagesB) & 1), abort_flag, P.status, false);
    }
    __syncwarp();
  } else {
    // a warp reads the TMEM lane quadrant (warp index mod 4); the 16 warps cover the four
    // quadrants for each of the four point quarters of a tile
    const int e = warp - 2, q = warp & 3, pq = e >> 2;
    const int j = 32 * q + lane;  // feature (D1, D3 lanes) / input feature k (D2 lanes)
    const float bj = P.bias[j];
    const float wo = top ? P.wout[j] : 0.f;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const int p0 = pq * NP;
    // rows ch * PT + p0 .. + NP - 1 of feature j: C = 4 -> 8 bytes (half a chunk) per
    // channel, C = 1 -> two 16-byte chunks
    auto row_addr = [&](uint32_t tile, int ch) -> uint32_t {
      const int r = ch * PT + p0;
      return tile + tile_chunk(j, r >> 3) + (uint32_t)(r & 7) * 2u;
    };
    float gb = 0.f, gwo = 0.f, gbo = 0.f;
    double lsum = 0.0;
    bool ok = true;

    // ---- epilogue 1 of tile it: g_Z from the recomputed Z and the incoming gradient
    auto epi1 = [&](int it) {
      const int s = it % kStagesB, zb = it & 1;
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      const uint32_t sg = sG + (uint32_t)s * kTile;
      const uint32_t gzt = sGZT + (uint32_t)zb * kTile;
      float z[NP], zx[NP], zy[NP], zl[NP];
      if (ok) ok = wait_warp(S.bar(kBD1F), (uint32_t)(it & 1), abort_flag, P.status);
      if (ok && !top) ok = wait_warp(S.bar(kBInF + s), (uint32_t)((it / kStagesB) & 1), abort_flag, P.status);
      if (ok) {
        tc_fence_after();
        if constexpr (C == 4) {
          uint32_t v[4][4];
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) tmem_ld4(D1 + lane_off + (uint32_t)(ch * 16 + p0), v[ch]);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            z[i] = __uint_as_float(v[0][i]) + bj;
            zx[i] = __uint_as_float(v[1][i]);
            zy[i] = __uint_as_float(v[2][i]);
            zl[i] = __uint_as_float(v[3][i]);
          }
        } else {
          uint32_t v[16];
          tmem_ld16(D1 + lane_off + (uint32_t)p0, v);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < NP; ++i) z[i] = __uint_as_float(v[i]) + bj;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(S.bar(kBD1E));
      } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) { z[i] = 0.f; zx[i] = 0.f; zy[i] = 0.f; zl[i] = 0.f; }
      }
      // top layer: the output layer and the loss, u = w_out . a + b_out (data) or
      // Delta u = w_out . Delta a (collocation), summed over the 128 features by the
      // shuffles of warp_sum_n and the four quadrant warps of this point quarter
      // a = tanh z and s = sech^2 z of this thread's points, computed once
      float ta[NP], ts[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) tanh_sech2(z[i], ta[i], ts[i]);
      float gu[NP];
      if (top) {
        float part[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          if constexpr (C == 4) part[i] = wo * fmaf(-2.0f * ta[i] * ts[i], zx[i] * zx[i] + zy[i] * zy[i], ts[i] * zl[i]);
          else part[i] = wo * ta[i];
        }
        int idx;
        const float tot = warp_sum_n<NP>(part, lane, idx);
        constexpr int kLanesPerValue = 32 / NP;
        // the scratch alternates between tiles, so one barrier per tile suffices: a
        // quarter's warps rewrite a half only after all of them passed the barrier of
        // the tile after the one that read it
        float* rb = red + (it & 1) * 256;
        if ((lane & (kLanesPerValue - 1)) == 0) rb[(pq * 4 + q) * 16 + idx] = tot;
        named_barrier_sync(2 + pq, 128);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const float sum = rb[(pq * 4 + 0) * 16 + i] + rb[(pq * 4 + 1) * 16 + i] + rb[(pq * 4 + 2) * 16 + i] +
                            rb[(pq * 4 + 3) * 16 + i];
          float d = sum;                                                       // Delta u
          if constexpr (C == 1) d = sum + *P.bout - P.Y[(size_t)t * PT + p0 + i];  // u - y
          gu[i] = P.gscale * d;
          if (q == 0 && lane == 0 && ok) {
            lsum += (double)d * (double)d;
            if constexpr (C == 1) gbo += gu[i];
          }
        }
      }
      if (ok) {
        float o[C][NP];
        if constexpr (C == 4) {
          float ga[4][NP];
          if (top) {
#pragma unroll
            for (int i = 0; i < NP; ++i) { ga[0][i] = 0.f; ga[1][i] = 0.f; ga[2][i] = 0.f; ga[3][i] = gu[i] * wo; }
          } else {
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
              const uint2 w = ld_shared_v2(row_addr(sg, ch));
              ga[ch][0] = __uint_as_float(w.x << 16);
              ga[ch][1] = __uint_as_float(w.x & 0xffff0000u);
              ga[ch][2] = __uint_as_float(w.y << 16);
              ga[ch][3] = __uint_as_float(w.y & 0xffff0000u);
            }
          }
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const float a = ta[i], sd = ts[i];
            const float td = -2.0f * a * sd;
            const float tp = -2.0f * sd * sd + 4.0f * a * a * sd;
            const float q2 = zx[i] * zx[i] + zy[i] * zy[i];
            const float gal = ga[3][i];
            if (top) gwo = fmaf(gu[i], fmaf(td, q2, sd * zl[i]), gwo);
            const float g0 = ga[0][i] * sd + (ga[1][i] * zx[i] + ga[2][i] * zy[i]) * td + gal * fmaf(tp, q2, td * zl[i]);
            o[0][i] = g0;
            o[1][i] = fmaf(ga[1][i], sd, 2.0f * gal * td * zx[i]);
            o[2][i] = fmaf(ga[2][i], sd, 2.0f * gal * td * zy[i]);
            o[3][i] = gal * sd;
            gb += g0;
          }
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
            st_shared_v2(row_addr(gzt, ch), pack2(o[ch][0], o[ch][1]), pack2(o[ch][2], o[ch][3]));
        } else {
          float ga[NP];
          if (top) {
#pragma unroll
            for (int i = 0; i < NP; ++i) ga[i] = gu[i] * wo;
          } else {
            unpack8(ld_shared_v4(sg + tile_chunk(j, p0 >> 3)), ga);
            unpack8(ld_shared_v4(sg + tile_chunk(j, (p0 >> 3) + 1)), ga + 8);
          }
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const float a = ta[i], sd = ts[i];
            if (top) gwo = fmaf(gu[i], a, gwo);
            o[0][i] = ga[i] * sd;
            gb += o[0][i];
          }
#pragma unroll
          for (int c = 0; c < 2; ++c)
            st_shared_v4(gzt + tile_chunk(j, (p0 >> 3) + c), pack2(o[0][8 * c], o[0][8 * c + 1]),
                         pack2(o[0][8 * c + 2], o[0][8 * c + 3]), pack2(o[0][8 * c + 4], o[0][8 * c + 5]),
                         pack2(o[0][8 * c + 6], o[0][8 * c + 7]));
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(S.bar(kBGZ + zb));
          mbar_arrive(S.bar(kBInE + s));
        }
      }
    };

    // ---- epilogue 2 of tile it: the gA_{l-1} tile (row = this thread's input feature),
    // written to staging tile it mod 2. One barrier per tile: before it, thread 0 waits
    // until the store of tile it-1 has read its staging tile, which tile it+1 rewrites.
    auto epi2 = [&](int it) {
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      const uint32_t sOutB = sOut + (uint32_t)(it & 1) * kTile;
      if (ok) ok = wait_warp(S.bar(kBD2F), (uint32_t)(it & 1), abort_flag, P.status);
      if (ok) {
        tc_fence_after();
        if constexpr (C == 4) {
          uint32_t v[4][4];
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) tmem_ld4(D2 + lane_off + (uint32_t)(ch * 16 + p0), v[ch]);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(S.bar(kBD2E));
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
            st_shared_v2(row_addr(sOutB, ch), pack2(__uint_as_float(v[ch][0]), __uint_as_float(v[ch][1])),
                         pack2(__uint_as_float(v[ch][2]), __uint_as_float(v[ch][3])));
        } else {
          uint32_t v[16];
          tmem_ld16(D2 + lane_off + (uint32_t)p0, v);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(S.bar(kBD2E));
#pragma unroll
          for (int c = 0; c < 2; ++c)
            st_shared_v4(sOutB + tile_chunk(j, (p0 >> 3) + c),
                         pack2(__uint_as_float(v[8 * c]), __uint_as_float(v[8 * c + 1])),
                         pack2(__uint_as_float(v[8 * c + 2]), __uint_as_float(v[8 * c + 3])),
                         pack2(__uint_as_float(v[8 * c + 4]), __uint_as_float(v[8 * c + 5])),
                         pack2(__uint_as_float(v[8 * c + 6]), __uint_as_float(v[8 * c + 7])));
        }
        fence_proxy_async_smem();
      }
      if (e == 0 && lane == 0) bulk_wait_read<0>();
      named_barrier_sync(1, kEpiB * 32);
      if (e == 0 && lane == 0 && ok && !*abort_flag) {
        bulk_s2g(P.gA_out + (size_t)t * kTile, sOutB, kTile);
        bulk_commit();
      }
    };

    if (n_it > 0) epi1(0);
    for (int it = 0; it < n_it; ++it) {
      if (it + 1 < n_it) epi1(it + 1);
      epi2(it);
    }
    if (e == 0 && lane == 0) bulk_wait_all<0>();
    // per-CTA partial sums: g_W (this warp's quadrant of rows, quarter of columns), g_b,
    // and at the top the output layer and the loss
    if (ok && n_it > 0) ok = wait_warp(S.bar(kBD3), 0, abort_flag, P.status);
    float* gwp = P.gW_part + (size_t)blockIdx.x * kW * kW;
    const int k0 = 32 * pq;
    if (ok && n_it > 0) {
      tc_fence_after();
      uint32_t v[32];
      tmem_ld32(D3 + lane_off + (uint32_t)k0, *reinterpret_cast<uint32_t(*)[32]>(v));
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *reinterpret_cast<float4*>(gwp + (size_t)j * kW + k0 + i) =
            make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]), __uint_as_float(v[i + 2]),
                        __uint_as_float(v[i + 3]));
    } else {
      for (int k = k0; k < k0 + 32; ++k) gwp[(size_t)j * kW + k] = 0.f;
    }
    P.gb_part[((size_t)blockIdx.x * 4 + pq) * kW + j] = ok ? gb : 0.f;
    if (top) {
      P.gwout_part[((size_t)blockIdx.x * 4 + pq) * kW + j] = ok ? gwo : 0.f;
      if (q == 0 && lane == 0) {
        P.loss_part[blockIdx.x * 4 + pq] = ok ? lsum : 0.0;
        P.gbout_part[blockIdx.x * 4 + pq] = ok ? gbo : 0.f;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------ first layer

// A_0 tiles: the input-split first layer (Eq. 8), z = Bf[f] + b0 + W2 x (FP32), in Taylor
// mode (z_x = W2[:,0], z_y = W2[:,1], Delta z = 0). One thread per (feature, 8 points):
// each channel of the 8 points is one 16-byte chunk of the feature's row.
__global__ void tc_first_fwd_kernel(const float* __restrict__ Bf, const float* __restrict__ W0,
                                    const float* __restrict__ b0, const float* __restrict__ X, int n, int R, int C,
                                    uint8_t* __restrict__ A0) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (R / 8) * kW) return;
  const int k = idx % kW, pt0 = 8 * (idx / kW);
  const int f = pt0 / n;
  const int PT = kTR / C, tile = pt0 / PT, p = pt0 % PT;
  const float w2x = W0[(size_t)k * 130 + 128], w2y = W0[(size_t)k * 130 + 129];
  const float bk = Bf[(size_t)f * kW + k] + b0[k];
  const float lap = w2x * w2x + w2y * w2y;
  float o[4][8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float x = X[2 * (size_t)(pt0 + i)], y = X[2 * (size_t)(pt0 + i) + 1];
    float a, sd;
    tanh_sech2(fmaf(w2y, y, fmaf(w2x, x, bk)), a, sd);
    o[0][i] = a;
    o[1][i] = sd * w2x;
    o[2][i] = sd * w2y;
    o[3][i] = -2.0f * a * sd * lap;
  }
  uint8_t* tb = A0 + (size_t)tile * kTile;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (c >= C) break;
    *reinterpret_cast<uint4*>(tb + tile_chunk(k, (c * PT + p) >> 3)) =
        make_uint4(pack2(o[c][0], o[c][1]), pack2(o[c][2], o[c][3]), pack2(o[c][4], o[c][5]), pack2(o[c][6], o[c][7]));
  }
}

// First-layer backward from the gA_0 tiles: g_z, g_zx, g_zy per (point, feature) and
// the block partials of sum g_z, sum g_z x + g_zx, sum g_z y + g_zy ([3][128] per block
// of 64 points; a block never spans two functions since n is a multiple of 64).
__global__ void tc_first_bwd_kernel(const float* __restrict__ Bf, const float* __restrict__ W0,
                                    const float* __restrict__ b0, const float* __restrict__ X, int n, int R, int C,
                                    const uint8_t* __restrict__ gA0, float* __restrict__ part) {
  const int j = threadIdx.x;  // 128 threads: one feature, 64 points
  const float w2x = W0[(size_t)j * 130 + 128], w2y = W0[(size_t)j * 130 + 129];
  const float bj = b0[j];
  const float lap = w2x * w2x + w2y * w2y;
  const int PT = kTR / C;
  float s0 = 0.f, sx = 0.f, sy = 0.f;
  const int pt1 = min(R, (blockIdx.x + 1) * 64);
  for (int pt0 = blockIdx.x * 64; pt0 < pt1; pt0 += 8) {
    const int f = pt0 / n;
    const float bk = Bf[(size_t)f * kW + j] + bj;
    const uint8_t* tb = gA0 + (size_t)(pt0 / PT) * kTile;
    const int p = pt0 % PT;
    float ga[4][8];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < C) unpack8(*reinterpret_cast<const uint4*>(tb + tile_chunk(j, (c * PT + p) >> 3)), ga[c]);
      else
#pragma unroll
        for (int i = 0; i < 8; ++i) ga[c][i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float x = X[2 * (size_t)(pt0 + i)], y = X[2 * (size_t)(pt0 + i) + 1];
      float a, sd;
      tanh_sech2(fmaf(w2y, y, fmaf(w2x, x, bk)), a, sd);
      const float td = -2.0f * a * sd;
      const float tp = -2.0f * sd * sd + 4.0f * a * a * sd;
      const float gz = ga[0][i] * sd + (ga[1][i] * w2x + ga[2][i] * w2y) * td + ga[3][i] * tp * lap;
      const float gzx = fmaf(ga[1][i], sd, 2.0f * ga[3][i] * td * w2x);
      const float gzy = fmaf(ga[2][i], sd, 2.0f * ga[3][i] * td * w2y);
      s0 += gz;
      sx += fmaf(gz, x, gzx);
      sy += fmaf(gz, y, gzy);
    }
  }
  float* o = part + (size_t)blockIdx.x * 3 * kW;
  o[j] = s0;
  o[kW + j] = sx;
  o[2 * kW + j] = sy;
}

// W (FP32, [out][in]) -> BF16 image in the K-major 128-byte-swizzled operand layout,
// as W itself (rows = out) or transposed (rows = in).
__global__ void tc_pack_kernel(const float* __restrict__ W, uint16_t* __restrict__ img, int transpose) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kW * kW) return;
  const int row = idx / kW, k = idx % kW;
  const float v = transpose ? W[(size_t)k * kW + row] : W[(size_t)row * kW + k];
  const uint32_t off = (uint32_t)(k >> 6) * (kW * 128u) + (uint32_t)row * 128u +
                       ((((uint32_t)(k & 63) >> 3) ^ (uint32_t)(row & 7)) << 4) + (uint32_t)(k & 7) * 2u;
  img[off / 2] = bf16_bits(v);
}

// out[j] (+)= sum over b < nblk of part[b * stride + j] (one thread per j): four
// interleaved partial sums (b mod 4) for latency, combined in a fixed order.
__global__ void tc_colsum_kernel(const float* __restrict__ part, int nblk, int stride, int n, float* __restrict__ out,
                                 int accumulate) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int b = 0;
  for (; b + 4 <= nblk; b += 4) {
    s0 += part[(size_t)b * stride + j];
    s1 += part[(size_t)(b + 1) * stride + j];
    s2 += part[(size_t)(b + 2) * stride + j];
    s3 += part[(size_t)(b + 3) * stride + j];
  }
  for (; b < nblk; ++b) s0 += part[(size_t)b * stride + j];
  const float s = (s0 + s1) + (s2 + s3);
  out[j] = accumulate ? out[j] + s : s;
}

__global__ void tc_sum_double_kernel(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += part[i];
  *out += s * scale;
}

__global__ void tc_sum_float_kernel(const float* __restrict__ part, int n, float* __restrict__ out) {
  if (threadIdx.x != 0) return;
  float s = 0.f;
  for (int i = 0; i < n; ++i) s += part[i];
  *out += s;
}

constexpr size_t kFwdSmem = 1024 + kStagesF * kTile + 2 * kTile + 8 * kFwdBars + 64;
constexpr size_t kBwdSmem = 1024 + 2 * kStagesB * kTile + 2 * kTile + 2 * kTile + 8 * kBwdBars + 16 + 64;
static_assert(kBwdSmem <= 232448, "backward kernel shared memory");

int grid_for(int n_tiles) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return n_tiles < sms ? n_tiles : sms;
}

}  // namespace

size_t tc_tile_bytes() { return kTile; }
int tc_partial_groups() { return 4; }
size_t tc_image_bytes() { return kWImg; }
int tc_partial_ctas() { return grid_for(1 << 30); }

cudaError_t tc_pack_weights(const float* W, void* img, void* imgT, cudaStream_t st) {
  tc_pack_kernel<<<kW * kW / 256, 256, 0, st>>>(W, static_cast<uint16_t*>(img), 0);
  tc_pack_kernel<<<kW * kW / 256, 256, 0, st>>>(W, static_cast<uint16_t*>(imgT), 1);
  return cudaGetLastError();
}

cudaError_t tc_first_fwd(const float* Bf, const float* W0, const float* b0, const float* X, int n, int R, int C,
                         void* A0, cudaStream_t st) {
  const int threads = (R / 8) * kW;
  tc_first_fwd_kernel<<<(threads + 255) / 256, 256, 0, st>>>(Bf, W0, b0, X, n, R, C, static_cast<uint8_t*>(A0));
  return cudaGetLastError();
}

cudaError_t tc_first_bwd(const float* Bf, const float* W0, const float* b0, const float* X, int n, int R, int C,
                         const void* gA0, float* part, cudaStream_t st) {
  tc_first_bwd_kernel<<<(R + 63) / 64, kW, 0, st>>>(Bf, W0, b0, X, n, R, C, static_cast<const uint8_t*>(gA0), part);
  return cudaGetLastError();
}

cudaError_t tc_layer_fwd(const TcFwdParams& p, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (p.n_tiles <= 0) return cudaSuccess;
  tc_fwd_kernel<<<grid_for(p.n_tiles), kThreadsTc, kFwdSmem, st>>>(p);
  return cudaGetLastError();
}

template <int C>
cudaError_t launch_bwd(const TcBwdParams& p, int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_bwd_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  tc_bwd_kernel<C><<<grid, kThreadsB, kBwdSmem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t tc_layer_bwd(const TcBwdParams& p, int* grid_used, cudaStream_t st) {
  const int grid = p.n_tiles > 0 ? grid_for(p.n_tiles) : 0;
  if (grid_used) *grid_used = grid;
  if (grid == 0) return cudaSuccess;
  if (p.C == 4) return launch_bwd<4>(p, grid, st);
  if (p.C == 1) return launch_bwd<1>(p, grid, st);
  return cudaErrorInvalidValue;
}

cudaError_t tc_colsum(const float* part, int nblk, int stride, int n, float* out, int accumulate, cudaStream_t st) {
  tc_colsum_kernel<<<(n + 63) / 64, 64, 0, st>>>(part, nblk, stride, n, out, accumulate);
  return cudaGetLastError();
}

cudaError_t tc_sum_double(const double* part, int n, double scale, double* out, cudaStream_t st) {
  tc_sum_double_kernel<<<1, 32, 0, st>>>(part, n, scale, out);
  return cudaGetLastError();
}

cudaError_t tc_sum_float(const float* part, int n, float* out, cudaStream_t st) {
  tc_sum_float_kernel<<<1, 32, 0, st>>>(part, n, out);
  return cudaGetLastError();
}

}  // namespace mf
