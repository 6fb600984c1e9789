// K7-K8 on the tensor cores: fused Taylor-mode layer kernels of the physics-informed
// training step (Eq. 3, Algorithm 1), BF16 operands with FP32 accumulators, width 128.
//
// Orientation. A layer computes Z^T = W A^T with M = 128 output features (TMEM lanes)
// and N = 128 GEMM rows of a tile: the four Taylor channels (value, d/dx, d/dy, Delta) of
// 32 points, or 128 points of the value channel alone. Each epilogue thread then owns one
// feature and holds every channel of its points, which is what the chain rules of the
// Taylor-mode tanh need (see mf_train.cu for the formulas). Every MMA of a tile is a
// 128 x 128 x 128 group.
//
// Activations and their gradients travel between layers in HBM as BF16 tiles of 128
// GEMM rows x 128 features, 32 KB each (row r = channel x (points per tile) + point),
// stored as two halves of 64 rows, each feature-major: in half h feature k owns 128
// bytes, and the 16-byte chunk c (rows 64h + 8c .. 64h + 8c + 7) sits at chunk c ^ (k mod 8).
// Each half is byte for byte the 128-byte-swizzled operand layout, so one bulk copy loads
// a tile that the MMAs read directly: as an MN-major operand with N = rows (two 64-row
// atoms 16 KB apart) and K = features (Z = W A^T, and gA^T = W^T g_Z^T), or half by half
// as a K-major operand with N = features and K = rows (g_W = g_Z^T A). An epilogue thread
// owns one feature and so reads and writes its rows with 16-byte accesses.
//
// A launch covers both loss terms of a chunk: the collocation points' tiles (four
// channels) first, then the data points' tiles (value channel); the MMAs and copies do not
// depend on the form, the epilogues take each tile's.
// Forward kernels (hidden layers 1..NH-1): load tile A_{l-1}; MMA into TMEM; epilogue
// applies the Taylor-mode tanh and writes tile A_l. The two-layer kernel then uses that
// tile, still in shared memory, as the operand of layer l+1's MMA (besides storing it).
// Pre-activations are never stored.
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
// The value channel of the data points is padded to whole tiles: the first layer writes
// zero rows past the last point, every later row of the padding stays finite, and the top
// layer gives those rows a zero residual, so their g_Z, gA and g_W contributions are 0.
//
// Roles per CTA (persistent, one CTA per SM, static tile schedule t = CTA + i x CTAs):
// warp 0 lane 0 issues the MMAs, warp 1 lane 0 issues the bulk loads, and the epilogue
// warps (warps 2-9 of the forward kernel, 2-17 in two stages of the two-layer one, 4-19
// of the backward kernel) each own the
// feature quadrant q = w mod 4, the TMEM lanes warp w may read. Every wait is bounded
// (mf_wait.cuh); after an abort the epilogue warps keep stepping through their loop
// without work, so that every named barrier is reached by every warp, and the CTA drains
// its MMAs and bulk copies before it frees TMEM and exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "mf_internal.cuh"
#include "mf_tc.cuh"
#include "mf_train_tc.cuh"
#include "mf_wait.cuh"

namespace mf {

namespace {

constexpr int kW = 128;                        // width H on the fused path
constexpr int kTR = 128;                       // GEMM rows per tile
constexpr uint32_t kHalf = 64 * kW * 2;        // 16 KB: 64 rows of a tile
constexpr uint32_t kTile = 2 * kHalf;          // 32 KB
constexpr uint32_t kWImg = kW * kW * 2;        // 32 KB
constexpr int kEpi = 8;                        // epilogue warps (forward)
constexpr int kThreadsTc = (2 + kEpi) * 32;    // MMA warp, load warp, epilogue
constexpr int kStagesF = 5;                    // input tiles in flight per CTA (forward)
constexpr uint32_t kIdescRows = idesc_bf16_bmn(128, kTR);  // B = tile, N = rows (MN-major)
constexpr uint32_t kIdescGW = idesc_bf16(128, kW);          // B = tile, N = features (K-major)

// Byte offset of the 16-byte chunk holding rows 8c..8c+7 (c = 0..15) of feature k.
__host__ __device__ __forceinline__ uint32_t tile_chunk(int k, int c) {
  return (uint32_t)(c >> 3) * kHalf + (uint32_t)k * 128u + ((uint32_t)((c & 7) ^ (k & 7)) << 4);
}
// K step ks (features 16ks..16ks+15) of a tile read MN-major: N = 128 rows in two 64-row
// atoms kHalf apart (leading byte offset), 8-feature groups 1 KB apart (stride byte offset).
__device__ __forceinline__ uint64_t desc_rows(uint32_t tile, int ks) {
  return desc_sw128_mn(tile + (uint32_t)ks * 2048u, kHalf, 1024u);
}
// Offset of K step ks (rows 16ks..16ks+15) of a tile read K-major, half by half.
__device__ __forceinline__ uint32_t kstep_rows(int ks) {
  return (uint32_t)(ks >> 2) * kHalf + (uint32_t)(ks & 3) * 32u;
}

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
               : "memory");
  return v;
}
// two floats as one BF16 pair (round to nearest even), lo in the low half: one paired
// conversion instead of two single ones
__device__ __forceinline__ uint32_t pack2(float lo, float hi) { return pack_bf16x2(lo, hi); }
// the 8 BF16 values of a chunk as floats
__device__ __forceinline__ void unpack8(uint4 v, float* f) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

// Register reallocation between the warpgroups of a CTA (all four warps of a warpgroup
// execute it; the increase waits until the registers it needs have been given back).
template <int N>
__device__ __forceinline__ void setmaxnreg_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}
template <int N>
__device__ __forceinline__ void setmaxnreg_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}

// dst[i] = sum over the four quadrant rows of row[q * stride + i], i = 0..3, added in the
// order q = 0, 1, 2, 3; 16-byte shared-memory loads (the values are broadcast to the warp)
__device__ __forceinline__ void quad_sum4(const float* row, int stride, float (&dst)[4]) {
  float4 a = *reinterpret_cast<const float4*>(row);
#pragma unroll
  for (int qq = 1; qq < 4; ++qq) {
    const float4 x = *reinterpret_cast<const float4*>(row + qq * stride);
    a.x += x.x; a.y += x.y; a.z += x.z; a.w += x.w;
  }
  dst[0] = a.x; dst[1] = a.y; dst[2] = a.z; dst[3] = a.w;
}

// BF16 value i (0..7) of a 16-byte chunk, as a float
__device__ __forceinline__ float bf16_word(const uint4& u, int i) {
  const uint32_t w = (i >> 1) == 0 ? u.x : (i >> 1) == 1 ? u.y : (i >> 1) == 2 ? u.z : u.w;
  return (i & 1) ? __uint_as_float(w & 0xffff0000u) : __uint_as_float(w << 16);
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

// Packed FP32 arithmetic, two points per instruction (the epilogues that use it are
// bound by their instruction issue).
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 f2(uint32_t x, uint32_t y) { return make_float2(__uint_as_float(x), __uint_as_float(y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// tanh_sech2 of two pre-activations. The exponential is taken as 4 e = 2^(2 - 2|z|/ln 2),
// so that s = (4 e) r^2 and 1 +- e = 1 +- (4 e) / 4 cost one packed operation each.
__device__ __forceinline__ void tanh_sech2_x2(float2 z, float2& a, float2& s) {
  const float2 e4 = make_float2(ex2_approx(fmaf(-2.8853900817779268f, fabsf(z.x), 2.0f)),
                                ex2_approx(fmaf(-2.8853900817779268f, fabsf(z.y), 2.0f)));
  const float2 d = fma2(e4, f2(0.25f), f2(1.0f));
  const float2 r = make_float2(rcp_approx(d.x), rcp_approx(d.y));
  const float2 m = mul2(fma2(e4, f2(-0.25f), f2(1.0f)), r);
  a = make_float2(copysignf(m.x, z.x), copysignf(m.y, z.y));
  s = mul2(mul2(e4, r), r);
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

// Bounded waits, inline (the backward kernel reallocates registers between warpgroups,
// so it calls no out-of-line function): a single thread (wait_fast) or a whole warp
// (wait_warp_fast, which continues only if every lane saw the phase complete).
__device__ __forceinline__ bool wait_fast(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  return wait_spin_inl(bar, parity, abort_flag, status);
}
__device__ __forceinline__ bool wait_warp_fast(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  return wait_warp_inl(bar, parity, abort_flag, status);
}

struct Smem {
  uint32_t base;
  __device__ uint32_t bar(int i) const { return base + 8u * (uint32_t)i; }
};

// ------------------------------------------------------------------ forward kernel

// barriers: 1+s in_full[s]; 6+s in_empty[s]; 11+b acc_full[b]; 13+b acc_empty[b]; 15 drain
constexpr int kFwdBars = 16;
enum { kFInF = 1, kFInE = 6, kFAccF = 11, kFAccE = 13, kFDrain = 15 };

// Taylor-mode tanh of 8 points of one feature (value, d/dx, d/dy, Delta channels) from
// the accumulator words v[ch][0..7], written as one 16-byte chunk per channel.
__device__ __forceinline__ void fwd_taylor8(const uint32_t (&v)[4][8], float bj, uint32_t stage, int j, int c0) {
  uint32_t w[4][4];
#pragma unroll
  for (int i = 0; i < 8; i += 2) {  // points i and i + 1
    const float2 z = add2(f2(v[0][i], v[0][i + 1]), f2(bj));
    const float2 zx = f2(v[1][i], v[1][i + 1]), zy = f2(v[2][i], v[2][i + 1]), zl = f2(v[3][i], v[3][i + 1]);
    float2 a, sd;
    tanh_sech2_x2(z, a, sd);
    const float2 o1 = mul2(sd, zx), o2 = mul2(sd, zy);
    const float2 o3 = fma2(mul2(mul2(a, f2(-2.0f)), sd), fma2(zx, zx, mul2(zy, zy)), mul2(sd, zl));
    w[0][i >> 1] = pack2(a.x, a.y);
    w[1][i >> 1] = pack2(o1.x, o1.y);
    w[2][i >> 1] = pack2(o2.x, o2.y);
    w[3][i >> 1] = pack2(o3.x, o3.y);
  }
  // channel ch of points 8 c0 .. 8 c0 + 7: chunk 4 ch + c0
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) st_shared_v4(stage + tile_chunk(j, 4 * ch + c0), w[ch][0], w[ch][1], w[ch][2], w[ch][3]);
}

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
  const int n_it = P.n_tiles > (int)blockIdx.x ? (P.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesF; ++s) { mbar_init(S.bar(kFInF + s), 1); mbar_init(S.bar(kFInE + s), 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(S.bar(kFAccF + b), 1); mbar_init(S.bar(kFAccE + b), kEpi); }
    mbar_init(S.bar(kFDrain), 1);
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
  // TMEM columns: accumulators [0, 256) (two buffers of 128), W as the A operand [256, 320)
  const uint32_t Wt = tmem + 256;
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
        ok = wait_fast(S.bar(kFInF + s), (uint32_t)((it / kStagesF) & 1), abort_flag, P.status);
        if (ok && it >= 2) ok = wait_fast(S.bar(kFAccE + b), (uint32_t)(((it >> 1) - 1) & 1), abort_flag, P.status);
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
    // all four quadrants, one half of the tile's points each
    const int e = warp - 2, q = warp & 3, hh = e >> 2;
    const int j = 32 * q + lane;
    const float bj = P.bias[j];
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    bool ok = true;
    for (int it = 0; it < n_it; ++it) {
      const int b = it & 1;
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      if (ok) ok = wait_warp_fast(S.bar(kFAccF + b), (uint32_t)((it >> 1) & 1), abort_flag, P.status);
      const uint32_t stage = sOut + (uint32_t)b * kTile;
      if (ok) {
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * kTR) + lane_off;
        if (t < P.n_tiles4) {
          // collocation tile, points 16 hh .. 16 hh + 15 of its 32: two groups of 8
          uint32_t v0[4][8], v1[4][8];
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) {
            tmem_ld8(acc + (uint32_t)(ch * 32 + 16 * hh), v0[ch]);
            tmem_ld8(acc + (uint32_t)(ch * 32 + 16 * hh + 8), v1[ch]);
          }
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(S.bar(kFAccE + b));
          fwd_taylor8(v0, bj, stage, j, 2 * hh);
          fwd_taylor8(v1, bj, stage, j, 2 * hh + 1);
        } else {
          // rows 64 hh .. 64 hh + 63: chunks 8 hh .. 8 hh + 7
          uint32_t v[2][32];
          tmem_ld32(acc + (uint32_t)(64 * hh), v[0]);
          tmem_ld32(acc + (uint32_t)(64 * hh + 32), v[1]);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(S.bar(kFAccE + b));
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            float o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float sd;
              tanh_sech2(__uint_as_float(v[c >> 2][8 * (c & 3) + i]) + bj, o[i], sd);
            }
            st_shared_v4(stage + tile_chunk(j, 8 * hh + c), pack2(o[0], o[1]), pack2(o[2], o[3]), pack2(o[4], o[5]),
                         pack2(o[6], o[7]));
          }
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
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------ two-layer forward kernel

// Forward of two consecutive hidden layers l and l+1 in one pass over the tiles. The
// activations A_l of a tile are written by the first epilogue stage into a shared-memory
// tile that is both stored to HBM (the backward pass needs A_l) and read directly as the
// B operand of layer l+1's MMA, so A_l is never read back from HBM: a pair moves 3 tiles
// per tile of input instead of the 4 of two single-layer launches.
// Warps: 0 MMA issuer, 1 loads, 2-9 stage a (layer l: accumulator 1 -> tile X), 10-17
// stage b (layer l+1: accumulator 2 -> staging tile Y), 18-21 first-layer producers. In
// the launch of layers 1 and 2 the producers (one thread per feature) form each A_0 tile
// in its input slot from the per-function boundary term and the points (Eq. 8, the
// Taylor-mode first layer of tc_first_fwd_kernel) and store it for the backward pass, so
// A_0 is written once and never read back; otherwise the load warp fills the slots and
// the producers idle. TMEM: accumulator 1 double-buffered [0, 256), accumulator 2
// [256, 384), W_l [384, 448), W_{l+1} [448, 512).
// Shared memory: three input slots, two X tiles, two Y tiles (224 KB).
// Barriers: 1..3 in_full[s]; 4..6 in_empty[s]; 7, 8 acc1_full[b]; 9, 10 acc1_empty[b]
// (8 warps); 11, 12 x_full[b] (8 warps); 13, 14 x_empty[b] (MMA 2 done); 15 acc2_full;
// 16 acc2_empty (8 warps); 17 drain.
constexpr int kF2Stages = 3;
constexpr int kF2Prod = 18;  // first producer warp
constexpr int kThreadsF2 = (kF2Prod + 4) * 32;
constexpr int kF2Bars = 18;
enum {
  kF2InF = 1, kF2InE = 4, kF2A1F = 7, kF2A1E = 9, kF2XF = 11, kF2XE = 13, kF2A2F = 15, kF2A2E = 16,
  kF2Drain = 17
};

// Taylor-mode tanh of one accumulator tile's rows owned by this thread (feature j, point
// half hh) into a swizzled shared-memory tile, 8 points (four channels) or 8 rows (value
// channel) at a time; returns after the accumulator has been read (the caller releases it).
__device__ __forceinline__ void fwd_epilogue_tile(uint32_t acc, bool c4, int hh, int j, float bj, uint32_t dst) {
  if (c4) {
#pragma unroll 1
    for (int g = 0; g < 2; ++g) {
      uint32_t v[4][8];
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) tmem_ld8(acc + (uint32_t)(ch * 32 + 16 * hh + 8 * g), v[ch]);
      tmem_wait_ld();
      fwd_taylor8(v, bj, dst, j, 2 * hh + g);
    }
  } else {
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
      uint32_t v[8];
      tmem_ld8(acc + (uint32_t)(64 * hh + 8 * c), v);
      tmem_wait_ld();
      float o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float sd;
        tanh_sech2(__uint_as_float(v[i]) + bj, o[i], sd);
      }
      st_shared_v4(dst + tile_chunk(j, 8 * hh + c), pack2(o[0], o[1]), pack2(o[2], o[3]), pack2(o[4], o[5]),
                   pack2(o[6], o[7]));
    }
  }
}

// Warp-uniform bounded wait that sleeps between polls: for the first-layer producers,
// which run ahead of the MMA issuer, so that their waiting leaves the issue slots to the
// epilogue warps of the same scheduler.
__device__ __forceinline__ bool wait_warp_nap(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  return __all_sync(0xffffffffu, wait_nap_inl(bar, parity, abort_flag, status));
}

// One A_0 tile of C channels (PT = 128 / C points from p_begin) into the swizzled tile at
// ts: thread k (feature k) evaluates the first layer (Eq. 8) in Taylor mode for every
// point, z = B[f][k] + b0[k] + w2x x + w2y y, and stores tanh z, and for C = 4 also the
// derivative channels sech^2 z w2x, sech^2 z w2y and -2 tanh z sech^2 z |w2|^2. Point p of
// the tile is (coords[2p], coords[2p + 1]); bk_first is B[f][k] of the tile's first point.
template <int C>
__device__ __forceinline__ void first_layer_tile(uint32_t ts, const float* coords, int k, int p_begin, int R, int n,
                                                 const float* __restrict__ Bf, float bk_first, float bk0, float w2x,
                                                 float w2y, float nlap) {
  constexpr int PT = kTR / C;
  int fnext = (p_begin / n + 1) * n;  // first point of the next function
  float bk = bk_first + bk0;
#pragma unroll 1
  for (int p = 0; p < PT; p += 8) {
    const int pt0 = p_begin + p;
    if (pt0 >= R) {
#pragma unroll
      for (int c = 0; c < C; ++c) st_shared_v4(ts + tile_chunk(k, (c * PT + p) >> 3), 0u, 0u, 0u, 0u);
      continue;
    }
    if (pt0 >= fnext) {  // the tile crosses into the next function
      const int f = pt0 / n;
      fnext = (f + 1) * n;
      bk = __ldg(Bf + (size_t)f * kW + k) + bk0;
    }
    uint32_t w[C][4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      float o[4][2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float2 xy = *reinterpret_cast<const float2*>(coords + 2 * (p + i + u));
        float a, sd;
        tanh_sech2(fmaf(w2y, xy.y, fmaf(w2x, xy.x, bk)), a, sd);
        o[0][u] = a;
        o[1][u] = sd * w2x;
        o[2][u] = sd * w2y;
        o[3][u] = a * sd * nlap;
      }
#pragma unroll
      for (int c = 0; c < C; ++c) w[c][i >> 1] = pack2(o[c][0], o[c][1]);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) st_shared_v4(ts + tile_chunk(k, (c * PT + p) >> 3), w[c][0], w[c][1], w[c][2], w[c][3]);
  }
}

__global__ void __launch_bounds__(kThreadsF2, 1) tc_fwd2_kernel(const __grid_constant__ TcFwd2Params P) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen = smem_raw + (base - raw);
  const uint32_t sIn = base;                              // kF2Stages input tiles
  const uint32_t sX = sIn + kF2Stages * kTile;            // 2 tiles of A_l (MMA 2 operand, stored)
  const uint32_t sY = sX + 2 * kTile;                     // 2 staging tiles of A_{l+1}
  const uint32_t sBar = sY + 2 * kTile;
  Smem S{sBar};
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gen + (sBar - base) + 8 * kF2Bars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gen + (sBar - base) + 8 * kF2Bars + 8);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_it = P.n_tiles > (int)blockIdx.x ? (P.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kF2Stages; ++s) { mbar_init(S.bar(kF2InF + s), 1); mbar_init(S.bar(kF2InE + s), 1); }
    for (int b = 0; b < 2; ++b) {
      mbar_init(S.bar(kF2A1F + b), 1);
      mbar_init(S.bar(kF2A1E + b), 8);
      mbar_init(S.bar(kF2XF + b), 8);
      mbar_init(S.bar(kF2XE + b), 1);
    }
    mbar_init(S.bar(kF2A2F), 1);
    mbar_init(S.bar(kF2A2E), 8);
    mbar_init(S.bar(kF2Drain), 1);
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
  const uint32_t A1 = tmem, A2 = tmem + 256, W1t = tmem + 384, W2t = tmem + 448;
  if (warp >= 2 && warp < kF2Prod) {
    const int stage_b = warp >= 10 ? 1 : 0;
    const int hh = ((warp - 2) >> 2) & 1;
    const uint8_t* img = static_cast<const uint8_t*>(stage_b ? P.wimg2 : P.wimg1);
    const uint32_t wt = stage_b ? W2t : W1t;
    weights_to_tmem(img, wt, warp & 3, lane, 2 * hh);
    weights_to_tmem(img, wt, warp & 3, lane, 2 * hh + 1);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      for (int it = 0; ok && it <= n_it; ++it) {
        if (it < n_it) {  // MMA 1 of tile it: A_l^T = W_l A_{l-1}^T
          const int s = it % kF2Stages, b = it & 1;
          ok = wait_fast(S.bar(kF2InF + s), (uint32_t)((it / kF2Stages) & 1), abort_flag, P.status);
          if (ok && it >= 2) ok = wait_fast(S.bar(kF2A1E + b), (uint32_t)(((it >> 1) - 1) & 1), abort_flag, P.status);
          if (!ok) break;
          tc_fence_after();
          const uint32_t tin = sIn + (uint32_t)s * kTile;
          const uint32_t acc = A1 + (uint32_t)(b * kTR);
#pragma unroll
          for (int ks = 0; ks < kW / 16; ++ks) {
            if (ks == 0) mma_ts<0>(acc, W1t + (uint32_t)(8 * ks), desc_rows(tin, ks), kIdescRows);
            else mma_ts<1>(acc, W1t + (uint32_t)(8 * ks), desc_rows(tin, ks), kIdescRows);
          }
          mma_commit(S.bar(kF2A1F + b));
          mma_commit(S.bar(kF2InE + s));
        }
        if (it >= 1) {  // MMA 2 of tile it-1: A_{l+1}^T = W_{l+1} A_l^T, A_l from tile X
          const int i2 = it - 1, b2 = i2 & 1;
          ok = wait_fast(S.bar(kF2XF + b2), (uint32_t)((i2 >> 1) & 1), abort_flag, P.status);
          if (ok && i2 >= 1) ok = wait_fast(S.bar(kF2A2E), (uint32_t)((i2 - 1) & 1), abort_flag, P.status);
          if (!ok) break;
          tc_fence_after();
          const uint32_t tx = sX + (uint32_t)b2 * kTile;
#pragma unroll
          for (int ks = 0; ks < kW / 16; ++ks) {
            if (ks == 0) mma_ts<0>(A2, W2t + (uint32_t)(8 * ks), desc_rows(tx, ks), kIdescRows);
            else mma_ts<1>(A2, W2t + (uint32_t)(8 * ks), desc_rows(tx, ks), kIdescRows);
          }
          mma_commit(S.bar(kF2A2F));
          mma_commit(S.bar(kF2XE + b2));
        }
      }
      mma_commit(S.bar(kF2Drain));
      wait_bounded(S.bar(kF2Drain), 0, abort_flag, P.status, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0 && !P.first) {
      int issued = 0;
      for (int it = 0; it < n_it; ++it) {
        const int s = it % kF2Stages;
        if (it >= kF2Stages &&
            !wait_bounded(S.bar(kF2InE + s), (uint32_t)(((it / kF2Stages) - 1) & 1), abort_flag, P.status, true))
          break;
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        mbar_arrive_expect_tx(S.bar(kF2InF + s), kTile);
        bulk_g2s(sIn + (uint32_t)s * kTile, P.A_in + (size_t)t * kTile, kTile, S.bar(kF2InF + s));
        issued = it + 1;
      }
      for (int it = (issued > kF2Stages ? issued - kF2Stages : 0); it < issued; ++it)
        wait_bounded(S.bar(kF2InF + it % kF2Stages), (uint32_t)((it / kF2Stages) & 1), abort_flag, P.status, false);
    }
    __syncwarp();
  } else if (warp >= kF2Prod) {
    if (P.first) {
      // first-layer producers: thread k = feature k; one named barrier (3) per tile before
      // and after the slot is written, reached by all four warps, aborted or not. The
      // points' coordinates and the boundary term are fetched one tile ahead (registers,
      // then the coordinate buffer once every producer is done with the current tile),
      // so the loads' latency is hidden behind the current tile's arithmetic.
      const int k = threadIdx.x - kF2Prod * 32;
      const bool lead = k == 0;
      const float w2x = P.W0[(size_t)k * 130 + 128], w2y = P.W0[(size_t)k * 130 + 129];
      const float nlap = -2.0f * (w2x * w2x + w2y * w2y);
      const float bk0 = P.b0[k];
      float* coords = reinterpret_cast<float*>(gen + (sBar - base) + 8 * kF2Bars + 64);
      // tile it's coordinate floats k and k + 128 and the boundary term of its first function
      auto fetch = [&](int it, float& c0, float& c1, float& bf) {
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        const int term = t < P.n_tiles4 ? 0 : 1;
        const int PT = term == 0 ? kTR / 4 : kTR, tt = term == 0 ? t : t - P.n_tiles4;
        const int R = P.R[term], p0 = tt * PT;
        const float* X = P.X[term] + 2 * (size_t)p0;
        c0 = k < 2 * PT && p0 + (k >> 1) < R ? __ldg(X + k) : 0.0f;
        c1 = k + 128 < 2 * PT && p0 + ((k + 128) >> 1) < R ? __ldg(X + k + 128) : 0.0f;
        bf = p0 < R ? __ldg(P.Bf + (size_t)(p0 / P.n[term]) * kW + k) : 0.0f;
      };
      float c0 = 0.0f, c1 = 0.0f, bkf = 0.0f;
      if (n_it > 0) {
        fetch(0, c0, c1, bkf);
        coords[k] = c0;
        coords[k + 128] = c1;
      }
      bool ok = true;
      for (int it = 0; it < n_it; ++it) {
        const int s = it % kF2Stages;
        const int t = (int)blockIdx.x + it * (int)gridDim.x;
        const float bkt = bkf;
        if (it + 1 < n_it) fetch(it + 1, c0, c1, bkf);
        // MMA 1 of the slot's previous tile is done with it ...
        if (ok && it >= kF2Stages)
          ok = wait_warp_nap(S.bar(kF2InE + s), (uint32_t)(((it / kF2Stages) - 1) & 1), abort_flag, P.status);
        // ... and so is the store of that tile's A_0 (at most the two newer ones pending)
        if (lead) bulk_wait_read<kF2Stages - 1>();
        named_barrier_sync(3, 128);
        const uint32_t ts = sIn + (uint32_t)s * kTile;
        if (ok) {
          if (t < P.n_tiles4)
            first_layer_tile<4>(ts, coords, k, t * (kTR / 4), P.R[0], P.n[0], P.Bf, bkt, bk0, w2x, w2y, nlap);
          else
            first_layer_tile<1>(ts, coords, k, (t - P.n_tiles4) * kTR, P.R[1], P.n[1], P.Bf, bkt, bk0, w2x, w2y, nlap);
          fence_proxy_async_smem();
        }
        named_barrier_sync(3, 128);
        if (lead && ok && !*abort_flag) {
          bulk_s2g(P.A0_out + (size_t)t * kTile, ts, kTile);
          bulk_commit();
          mbar_arrive(S.bar(kF2InF + s));
        }
        // every producer has read this tile's coordinates: the next tile's replace them
        coords[k] = c0;
        coords[k + 128] = c1;
      }
      if (lead) bulk_wait_all<0>();
    }
  } else {
    const bool stage_b = warp >= 10;
    const int e = warp - (stage_b ? 10 : 2);  // 0..7 within the stage
    const int q = warp & 3, hh = e >> 2;
    const int j = 32 * q + lane;
    const float bj = (stage_b ? P.bias2 : P.bias1)[j];
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const int named = stage_b ? 2 : 1;
    bool ok = true;
    for (int it = 0; it < n_it; ++it) {
      const int b = it & 1;
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      const bool c4 = t < P.n_tiles4;
      uint32_t dst;
      if (!stage_b) {
        if (ok) ok = wait_warp_fast(S.bar(kF2A1F + b), (uint32_t)((it >> 1) & 1), abort_flag, P.status);
        // MMA 2 of tile it-2 has finished reading the X tile this tile rewrites
        if (ok && it >= 2) ok = wait_warp_fast(S.bar(kF2XE + b), (uint32_t)(((it >> 1) - 1) & 1), abort_flag, P.status);
        dst = sX + (uint32_t)b * kTile;
        if (ok) {
          tc_fence_after();
          fwd_epilogue_tile(A1 + (uint32_t)(b * kTR) + lane_off, c4, hh, j, bj, dst);
          tc_fence_before();
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(S.bar(kF2A1E + b));
            mbar_arrive(S.bar(kF2XF + b));
          }
        }
      } else {
        if (ok) ok = wait_warp_fast(S.bar(kF2A2F), (uint32_t)(it & 1), abort_flag, P.status);
        dst = sY + (uint32_t)b * kTile;
        if (ok) {
          tc_fence_after();
          fwd_epilogue_tile(A2 + lane_off, c4, hh, j, bj, dst);
          tc_fence_before();
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(S.bar(kF2A2E));
        }
      }
      // one barrier per tile and stage, reached by its 8 warps, aborted or not: before it,
      // the stage's thread 0 waits until the store of tile it-1 has read its tile, which
      // tile it+1 rewrites
      if (e == 0 && lane == 0) bulk_wait_read<0>();
      named_barrier_sync(named, 8 * 32);
      if (e == 0 && lane == 0 && ok && !*abort_flag) {
        bulk_s2g((stage_b ? P.A_out2 : P.A_out1) + (size_t)t * kTile, dst, kTile);
        bulk_commit();
      }
    }
    if (e == 0 && lane == 0) bulk_wait_all<0>();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------ backward kernel

// Backward kernel: 20 warps in five warpgroups. Warpgroup 0 holds the MMA issuer (warp
// 0) and the load issuer (warp 1); warps 4-19 are the epilogue (feature quadrant
// q = w mod 4, point quarter pq = (w-4)/4). The CTA is launched with kRegsLaunch registers
// per thread; warpgroup 0 then gives registers back (setmaxnreg.dec to kRegsIssue) and the
// epilogue takes them (setmaxnreg.inc to kRegsEpi), so that its chain-rule arithmetic runs
// without spills: 128 kRegsIssue + 512 kRegsEpi <= 640 kRegsLaunch. Every warp returns to
// kRegsLaunch before the common tail of the kernel; the warps of a warpgroup pass a named
// barrier between two setmaxnreg instructions (barrier 6 for warpgroup 0, 1 for the
// epilogue). Shared memory: three A_{l-1} slots (each held from MMA 1 to MMA 3 of its
// tile), two gA_l slots (held until epilogue 1 has read them), one g_Z^T tile and one
// staging tile for gA_{l-1}: 224 KB. Epilogue order 1(0), then per t: 1(t+1), 2(t), so
// that epilogue 1 of tile t+1 runs while MMAs 2 and 3 of tile t execute. W and W^T are the
// A operands of MMAs 1 and 2 from tensor memory. Barriers: 1..3 a_full[slot];
// 4..6 a_empty[slot] (MMA 3 done); 7, 8 g_full[slot]; 9, 10 g_empty[slot] (16 warps);
// 11 d1_full; 12 d1_empty; 13 gz_full; 14 gz_empty (MMA 3 done); 15 d2_full (MMA 2 done);
// 16 d2_empty; 17 d3_done; 18 drain; 19 gz_empty of the second g_Z^T buffer. The top
// layer, which loads no gA tiles, keeps two g_Z^T buffers (the second in gA slot 1), so
// that epilogue 1 of tile t need not wait for MMA 3 of tile t-1. Each barrier is waited
// on before it can complete again.
constexpr int kEpiB = 16;
constexpr int kEpiWarp0 = 4;                        // first epilogue warp
constexpr int kThreadsB = (kEpiWarp0 + kEpiB) * 32;  // 640
constexpr int kRegsLaunch = 96;                     // 65536 / 640, rounded down to a multiple of 8
constexpr int kRegsIssue = 56;
constexpr int kRegsEpi = 104;
static_assert(128 * kRegsIssue + 32 * kEpiB * kRegsEpi <= kThreadsB * kRegsLaunch,
              "the register split must fit in the launch allocation");
static_assert(32 * (kRegsIssue + 4 * kRegsEpi) <= 16384, "registers of one SM sub-partition");
constexpr int kSlotsA = 3;
constexpr int kSlotsG = 2;
constexpr int kBwdBars = 20;
enum {
  kBAF = 1, kBAE = 4, kBGF = 7, kBGE = 9, kBD1F = 11, kBD1E = 12, kBGZF = 13, kBGZE = 14, kBD2F = 15, kBD2E = 16,
  kBD3 = 17, kBDrain = 18, kBGZE1 = 19
};

// Sum of v[0..N-1] (N a power of 2 up to 32) over the 32 lanes of a warp: in the first log2 N
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

template <bool kTop, bool kFirst>
__global__ void __launch_bounds__(kThreadsB, 1) tc_bwd_kernel(const __grid_constant__ TcBwdParams P) {
  // tiles 0 .. n4-1 hold collocation points (C = 4 channels, 32 points: PT = 32, 8 points
  // per epilogue thread), the rest the value channel of data points (C = 1, PT = 128, 32
  // per thread); the epilogue takes the form of each tile
  using C4 = std::integral_constant<int, 4>;
  using C1 = std::integral_constant<int, 1>;
  const int n4 = P.term[0].n_tiles;
  const int n_all = n4 + P.term[1].n_tiles;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen = smem_raw + (base - raw);
  const uint32_t sA = base;                              // kSlotsA tiles of A_{l-1}
  const uint32_t sG = sA + kSlotsA * kTile;              // kSlotsG tiles of gA_l
  const uint32_t sGZ = sG + kSlotsG * kTile;             // the g_Z^T tile
  const uint32_t sOut = sGZ + kTile;                     // staging tile of gA_{l-1}
  // the g_Z^T buffer of tile `it` (two alternating buffers at the top), and the
  // barrier its MMA 3 completes: it waits for tile it-1 (one buffer) or it-2 (two)
  auto gz_buf = [&](int it) -> uint32_t { return (kTop && (it & 1)) ? sG + kTile : sGZ; };
  auto gz_empty_bar = [&](int it) -> int { return (kTop && (it & 1)) ? kBGZE1 : kBGZE; };
  const uint32_t sBar = sOut + kTile;
  Smem S{sBar};
  uint8_t* genBar = gen + (sBar - base);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(genBar + 8 * kBwdBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(genBar + 8 * kBwdBars + 8);
  // top layer only (no gA tiles are loaded there): the reduction scratch of the output
  // layer, [2][4 quarters][4 quadrants][up to 32 points], lives in the first gA slot
  float* red = reinterpret_cast<float*>(gen + (sG - base));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool top = kTop;
  const int n_it = n_all > (int)blockIdx.x ? (n_all - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlotsA; ++s) { mbar_init(S.bar(kBAF + s), 1); mbar_init(S.bar(kBAE + s), 1); }
    for (int s = 0; s < kSlotsG; ++s) { mbar_init(S.bar(kBGF + s), 1); mbar_init(S.bar(kBGE + s), kEpiB); }
    mbar_init(S.bar(kBD1F), 1);
    mbar_init(S.bar(kBD1E), kEpiB);
    mbar_init(S.bar(kBGZF), kEpiB);
    mbar_init(S.bar(kBGZE), 1);
    mbar_init(S.bar(kBGZE1), 1);
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
  // TMEM columns: D1 = Z^T [0, 128), D2 = gA^T [128, 256), D3 = g_W [256, 384),
  // W [384, 448) and W^T [448, 512) as A operands
  const uint32_t D1 = tmem, D2 = tmem + 128, D3 = tmem + 256, Wt = tmem + 384, WTt = tmem + 448;
  if (warp >= kEpiWarp0) {
    const int cq = (warp - kEpiWarp0) >> 2;
    weights_to_tmem(static_cast<const uint8_t*>(P.wimg), Wt, warp & 3, lane, cq);
    weights_to_tmem(static_cast<const uint8_t*>(P.wimgT), WTt, warp & 3, lane, cq);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // warpgroup 0 (issuers) gives registers to the epilogue warpgroups and takes them
  // back at the end, each warpgroup at one setmaxnreg site
  if (warp < kEpiWarp0) {
    setmaxnreg_dec<kRegsIssue>();
    if (warp == 0) {
      if (lane == 0) {
        bool ok = true;
        // MMA 1 (Z^T = W A^T) of tile `it`, once its A tile is in and D1 has been read out
        auto mma1 = [&](int it) -> bool {
          const int s = it % kSlotsA;
          if (!wait_fast(S.bar(kBAF + s), (uint32_t)((it / kSlotsA) & 1), abort_flag, P.status)) return false;
          if (it > 0 && !wait_fast(S.bar(kBD1E), (uint32_t)((it - 1) & 1), abort_flag, P.status)) return false;
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
        if (n_it > 0) ok = mma1(0);
        for (int it = 0; ok && it < n_it; ++it) {
          const int s = it % kSlotsA;
          const uint32_t ta = sA + (uint32_t)s * kTile;
          // the next tile's recompute runs while epilogue 1 of this tile works
          if (it + 1 < n_it && !mma1(it + 1)) { ok = false; break; }
          ok = wait_fast(S.bar(kBGZF), (uint32_t)(it & 1), abort_flag, P.status);
          if (ok && it > 0) ok = wait_fast(S.bar(kBD2E), (uint32_t)((it - 1) & 1), abort_flag, P.status);
          if (!ok) break;
          tc_fence_after();
          // MMA 2: gA^T = W^T g_Z^T (g_Z^T tile read MN-major: N = rows, K = features)
  #pragma unroll
          for (int ks = 0; ks < kW / 16; ++ks) {
            if (ks == 0) mma_ts<0>(D2, WTt + (uint32_t)(8 * ks), desc_rows(gz_buf(it), ks), kIdescRows);
            else mma_ts<1>(D2, WTt + (uint32_t)(8 * ks), desc_rows(gz_buf(it), ks), kIdescRows);
          }
          mma_commit(S.bar(kBD2F));
          // MMA 3: g_W += g_Z^T A (both tiles read K-major: M, N = features, K = rows)
          const uint64_t gzd = desc_sw128(gz_buf(it)), tad = desc_sw128(ta);
  #pragma unroll
          for (int ks = 0; ks < kTR / 16; ++ks) {
            const uint64_t a_op = desc_add(gzd, kstep_rows(ks));
            const uint64_t b_op = desc_add(tad, kstep_rows(ks));
            if (it == 0 && ks == 0) mma_ss<0>(D3, a_op, b_op, kIdescGW);
            else mma_ss<1>(D3, a_op, b_op, kIdescGW);
          }
          mma_commit(S.bar(gz_empty_bar(it)));
          mma_commit(S.bar(kBAE + s));
        }
        mma_commit(S.bar(kBD3));  // every MMA issued, including the last g_W accumulation, done
        mma_commit(S.bar(kBDrain));
        wait_bounded_inl(S.bar(kBDrain), 0, abort_flag, P.status, false);
      }
      __syncwarp();
    } else if (warp == 1) {
      if (lane == 0) {
        // loads in the order they fall due: gA_l of tile it, then A_{l-1} of tile it+1
        auto load = [&](int it, int slots, int full, int empty, uint32_t dst0, const uint8_t* src) -> bool {
          const int s = it % slots;
          if (it >= slots &&
              !wait_bounded_inl(S.bar(empty + s), (uint32_t)(((it / slots) - 1) & 1), abort_flag, P.status, true))
            return false;
          const int t = (int)blockIdx.x + it * (int)gridDim.x;
          mbar_arrive_expect_tx(S.bar(full + s), kTile);
          bulk_g2s(dst0 + (uint32_t)s * kTile, src + (size_t)t * kTile, kTile, S.bar(full + s));
          return true;
        };
        int na = 0, ng = 0;
        bool ok = n_it > 0 && load(0, kSlotsA, kBAF, kBAE, sA, P.A_in);
        if (ok) na = 1;
        for (int it = 0; ok && it < n_it; ++it) {
          if (!top) {
            ok = load(it, kSlotsG, kBGF, kBGE, sG, P.gA_in);
            if (ok) ng = it + 1;
          }
          if (ok && it + 1 < n_it) {
            ok = load(it + 1, kSlotsA, kBAF, kBAE, sA, P.A_in);
            if (ok) na = it + 2;
          }
        }
        // every load issued has landed before shared memory can go away
        for (int i = (na > kSlotsA ? na - kSlotsA : 0); i < na; ++i)
          wait_bounded_inl(S.bar(kBAF + i % kSlotsA), (uint32_t)((i / kSlotsA) & 1), abort_flag, P.status, false);
        for (int i = (ng > kSlotsG ? ng - kSlotsG : 0); i < ng; ++i)
          wait_bounded_inl(S.bar(kBGF + i % kSlotsG), (uint32_t)((i / kSlotsG) & 1), abort_flag, P.status, false);
      }
      __syncwarp();
    }
    // the four warps of a warpgroup synchronise between two setmaxnreg instructions
    named_barrier_sync(6, 128);
    setmaxnreg_inc<kRegsLaunch>();
  } else {
    setmaxnreg_inc<kRegsEpi>();
    // a warp reads the TMEM lane quadrant (warp index mod 4); the 16 warps cover the four
    // quadrants for each of the four point quarters of a tile
    const int e = warp - kEpiWarp0, q = warp & 3, pq = e >> 2;
    const int j = 32 * q + lane;  // feature (D1, D3 lanes) / input feature k (D2 lanes)
    const float bj = P.bias[j];
    const float wo = top ? P.wout[j] : 0.f;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    float gb = 0.f, gwo = 0.f, gbo = 0.f;
    // the running loss of each term: FP32 pair with compensation (an FP64 add per tile on
    // one lane costs hundreds of cycles and stalls its warp), turned into FP64 at the end
    float lsum[2] = {0.f, 0.f}, lcomp[2] = {0.f, 0.f};
    auto loss_add = [&](int term, float x) {
      const float y = x - lcomp[term];
      const float t2 = lsum[term] + y;
      lcomp[term] = (t2 - lsum[term]) - y;
      lsum[term] = t2;
    };
    bool ok = true;

    // MMA 3 of the tile that last used this tile's g_Z^T buffer has finished reading it
    auto wait_gz_empty = [&](int it) -> bool {
      const int back = kTop ? 2 : 1;
      if (it < back) return true;
      const int k = kTop ? (it >> 1) - 1 : it - 1;  // completion index of that barrier
      return wait_warp_fast(S.bar(gz_empty_bar(it)), (uint32_t)(k & 1), abort_flag, P.status);
    };

    // ---- epilogue 1 of tile it: g_Z from the recomputed Z and the incoming gradient
    // layer 1 (kFirst): the first layer's weights of feature j, and this warp's buffers in
    // the upper half of the staging tile (which layer 1 does not otherwise use): the
    // coordinates of its points (two tiles x 64 floats) and B[f][j] + b0[j] of their
    // function (two tiles x 32 lanes). Epilogue 1 of a tile loads them from global memory
    // at its start and stores them here at its end, so their latency is hidden behind
    // epilogue 1's work; epilogue 2 of the tile, an iteration later, reads them here.
    const float w2x = kFirst ? P.W0[(size_t)j * 130 + 128] : 0.f;
    const float w2y = kFirst ? P.W0[(size_t)j * 130 + 129] : 0.f;
    const float lap = w2x * w2x + w2y * w2y;
    const float lap6 = 6.0f * lap, lapm2 = -2.0f * lap, m4w2x = -4.0f * w2x, m4w2y = -4.0f * w2y;
    const float b0j = kFirst ? P.b0[j] : 0.f;
    float* first_buf = reinterpret_cast<float*>(gen + (sOut - base) + 16384) + e * 192;  // [2][64] xy, [2][32] B
    auto epi1_c = [&](int it, int t, auto Cc) {
      constexpr int C = decltype(Cc)::value;
      constexpr int PT = kTR / C;   // points per tile
      constexpr int NP = PT / 4;    // points per epilogue thread: 8 (C = 4) or 32 (C = 1)
      const int p0 = pq * NP;
      const TcTerm& T = P.term[C == 4 ? 0 : 1];
      const int tl = C == 4 ? t : t - n4;  // the tile within its term
      const int sgs = it % kSlotsG;
      const uint32_t sg = sG + (uint32_t)sgs * kTile;
      float* rb = red + (it & 1) * (16 * 32);  // top: [4 quarters][4 quadrants][NP points]
      [[maybe_unused]] float xc0 = 0.f, xc1 = 0.f, bkc = 0.f;
      if constexpr (kFirst) {
        // this warp's points' coordinates (NP points, 2 NP floats: lane l takes floats l and
        // 32 + l) and B + b0 of their function, for epilogue 2 of this tile
        const int pt_q = tl * PT + p0;
        const float* Xq = T.X + 2 * (size_t)pt_q;
        if (lane < 2 * NP && pt_q + (lane >> 1) < T.n_pts) xc0 = __ldg(Xq + lane);
        if (32 + lane < 2 * NP && pt_q + 16 + (lane >> 1) < T.n_pts) xc1 = __ldg(Xq + 32 + lane);
        if (pt_q < T.n_pts) bkc = __ldg(P.Bf + (size_t)(pt_q / T.n_per_fn) * kW + j) + b0j;
      }
      if (ok) ok = wait_warp_fast(S.bar(kBD1F), (uint32_t)(it & 1), abort_flag, P.status);
      if (ok && !top) ok = wait_warp_fast(S.bar(kBGF + sgs), (uint32_t)((it / kSlotsG) & 1), abort_flag, P.status);
      if (ok) tc_fence_after();
      if constexpr (C == 4) {
        // D1 columns of the 8 points: z, z_x, z_y, Delta z; D1 and the gA slot are released
        // as soon as they are read
        uint32_t v[4][8];
        uint4 gin[4];  // incoming gradient chunks, one per channel, as BF16 pairs
        if (ok) {
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) tmem_ld8(D1 + lane_off + (uint32_t)(ch * PT + p0), v[ch]);
          if (!top)
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) gin[ch] = ld_shared_v4(sg + tile_chunk(j, 4 * ch + pq));
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(S.bar(kBD1E));
            if (!top) mbar_arrive(S.bar(kBGE + sgs));
          }
        } else {
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
#pragma unroll
            for (int i = 0; i < 8; ++i) v[ch][i] = 0u;
        }
        float la[8], gu[8];  // top: Delta a of the points, and the gradient reaching Delta a
        float ta[8], ts[8];  // top: tanh and sech^2 of the points, kept for the chain rule
        if (top) {
          // Delta u = w_out . Delta a over the 128 features: shuffles (warp_sum_n) and the
          // four quadrant warps of this point quarter
          float part[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            tanh_sech2(__uint_as_float(v[0][i]) + bj, ta[i], ts[i]);
            const float a = ta[i], sd = ts[i];
            const float zx = __uint_as_float(v[1][i]), zy = __uint_as_float(v[2][i]);
            la[i] = fmaf(-2.0f * a * sd, zx * zx + zy * zy, sd * __uint_as_float(v[3][i]));
            part[i] = wo * la[i];
          }
          int idx;
          const float tot = warp_sum_n<8>(part, lane, idx);
          // the scratch alternates between tiles, so one barrier per tile suffices: a
          // quarter's warps rewrite a half only after all of them passed the barrier of
          // the tile after the one that read it
          if ((lane & 3) == 0) rb[(pq * 4 + q) * NP + idx] = tot;
          named_barrier_sync(2 + pq, 128);
          // the tile's squared residuals are summed in FP32, the running total in FP64
          float lt = 0.f;
          float dsum4[4];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            // Delta u of point i (collocation tiles are always full): the four quadrants'
            // sums, read 4 points at a time with 16-byte loads, added in quadrant order
            if ((i & 3) == 0) quad_sum4(rb + (pq * 4) * NP + i, NP, dsum4);
            const float d = dsum4[i & 3];
            const float g = T.gscale * d;
            gu[i] = g * wo;
            gwo = fmaf(g, la[i], gwo);
            lt = fmaf(d, d, lt);
          }
          if (ok) loss_add(0, lt);
        }
        // the g_Z^T buffer this tile rewrites is free again
        if (ok) ok = wait_gz_empty(it);
        if (ok) {
          uint32_t w[4][4];
          if constexpr (kTop || kFirst) {
            // the top and layer 1 are bound by their epilogues' instruction issue: two
            // points per packed instruction
#pragma unroll
            for (int i = 0; i < 8; i += 2) {  // points i and i + 1
              float2 a, sd, ga3;
              [[maybe_unused]] float2 ga0, ga1, ga2;  // not used at the top
              if constexpr (kTop) {
                a = make_float2(ta[i], ta[i + 1]);
                sd = make_float2(ts[i], ts[i + 1]);
                ga3 = make_float2(gu[i], gu[i + 1]);  // the top's gradient reaches Delta a only
              } else {
                tanh_sech2_x2(add2(f2(v[0][i], v[0][i + 1]), f2(bj)), a, sd);
                ga0 = make_float2(bf16_word(gin[0], i), bf16_word(gin[0], i + 1));
                ga1 = make_float2(bf16_word(gin[1], i), bf16_word(gin[1], i + 1));
                ga2 = make_float2(bf16_word(gin[2], i), bf16_word(gin[2], i + 1));
                ga3 = make_float2(bf16_word(gin[3], i), bf16_word(gin[3], i + 1));
              }
              const float2 zx = f2(v[1][i], v[1][i + 1]), zy = f2(v[2][i], v[2][i + 1]), zl = f2(v[3][i], v[3][i + 1]);
              // td = tanh''(z) = -2 a s and tp = tanh'''(z) = s (4 a^2 - 2 s)
              const float2 td = mul2(mul2(a, f2(-2.0f)), sd);
              const float2 tp = mul2(sd, fma2(mul2(a, a), f2(4.0f), mul2(sd, f2(-2.0f))));
              const float2 q2 = fma2(zx, zx, mul2(zy, zy));
              const float2 lap = fma2(tp, q2, mul2(td, zl));
              const float2 t2 = mul2(mul2(ga3, td), f2(2.0f));
              float2 g0, o1, o2;
              if constexpr (kTop) {
                g0 = mul2(ga3, lap);
                o1 = mul2(t2, zx);
                o2 = mul2(t2, zy);
              } else {
                g0 = fma2(ga0, sd, fma2(fma2(ga1, zx, mul2(ga2, zy)), td, mul2(ga3, lap)));
                o1 = fma2(ga1, sd, mul2(t2, zx));
                o2 = fma2(ga2, sd, mul2(t2, zy));
              }
              const float2 o3 = mul2(ga3, sd);
              gb += g0.x;
              gb += g0.y;
              w[0][i >> 1] = pack2(g0.x, g0.y);
              w[1][i >> 1] = pack2(o1.x, o1.y);
              w[2][i >> 1] = pack2(o2.x, o2.y);
              w[3][i >> 1] = pack2(o3.x, o3.y);
            }
          } else {
            // hidden layers are bound by DRAM; the scalar form needs fewer registers
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
              float o[4][2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int k = i + u;
                float a, sd;
                tanh_sech2(__uint_as_float(v[0][k]) + bj, a, sd);
                const float zx = __uint_as_float(v[1][k]), zy = __uint_as_float(v[2][k]), zl = __uint_as_float(v[3][k]);
                float ga[4];
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) ga[ch] = bf16_word(gin[ch], k);
                const float td = -2.0f * a * sd;
                const float tp = -2.0f * sd * sd + 4.0f * a * a * sd;
                const float q2 = zx * zx + zy * zy;
                const float g0 = ga[0] * sd + (ga[1] * zx + ga[2] * zy) * td + ga[3] * fmaf(tp, q2, td * zl);
                o[0][u] = g0;
                o[1][u] = fmaf(ga[1], sd, 2.0f * ga[3] * td * zx);
                o[2][u] = fmaf(ga[2], sd, 2.0f * ga[3] * td * zy);
                o[3][u] = ga[3] * sd;
                gb += g0;
              }
#pragma unroll
              for (int ch = 0; ch < 4; ++ch) w[ch][i >> 1] = pack2(o[ch][0], o[ch][1]);
          }
          }
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
            st_shared_v4(gz_buf(it) + tile_chunk(j, 4 * ch + pq), w[ch][0], w[ch][1], w[ch][2], w[ch][3]);
        }
      } else {
        // value channel: 32 points per thread in groups of 8, each group read from D1 (and
        // the gA slot) when it is worked on; both are released after the last group
        if (top) {
          // u = w_out . a + b_out over the 128 features
#pragma unroll 1
          for (int g8 = 0; g8 < 4; ++g8) {
            uint32_t v[8];
            if (ok) {
              tmem_ld8(D1 + lane_off + (uint32_t)(p0 + 8 * g8), v);
              tmem_wait_ld();
            }
            float part[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float a, sd;
              tanh_sech2(ok ? __uint_as_float(v[i]) + bj : 0.f, a, sd);
              part[i] = wo * a;
            }
            int idx;
            const float tot = warp_sum_n<8>(part, lane, idx);
            if ((lane & 3) == 0) rb[(pq * 4 + q) * NP + 8 * g8 + idx] = tot;
          }
          named_barrier_sync(2 + pq, 128);
        }
        if (ok) ok = wait_gz_empty(it);
        const float bo = top ? *P.bout : 0.f;
        float lt = 0.f, gt = 0.f;  // top: the tile's squared residuals and their gradients
#pragma unroll 1
        for (int g8 = 0; g8 < 4; ++g8) {
          uint32_t v[8];
          uint4 gin = make_uint4(0u, 0u, 0u, 0u);
          if (ok) {
            tmem_ld8(D1 + lane_off + (uint32_t)(p0 + 8 * g8), v);
            if (!top) gin = ld_shared_v4(sg + tile_chunk(j, 4 * pq + g8));
            tmem_wait_ld();
          }
          float o[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int k = 8 * g8 + i;
            float a, sd;
            tanh_sech2(ok ? __uint_as_float(v[i]) + bj : 0.f, a, sd);
            float ga;
            if (top) {
              const float sum = rb[(pq * 4 + 0) * NP + k] + rb[(pq * 4 + 1) * NP + k] + rb[(pq * 4 + 2) * NP + k] +
                                rb[(pq * 4 + 3) * NP + k];
              // u - y; the padding past the last data point has no residual
              const int pt = tl * PT + p0 + k;
              const float d = pt < T.n_pts ? sum + bo - T.Y[pt] : 0.f;
              const float g = T.gscale * d;
              ga = g * wo;
              gwo = fmaf(g, a, gwo);
              lt = fmaf(d, d, lt);
              gt += g;
            } else {
              ga = bf16_word(gin, i);
            }
            o[i] = ga * sd;
            gb += o[i];
          }
          if (ok)
            st_shared_v4(gz_buf(it) + tile_chunk(j, 4 * pq + g8), pack2(o[0], o[1]), pack2(o[2], o[3]), pack2(o[4], o[5]),
                         pack2(o[6], o[7]));
        }
        if (top && ok) {
          loss_add(1, lt);
          gbo += gt;
        }
        if (ok) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(S.bar(kBD1E));
            if (!top) mbar_arrive(S.bar(kBGE + sgs));
          }
        }
      }
      if (ok) {
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(S.bar(kBGZF));
      }
      if constexpr (kFirst) {
        __syncwarp();
        float* fb = first_buf + (it & 1) * 64;
        fb[lane] = xc0;
        fb[32 + lane] = xc1;
        first_buf[128 + (it & 1) * 32 + lane] = bkc;
        __syncwarp();
      }
    };

    auto tile_of = [&](int it) { return (int)blockIdx.x + it * (int)gridDim.x; };

    // ---- epilogue 2 of layer 1 (kFirst): gA_0 of this thread's points stays on chip and
    // goes through the first layer's backward (Eq. 8 in Taylor mode, the formulas of
    // tc_first_bwd_kernel) into per-32-point partial sums of g_z, g_z x + g_zx and
    // g_z y + g_zy for feature j; no gA_0 tile is written.
    auto epi2_first = [&](int it, int t, auto Cc) {
      constexpr int C = decltype(Cc)::value;
      constexpr int PT = kTR / C;
      constexpr int NP = PT / 4;
      const int p0 = pq * NP;
      const TcTerm& T = P.term[C == 4 ? 0 : 1];
      const int tl = C == 4 ? t : t - n4;
      const int pt_q = tl * PT + p0;  // this thread's first point
      // coordinates and B + b0, loaded by this warp's epilogue 1 of the tile
      const float* xyb = first_buf + (it & 1) * 64;
      const float bk = first_buf[128 + (it & 1) * 32 + lane];
      uint32_t v[C == 4 ? 4 : 1][C == 4 ? 8 : 32];
      if (ok) ok = wait_warp_fast(S.bar(kBD2F), (uint32_t)(it & 1), abort_flag, P.status);
      if (ok) {
        tc_fence_after();
        if constexpr (C == 4) {
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) tmem_ld8(D2 + lane_off + (uint32_t)(ch * PT + p0), v[ch]);
        } else {
          tmem_ld32(D2 + lane_off + (uint32_t)p0, v[0]);
        }
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(S.bar(kBD2E));
      }
      float s0 = 0.f, sx = 0.f, sy = 0.f;
      if (ok) {
#pragma unroll
        for (int g8 = 0; g8 < NP / 8; ++g8) {
          const int pt0 = pt_q + 8 * g8;
          if (pt0 >= T.n_pts) break;  // padding of the value channel's last tile
          float xy[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) xy[u] = xyb[16 * g8 + u];
          if constexpr (C == 4) {
            // two points per packed instruction, even and odd points in separate partial
            // sums (added after the group)
            float2 s02 = f2(0.f), sx2 = f2(0.f), sy2 = f2(0.f);
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
              const float2 x = make_float2(xy[2 * i], xy[2 * i + 2]), y = make_float2(xy[2 * i + 1], xy[2 * i + 3]);
              float2 a, sd;
              tanh_sech2_x2(fma2(f2(w2y), y, fma2(f2(w2x), x, f2(bk))), a, sd);
              const float2 g0 = f2(v[0][i], v[0][i + 1]), g1 = f2(v[1][i], v[1][i + 1]);
              const float2 g2 = f2(v[2][i], v[2][i + 1]), g3 = f2(v[3][i], v[3][i + 1]);
              // with s = sech^2 z, ds/dz = -2 tanh z s and d(-2 tanh z s)/dz = s (6 tanh^2 z - 2):
              //   g_z = s (g0 - 2 a (g1 w2x + g2 w2y) + g3 |w2|^2 (6 a^2 - 2)),
              //   g_w2x += g_z x + s (g1 - 4 a g3 w2x), g_w2y likewise
              const float2 gw = fma2(g1, f2(w2x), mul2(g2, f2(w2y)));
              const float2 q = fma2(f2(lap6), mul2(a, a), f2(lapm2));
              const float2 gz = mul2(sd, fma2(mul2(a, f2(-2.0f)), gw, fma2(g3, q, g0)));
              const float2 t3 = mul2(g3, a);
              s02 = add2(s02, gz);
              sx2 = fma2(sd, fma2(t3, f2(m4w2x), g1), fma2(gz, x, sx2));
              sy2 = fma2(sd, fma2(t3, f2(m4w2y), g2), fma2(gz, y, sy2));
            }
            s0 += s02.x + s02.y;
            sx += sx2.x + sx2.y;
            sy += sy2.x + sy2.y;
          }
          if constexpr (C == 1) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float x = xy[2 * i], y = xy[2 * i + 1];
              float a, sd;
              tanh_sech2(fmaf(w2y, y, fmaf(w2x, x, bk)), a, sd);
              const float gz = __uint_as_float(v[0][8 * g8 + i]) * sd;
              s0 += gz;
              sx = fmaf(gz, x, sx);
              sy = fmaf(gz, y, sy);
            }
          }
        }
      }
      if constexpr (C == 4) {
        // the tile's 32 points are one group: the four point quarters are added through
        // shared memory (the idle staging tile), alternating halves so that one barrier
        // per tile suffices. Only the four warps of this lane quadrant (features
        // 32 q .. 32 q + 31, one warp per point quarter) touch these entries, so the
        // barrier is theirs alone (ids 7 + q).
        float* r2 = reinterpret_cast<float*>(gen + (sOut - base)) + (it & 1) * (4 * 3 * kW);
        r2[(pq * 3 + 0) * kW + j] = s0;
        r2[(pq * 3 + 1) * kW + j] = sx;
        r2[(pq * 3 + 2) * kW + j] = sy;
        named_barrier_sync(7 + q, 128);
        if (pq == 0 && ok) {
          float* o = T.part32 + (size_t)tl * 3 * kW;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            o[c * kW + j] = (r2[c * kW + j] + r2[(3 + c) * kW + j]) + (r2[(6 + c) * kW + j] + r2[(9 + c) * kW + j]);
        }
      } else {
        // each point quarter (32 points) is one group
        if (ok && pt_q < T.n_pts) {
          float* o = T.part32 + (size_t)(pt_q / 32) * 3 * kW;
          o[j] = s0;
          o[kW + j] = sx;
          o[2 * kW + j] = sy;
        }
      }
    };

    // ---- epilogue 2 of tile it: the gA_{l-1} tile (row = this thread's input feature).
    // Two barriers: the store of tile it-1 has read the staging tile before anyone
    // rewrites it, and every row is written before thread 0 stores the tile. D2 is
    // released after the staging writes.
    auto epi2_c = [&](int it, int t, auto Cc) {
      constexpr int C = decltype(Cc)::value;
      constexpr int PT = kTR / C;
      constexpr int NP = PT / 4;
      [[maybe_unused]] const int p0 = pq * NP;
      // chunk of channel ch of this thread's points: C = 4 -> one chunk (8 points) per
      // channel, C = 1 -> chunks 4 pq .. 4 pq + 3 (cc = 0..3)
      auto chunk = [&](int ch, int cc) -> int { return C == 4 ? 4 * ch + pq : 4 * pq + cc; };
      if constexpr (kFirst) {
        epi2_first(it, t, Cc);
      } else {
      uint32_t v[C == 4 ? 4 : 1][C == 4 ? 8 : 32];
      if (ok) ok = wait_warp_fast(S.bar(kBD2F), (uint32_t)(it & 1), abort_flag, P.status);
      if (ok) {
        tc_fence_after();
        if constexpr (C == 4) {
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) tmem_ld8(D2 + lane_off + (uint32_t)(ch * PT + p0), v[ch]);
        } else {
          tmem_ld32(D2 + lane_off + (uint32_t)p0, v[0]);
        }
        tmem_wait_ld();
      }
      if (e == 0 && lane == 0) bulk_wait_read<0>();
      named_barrier_sync(1, kEpiB * 32);
      if (ok) {
#pragma unroll
        for (int ch = 0; ch < C; ++ch)
#pragma unroll
          for (int cc = 0; cc < NP / 8; ++cc) {
            const uint32_t* w = v[ch] + 8 * cc;
            st_shared_v4(sOut + tile_chunk(j, chunk(ch, cc)), pack2(__uint_as_float(w[0]), __uint_as_float(w[1])),
                         pack2(__uint_as_float(w[2]), __uint_as_float(w[3])),
                         pack2(__uint_as_float(w[4]), __uint_as_float(w[5])),
                         pack2(__uint_as_float(w[6]), __uint_as_float(w[7])));
          }
        fence_proxy_async_smem();
        // D2 is released only now: MMAs 2 and 3 of the next tile, which it lets start,
        // read shared memory at full rate and would slow these stores down
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(S.bar(kBD2E));
      }
      named_barrier_sync(1, kEpiB * 32);
      if (e == 0 && lane == 0 && ok && !*abort_flag) {
        bulk_s2g(P.gA_out + (size_t)t * kTile, sOut, kTile);
        bulk_commit();
      }
      }
    };
    // Epilogue order 1(0), then per it: 1(it+1), 2(it). This CTA's collocation tiles are
    // its iterations 0 .. k4-1, its data tiles k4 .. n_it-1; each stretch runs in a loop
    // of its own form (one loop body holding both forms would not fit the registers), with
    // one iteration in between that ends the first form and starts the second.
    const int k4 = n4 > (int)blockIdx.x ? (n4 - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (n_it > 0) {
      if (k4 > 0) epi1_c(0, tile_of(0), C4{});
      else epi1_c(0, tile_of(0), C1{});
    }
    for (int it = 0; it + 1 < k4; ++it) {
      epi1_c(it + 1, tile_of(it + 1), C4{});
      epi2_c(it, tile_of(it), C4{});
    }
    if (k4 > 0) {
      if (k4 < n_it) epi1_c(k4, tile_of(k4), C1{});
      epi2_c(k4 - 1, tile_of(k4 - 1), C4{});
    }
    for (int it = k4; it < n_it; ++it) {
      if (it + 1 < n_it) epi1_c(it + 1, tile_of(it + 1), C1{});
      epi2_c(it, tile_of(it), C1{});
    }
    if (e == 0 && lane == 0) bulk_wait_all<0>();
    // per-CTA partial sums: g_W (this warp's quadrant of rows, quarter of columns), g_b,
    // and at the top the output layer and the loss
    if (ok && n_it > 0) ok = wait_warp_fast(S.bar(kBD3), 0, abort_flag, P.status);
    float* gwp = P.gW_part + (size_t)blockIdx.x * kW * kW;
    const int k0 = 32 * pq;
    if (ok && n_it > 0) {
      tc_fence_after();
      uint32_t v[32];
      tmem_ld32(D3 + lane_off + (uint32_t)k0, v);
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
        if (P.term[0].loss_part) P.term[0].loss_part[blockIdx.x * 4 + pq] = ok ? (double)lsum[0] - (double)lcomp[0] : 0.0;
        if (P.term[1].loss_part) P.term[1].loss_part[blockIdx.x * 4 + pq] = ok ? (double)lsum[1] - (double)lcomp[1] : 0.0;
        P.gbout_part[blockIdx.x * 4 + pq] = ok ? gbo : 0.f;
      }
    }
    named_barrier_sync(1, kEpiB * 32);
    setmaxnreg_dec<kRegsLaunch>();
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
// mode (z_x = W2[:,0], z_y = W2[:,1], Delta z = 0). One block of 128 threads per tile:
// thread k computes feature k, 8 points at a time (each channel of the 8 points is one
// 16-byte chunk), into the tile in shared memory; the block then writes the 32 KB tile
// out with coalesced 16-byte stores. Rows past the last point (the padding of the last
// tile) are zeros.
__global__ void __launch_bounds__(kW) tc_first_fwd_kernel(const float* __restrict__ Bf, const float* __restrict__ W0,
                                                          const float* __restrict__ b0, const float* __restrict__ X,
                                                          int n, int R, int C, uint8_t* __restrict__ A0) {
  __shared__ __align__(16) uint8_t tile_s[kTile];
  const int k = threadIdx.x;
  const int PT = kTR / C, t = blockIdx.x;
  const uint32_t ts = smem_addr(tile_s);
  const float w2x = W0[(size_t)k * 130 + 128], w2y = W0[(size_t)k * 130 + 129];
  const float lap = w2x * w2x + w2y * w2y;
  const float bk0 = b0[k];
  for (int p = 0; p < PT; p += 8) {
    const int pt0 = t * PT + p;
    if (pt0 >= R) {
      for (int c = 0; c < C; ++c) st_shared_v4(ts + tile_chunk(k, (c * PT + p) >> 3), 0u, 0u, 0u, 0u);
      continue;
    }
    const float bk = Bf[(size_t)(pt0 / n) * kW + k] + bk0;
    uint32_t w[4][4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      float o[4][2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float x = X[2 * (size_t)(pt0 + i + u)], y = X[2 * (size_t)(pt0 + i + u) + 1];
        float a, sd;
        tanh_sech2(fmaf(w2y, y, fmaf(w2x, x, bk)), a, sd);
        o[0][u] = a;
        o[1][u] = sd * w2x;
        o[2][u] = sd * w2y;
        o[3][u] = -2.0f * a * sd * lap;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) w[c][i >> 1] = pack2(o[c][0], o[c][1]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < C) st_shared_v4(ts + tile_chunk(k, (c * PT + p) >> 3), w[c][0], w[c][1], w[c][2], w[c][3]);
  }
  __syncthreads();
  const uint4* src = reinterpret_cast<const uint4*>(tile_s);
  uint4* dst = reinterpret_cast<uint4*>(A0 + (size_t)t * kTile);
#pragma unroll 4
  for (int i = threadIdx.x; i < (int)(kTile / 16); i += kW) dst[i] = src[i];
}

// First-layer backward from the gA_0 tiles: g_z, g_zx, g_zy per (point, feature) and
// the block partials of sum g_z, sum g_z x + g_zx, sum g_z y + g_zy ([3][128] per block
// of 64 points; a block never spans two functions since n is a multiple of 64). The
// block's rows of gA_0 (two tiles for the four channels, one 64-row half of a tile for the
// value channel) are first copied to shared memory with coalesced 16-byte loads.
__global__ void __launch_bounds__(kW) tc_first_bwd_kernel(const float* __restrict__ Bf, const float* __restrict__ W0,
                                                          const float* __restrict__ b0, const float* __restrict__ X,
                                                          int n, int R, int C, const uint8_t* __restrict__ gA0,
                                                          float* __restrict__ part) {
  __shared__ __align__(16) uint8_t tile_s[kTile];
  const int j = threadIdx.x;  // 128 threads: one feature, 64 points
  const float w2x = W0[(size_t)j * 130 + 128], w2y = W0[(size_t)j * 130 + 129];
  const float bj = b0[j];
  const float lap = w2x * w2x + w2y * w2y;
  const int PT = kTR / C;
  const uint32_t ts = smem_addr(tile_s);
  float s0 = 0.f, sx = 0.f, sy = 0.f;
  const int pt_begin = blockIdx.x * 64;
  const int piece = C == 4 ? PT : 64;  // points per shared-memory piece
  for (int q0 = pt_begin; q0 < pt_begin + 64 && q0 < R; q0 += piece) {
    // the piece: tile q0 / PT (C = 4), or its 64-row half holding points q0 .. q0 + 63 (C = 1)
    const uint32_t base_off = C == 4 ? 0u : (uint32_t)((q0 % PT) / 64) * kHalf;
    const uint32_t bytes = C == 4 ? kTile : kHalf;
    const uint4* src = reinterpret_cast<const uint4*>(gA0 + (size_t)(q0 / PT) * kTile + base_off);
    __syncthreads();  // the previous piece has been read
    uint4* dst = reinterpret_cast<uint4*>(tile_s);
#pragma unroll 4
    for (int i = threadIdx.x; i < (int)(bytes / 16); i += kW) dst[i] = src[i];
    __syncthreads();
    const int f = q0 / n;
    const float bk = Bf[(size_t)f * kW + j] + bj;
    for (int pt0 = q0; pt0 < q0 + piece; pt0 += 8) {
      const int p = pt0 % PT;
      float ga[4][8];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < C) unpack8(ld_shared_v4(ts + tile_chunk(j, (c * PT + p) >> 3) - base_off), ga[c]);
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
  }
  float* o = part + (size_t)blockIdx.x * 3 * kW;
  o[j] = s0;
  o[kW + j] = sx;
  o[2 * kW + j] = sy;
}

// Every hidden layer's W (FP32, [out][in]) -> its two BF16 images in the K-major
// 128-byte-swizzled operand layout, W itself (rows = out) and W^T (rows = in), in one
// launch: block (element block, orientation, layer).
__global__ void tc_pack_kernel(TcPackLayers L, uint16_t* __restrict__ images) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kW * kW) return;
  const int transpose = blockIdx.y, l = blockIdx.z;
  const float* __restrict__ W = L.W[l];
  uint16_t* img = images + ((size_t)l * 2 + transpose) * (kWImg / 2);
  const int row = idx / kW, k = idx % kW;
  const float v = transpose ? W[(size_t)k * kW + row] : W[(size_t)row * kW + k];
  const uint32_t off = (uint32_t)(k >> 6) * (kW * 128u) + (uint32_t)row * 128u +
                       ((((uint32_t)(k & 63) >> 3) ^ (uint32_t)(row & 7)) << 4) + (uint32_t)(k & 7) * 2u;
  img[off / 2] = bf16_bits(v);
}

// Sum of p[b * stride] over the rows b = r0, r0 + 8, r0 + 16, ... below r1, in four
// interleaved partial sums (rows 32k + r0, + 8, + 16, + 24) added in a fixed order, so
// that four loads are in flight per thread and the result does not depend on timing.
__device__ __forceinline__ float col_sum_stride8(const float* __restrict__ p, int r0, int r1, size_t stride) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  int b = r0;
  for (; b + 24 < r1; b += 32) {
    a0 += p[(size_t)b * stride];
    a1 += p[(size_t)(b + 8) * stride];
    a2 += p[(size_t)(b + 16) * stride];
    a3 += p[(size_t)(b + 24) * stride];
  }
  if (b < r1) a0 += p[(size_t)b * stride];
  if (b + 8 < r1) a1 += p[(size_t)(b + 8) * stride];
  if (b + 16 < r1) a2 += p[(size_t)(b + 16) * stride];
  return (a0 + a1) + (a2 + a3);
}

// out[j] (+)= sum over b < nblk of part[b * stride + j]. A block covers 32 columns with
// 8 row groups (group r adds rows r, r + 8, ... with col_sum_stride8); the group sums
// are combined in a fixed order, so the result does not depend on timing.
__global__ void tc_colsum_kernel(const float* __restrict__ part, int nblk, int stride, int n, float* __restrict__ out,
                                 int accumulate) {
  __shared__ float sm[8][32];
  const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + c;
  sm[r][c] = j < n ? col_sum_stride8(part + j, r, nblk, (size_t)stride) : 0.f;
  __syncthreads();
  if (r == 0 && j < n) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += sm[k][c];
    out[j] = accumulate ? out[j] + t : t;
  }
}

// Column sums of a tall matrix (nrows x ncols, row stride `stride`), first stage: block
// (x, g) adds rows [g rpc, (g + 1) rpc) of columns 32x .. 32x + 31 into scratch[g][col]
// (8 row groups per block, combined in a fixed order). The second stage is
// tc_colsum_kernel over the G rows of scratch.
__global__ void tc_colsum_stage1_kernel(const float* __restrict__ part, int nrows, int stride, int ncols, int rpc,
                                        float* __restrict__ scratch) {
  __shared__ float sm[8][32];
  const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + c;
  const int r0 = blockIdx.y * rpc, r1 = min(nrows, r0 + rpc);
  sm[r][c] = col < ncols ? col_sum_stride8(part + col, r0 + r, r1, (size_t)stride) : 0.f;
  __syncthreads();
  if (r == 0 && col < ncols) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += sm[k][c];
    scratch[(size_t)blockIdx.y * ncols + col] = t;
  }
}

// Column sums of several layers' partials at once: layer l = blockIdx.y has an
// nrows x ncols matrix at part + l layer_stride, added into out + off[l]; per column the
// same 8-row-group scheme as tc_colsum_kernel.
struct TcLayerOffsets {
  long long off[kTcMaxLayers];
};
__global__ void tc_colsum_layers_kernel(const float* __restrict__ part, size_t layer_stride, int nrows, int ncols,
                                        float* __restrict__ out, const TcLayerOffsets offs) {
  __shared__ float sm[8][32];
  const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + c;
  const float* pl = part + (size_t)blockIdx.y * layer_stride;
  sm[r][c] = j < ncols ? col_sum_stride8(pl + j, r, nrows, (size_t)ncols) : 0.f;
  __syncthreads();
  if (r == 0 && j < ncols) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += sm[k][c];
    out[offs.off[blockIdx.y] + j] += t;
  }
}

// *out += scale x (sum of part[0..n)), one warp: lane l adds part[l], part[l + 32], ...,
// then the 32 lane sums are combined by a fixed butterfly, so the result does not depend
// on timing.
__global__ void tc_sum_double_kernel(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) s += part[i];
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if (threadIdx.x == 0) *out += s * scale;
}

// *out += sum of part[0..n), one warp in the same fixed order as tc_sum_double_kernel
__global__ void tc_sum_float_kernel(const float* __restrict__ part, int n, float* __restrict__ out) {
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += 32) s += part[i];
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if (threadIdx.x == 0) *out += s;
}

constexpr size_t kFwdSmem = 1024 + kStagesF * kTile + 2 * kTile + 8 * kFwdBars + 16 + 64;
constexpr size_t kBwdSmem = 1024 + (kSlotsA + kSlotsG + 2) * kTile + 8 * kBwdBars + 16 + 64;
constexpr size_t kFwd2Smem = 1024 + (kF2Stages + 4) * kTile + 8 * kF2Bars + 64 + 1024;  // + point coordinates
static_assert(kFwd2Smem <= 232448, "two-layer forward kernel shared memory");
static_assert(kFwdSmem <= 232448, "forward kernel shared memory");
static_assert(kBwdSmem <= 232448, "backward kernel shared memory");

int grid_for(int n_tiles) {
  int sms = 0;
  if (device_sms(&sms) != cudaSuccess || sms < 1) sms = 1;
  return n_tiles < sms ? n_tiles : sms;
}

}  // namespace

size_t tc_tile_bytes() { return kTile; }
int tc_tiles(int R, int C) { return (int)(((long long)R * C + kTR - 1) / kTR); }
int tc_partial_groups() { return 4; }
size_t tc_image_bytes() { return kWImg; }
int tc_partial_ctas() { return grid_for(1 << 30); }

cudaError_t tc_pack_layers(const TcPackLayers& L, int n_layers, void* images, cudaStream_t st) {
  if (n_layers < 1 || n_layers > kTcMaxLayers) return cudaErrorInvalidValue;
  tc_pack_kernel<<<dim3(kW * kW / 256, 2, n_layers), 256, 0, st>>>(L, static_cast<uint16_t*>(images));
  return cudaGetLastError();
}

cudaError_t tc_first_fwd(const float* Bf, const float* W0, const float* b0, const float* X, int n, int R, int C,
                         void* A0, cudaStream_t st) {
  const int tiles = tc_tiles(R, C);
  if (tiles == 0) return cudaSuccess;
  tc_first_fwd_kernel<<<tiles, kW, 0, st>>>(Bf, W0, b0, X, n, R, C, static_cast<uint8_t*>(A0));
  return cudaGetLastError();
}

cudaError_t tc_first_bwd(const float* Bf, const float* W0, const float* b0, const float* X, int n, int R, int C,
                         const void* gA0, float* part, cudaStream_t st) {
  tc_first_bwd_kernel<<<(R + 63) / 64, kW, 0, st>>>(Bf, W0, b0, X, n, R, C, static_cast<const uint8_t*>(gA0), part);
  return cudaGetLastError();
}

cudaError_t tc_layer_fwd2(const TcFwd2Params& p, cudaStream_t st) {
  static PerDevice pd;
  cudaError_t e = per_device(pd, [](int, int*, size_t*) {
    return cudaFuncSetAttribute(tc_fwd2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwd2Smem);
  });
  if (e != cudaSuccess) return e;
  if (p.n_tiles <= 0) return cudaSuccess;
  tc_fwd2_kernel<<<grid_for(p.n_tiles), kThreadsF2, kFwd2Smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t tc_layer_fwd(const TcFwdParams& p, cudaStream_t st) {
  static PerDevice pd;
  cudaError_t e = per_device(pd, [](int, int*, size_t*) {
    return cudaFuncSetAttribute(tc_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
  });
  if (e != cudaSuccess) return e;
  if (p.n_tiles <= 0) return cudaSuccess;
  tc_fwd_kernel<<<grid_for(p.n_tiles), kThreadsTc, kFwdSmem, st>>>(p);
  return cudaGetLastError();
}

template <bool kTop, bool kFirst>
cudaError_t launch_bwd(const TcBwdParams& p, int grid, cudaStream_t st) {
  static PerDevice pd;
  cudaError_t e = per_device(pd, [](int, int*, size_t*) {
    return cudaFuncSetAttribute(tc_bwd_kernel<kTop, kFirst>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kBwdSmem);
  });
  if (e != cudaSuccess) return e;
  tc_bwd_kernel<kTop, kFirst><<<grid, kThreadsB, kBwdSmem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t tc_layer_bwd(const TcBwdParams& p, int* grid_used, cudaStream_t st) {
  const int n = p.term[0].n_tiles + p.term[1].n_tiles;
  const int grid = n > 0 ? grid_for(n) : 0;
  if (grid_used) *grid_used = grid;
  if (grid == 0) return cudaSuccess;
  if (p.top && p.first) return cudaErrorInvalidValue;  // one hidden layer: the first layer runs on its own
  if (p.top) return launch_bwd<true, false>(p, grid, st);
  if (p.first) return launch_bwd<false, true>(p, grid, st);
  return launch_bwd<false, false>(p, grid, st);
}

cudaError_t tc_colsum(const float* part, int nblk, int stride, int n, float* out, int accumulate, cudaStream_t st) {
  tc_colsum_kernel<<<(n + 31) / 32, 256, 0, st>>>(part, nblk, stride, n, out, accumulate);
  return cudaGetLastError();
}

cudaError_t tc_colsum_tall(const float* part, int nrows, int stride, int ncols, float* scratch, int scratch_floats,
                           float* out, int accumulate, cudaStream_t st) {
  int groups = (nrows + 255) / 256;
  if (groups > 64) groups = 64;
  if (groups < 1) groups = 1;
  if ((size_t)groups * ncols > (size_t)scratch_floats) return cudaErrorInvalidValue;
  const int rpc = (nrows + groups - 1) / groups;
  tc_colsum_stage1_kernel<<<dim3((ncols + 31) / 32, groups), 256, 0, st>>>(part, nrows, stride, ncols, rpc, scratch);
  tc_colsum_kernel<<<(ncols + 31) / 32, 256, 0, st>>>(scratch, groups, ncols, ncols, out, accumulate);
  return cudaGetLastError();
}

cudaError_t tc_colsum_layers(const float* part, int n_layers, size_t layer_stride, int nrows, int ncols, float* out,
                             const long long* out_off, cudaStream_t st) {
  if (n_layers < 1 || n_layers > kTcMaxLayers) return cudaErrorInvalidValue;
  TcLayerOffsets o{};
  for (int l = 0; l < n_layers; ++l) o.off[l] = out_off[l];
  tc_colsum_layers_kernel<<<dim3((ncols + 31) / 32, n_layers), 256, 0, st>>>(part, layer_stride, nrows, ncols, out, o);
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
