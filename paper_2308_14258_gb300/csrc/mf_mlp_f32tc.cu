// K3t: the FP32 SDNet on the 5th-generation tensor cores, fused with the scatter.
//
// The same contract as the FP32 SIMT kernel (mf_mlp_fp32.cu): every row r = (subdomain,
// interior point) of a colour goes through the input-split first layer (Eq. 8), the
// hidden tanh layers and the linear output, and the prediction is written to its grid
// point. The tolerance is that of an FP32 evaluation (1e-5 per sweep against the FP64
// oracle), so the hidden-layer products cannot run in one 16-bit pass. Each is split in
// three F16 products with FP32 accumulation in tensor memory:
//     W h ~ W_hi h_hi + W_hi h_lo + W_lo h_hi,
// where x_hi = f16(x) and x_lo = f16(x - x_hi) (round to nearest even). The dropped
// term W_lo h_lo and the rounding of the low parts are about 2^-22 of |W h| per
// product, against 2^-24 for an FP32 product.
//
// Orientation (as in the training kernels): a layer computes Z^T = W H^T with M = 128
// output features in the TMEM lanes and N = 64 rows of a tile in the columns, so an
// epilogue thread owns one feature j for 32 rows: its bias is one register, and its 32
// new activations are contiguous along the rows of the next layer's B operand (MN-major,
// 128-byte swizzle: feature j owns 128 bytes of 64 rows, 16-byte chunk c at c ^ (j mod 8),
// 8-feature groups 1 KB apart), written with 16-byte stores.
// tanh(z) = 1 - 2 / (1 + e) with e = exp(2 z) (hardware base-2 exponential and
// reciprocal; e overflows to infinity or flushes to zero at the ends): absolute error
// about 1e-7, enough for FP32 accuracy of what follows. The epilogue arithmetic uses
// the packed FP32 operations, two rows per instruction.
// The output layer u = w_out . h + b_out is a sum over features, i.e. over the lanes of
// four warps: each warp reduces its 32 features x 32 rows by a shuffle reduce-scatter
// (lane l ends with row l's sum), and the four quadrant sums are added in a fixed order.
//
// Persistent CTA per SM, 18 warps:
//   warps 0-15  epilogue: warp w serves tile slot w/8, TMEM lane quadrant (features)
//               32 (w mod 4).., rows 32 ((w/4) mod 2).. of the slot's 64-row tile
//   warps 16-17 lane 0 issues the MMAs of slot w-16; warp 16 also allocates TMEM and
//               loads the shared-memory weight images
// Weights: hidden layers 1..3 in TMEM as A operands (hi and lo images, 64 columns each),
// layers 4..5 in shared memory (K-major, 128-byte swizzle). TMEM: two 64-column FP32
// accumulators (one per slot) + six weight images = 512 columns. Shared memory: two
// weight layers (128 KB) + two slots x (hi, lo) activation tiles (64 KB) + output sums.
// The accumulator of a slot is single-buffered: an epilogue warp loads its part of the
// accumulator before it signals its share of the next activations, and the next layer's
// MMAs wait for all eight warps' signals.
//
// Every wait is bounded (mf_wait.cuh). After an abort the epilogue warps keep stepping
// through their tiles without work, so that every named barrier is reached by every warp.
#include <cuda_fp16.h>
#include <stdint.h>

#include "mf_internal.cuh"
#include "mf_tc.cuh"
#include "mf_wait.cuh"

namespace mf {

namespace {

constexpr int kH = 128;
constexpr int kNR = 64;                          // rows per tile (N of every MMA)
constexpr int kMaxHid = 5;
constexpr int kTmemLayers = 3;                   // hidden layers with their weights in TMEM
constexpr int kTSlots = 2;
constexpr int kEpiW = 16;
constexpr int kThreadsT = (kEpiW + 2) * 32;
constexpr uint32_t kImg = kH * kH * 2;           // one F16 128 x 128 image
constexpr uint32_t kXT = kNR * kH * 2;           // one F16 activation tile (64 rows x 128 features)
constexpr uint32_t kRedBytes = kTSlots * 2 * 4 * kNR * 4;  // [slot][tile parity][quadrant][row] floats
constexpr uint32_t kBarBytesT = 128;
// kind::f16, F16 A (K-major) and F16 B (MN-major), FP32 accumulator, M = 128, N = 64
constexpr uint32_t kIdescT = (1u << 4) | (1u << 16) | ((uint32_t)(kNR >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__host__ __device__ constexpr int smem_layers(int nh) { return nh > kTmemLayers ? nh - kTmemLayers : 0; }
__host__ __device__ constexpr size_t f32tc_smem(int nh) {
  return 1024 + (size_t)smem_layers(nh) * 2 * kImg + (size_t)kTSlots * 2 * kXT + kRedBytes + kBarBytesT;
}

struct F32tcParams {
  const float* B;        // [n_c][128] first-layer boundary term (b0 included)
  float* u;              // grid
  const uint8_t* wimg;   // [n_hidden][hi, lo] F16 images, K-major 128-byte swizzle
  int* status;
  ColourGeom g;
  int n_rows, n_tiles, additive;
  float bout;
  float bias[kMaxHid][kH];
  float wout[kH];
  float w2[kH][2];
};

__device__ __forceinline__ float ex2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// tanh(z) = 1 - 2 / (1 + e), e = 2^(2 z / ln 2) = exp(2 z): e overflows to +inf for large
// z (then 1 - 2 / inf = 1) and flushes to 0 for very negative z (then -1); about 1e-7
// absolute error, from the rounding of 1 - 2 r. (Measured: the hardware reciprocal beats
// two Newton steps on the FMA pipe here.)
constexpr float kTwoLog2e = 2.8853900817779268f;  // 2 / ln 2
__device__ __forceinline__ float tanh_acc(float z) {
  const float e = ex2_fast(kTwoLog2e * z);
  return fmaf(-2.0f, rcp_fast(1.0f + e), 1.0f);
}
template <int ACT>
__device__ __forceinline__ float first_act(float z) {
  if constexpr (ACT == kActGelu) return act_exact<kActGelu>(z);
  else return tanh_acc(z);
}
// (hi, lo) F16 pairs of two FP32 values: hi = f16(a), lo = f16(a - hi), packed with the
// first value in the low half
__device__ __forceinline__ void split2(float a0, float a1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a0, a1);
  // a - f32(hi) for both values in one packed FMA (exact: the difference is representable)
  const float2 r = __ffma2_rn(__half22float2(h), make_float2(-1.0f, -1.0f), make_float2(a0, a1));
  const __half2 l = __floats2half2_rn(r.x, r.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Byte offset of the chunk holding rows 8c..8c+7 of feature j in an activation tile.
__device__ __forceinline__ uint32_t xchunk(int j, int c) {
  return (uint32_t)(j >> 3) * 1024u + (uint32_t)(j & 7) * 128u + ((uint32_t)((c ^ j) & 7) << 4);
}
// K step ks (features 16 ks .. 16 ks + 15) of an activation tile as an MN-major operand:
// one 64-row atom along N (so the leading byte offset, the distance to a second atom, is
// not used; it is set to 1 KB, which keeps any address it could form inside this CTA's
// shared memory); 8-feature groups 1 KB apart.
__device__ __forceinline__ uint64_t xdesc(uint32_t tile, int ks) {
  return desc_sw128_mn(tile + (uint32_t)ks * 2048u, 1024u, 1024u);
}

// Columns [16 cq, 16 cq + 16) of this warp's 32 TMEM lanes <- K elements [32 cq, 32 cq + 32)
// of rows 32 q .. 32 q + 31 of a 128 x 128 F16 image (K-major, 128-byte swizzle, global).
__device__ __forceinline__ void image_to_tmem(const uint8_t* __restrict__ img, uint32_t tcol, int q, int lane, int cq) {
  const int row = 32 * q + lane;
  uint32_t v[16];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int chunk = (cq & 1) * 4 + c;
    const uint4 w = *reinterpret_cast<const uint4*>(img + (size_t)(cq >> 1) * (kH * 128) + (size_t)row * 128 +
                                                    ((uint32_t)(chunk ^ (row & 7)) << 4));
    v[4 * c] = w.x; v[4 * c + 1] = w.y; v[4 * c + 2] = w.z; v[4 * c + 3] = w.w;
  }
  tmem_st16(tcol + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * cq), v);
}

__device__ __forceinline__ int t_tile(int round, int slot) {
  return (round * (int)gridDim.x + (int)blockIdx.x) * kTSlots + slot;
}

// ACT: kActTanh, or kActGelu (the exact x Phi(x) with CUDA's erff, as the SIMT kernel).
template <int NH, int ACT>
__global__ void __launch_bounds__(kThreadsT, 1) mlp_f32tc_kernel(const __grid_constant__ F32tcParams P) {
  constexpr int kSL = smem_layers(NH);
  constexpr int kTL = NH < kTmemLayers ? NH : kTmemLayers;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen = smem_raw + (base - raw);
  const uint32_t sW = base;                                   // kSL layers x (hi, lo)
  const uint32_t sX = sW + (uint32_t)kSL * 2 * kImg;          // [slot][hi, lo] tiles
  const uint32_t offRed = (uint32_t)kSL * 2 * kImg + kTSlots * 2 * kXT;
  float* red = reinterpret_cast<float*>(gen + offRed);         // [slot][parity][quadrant][row]
  const uint32_t sBar = sX + kTSlots * 2 * kXT + kRedBytes;
  // barriers: 0 shared-memory weights loaded; 1 + s: slot s's activations written (8
  // warps); 3 + s: slot s's accumulator ready; 5 + s: MMA drain of slot s's issuer;
  // 7 + s: slot s may run its next epilogue phase (8 arrivals of the other slot)
  auto bar = [&](int i) { return sBar + 8u * (uint32_t)i; };
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gen + offRed + kRedBytes + 96);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gen + offRed + kRedBytes + 104);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(bar(0), 1);
    for (int i = 1; i <= 2; ++i) mbar_init(bar(i), 8);
    for (int i = 3; i <= 6; ++i) mbar_init(bar(i), 1);
    for (int i = 7; i <= 8; ++i) mbar_init(bar(i), 8);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == kEpiW) {
    tmem_alloc(smem_addr(tmem_holder), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const uint32_t tW = tmem + 128;  // TMEM weight images: layer l hi at tW + 128 l, lo at + 64

  // TMEM weights: the 16 epilogue warps store the images of layers 1..kTL (4 warps per
  // lane quadrant, each a quarter of the 16-column groups)
  if (warp < kEpiW) {
    const int q = warp & 3, part = warp >> 2;  // part 0..3
    for (int idx = part; idx < kTL * 2 * 4; idx += 4) {
      const int img = idx >> 2, cq = idx & 3;   // image (layer, hi/lo), column group of 16
      const uint8_t* src = P.wimg + (size_t)img * kImg;
      image_to_tmem(src, tW + (uint32_t)(img * 64), q, lane, cq);
    }
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp >= kEpiW) {
    if (lane == 0) {
      const int s = warp - kEpiW;
      bool ok = true;
      if (kSL > 0) {
        if (s == 0) {
          mbar_arrive_expect_tx(bar(0), (uint32_t)kSL * 2 * kImg);
#pragma unroll
          for (int i = 0; i < kSL * 2; ++i)
            bulk_g2s(sW + (uint32_t)i * kImg, P.wimg + (size_t)(kTL * 2 + i) * kImg, kImg, bar(0));
        }
        ok = wait_bounded(bar(0), 0, abort_flag, P.status, true);
      }
      const uint32_t acc = tmem + (uint32_t)(s * kNR);
      const uint32_t xh = sX + (uint32_t)s * 2 * kXT, xl = xh + kXT;
      const uint64_t dxh = xdesc(xh, 0), dxl = xdesc(xl, 0);  // K step ks: + 2048 ks bytes
      uint32_t ph = 0u;
      for (int k = 0; ok && t_tile(k, s) < P.n_tiles; ++k) {
#pragma unroll 1
        for (int m = 1; m <= NH; ++m) {
          ok = wait_spin(bar(1 + s), ph, abort_flag, P.status);
          if (!ok) break;
          ph ^= 1u;
          tc_fence_after();
          if (m <= kTmemLayers) {
            const uint32_t ah = tW + (uint32_t)((m - 1) * 128), al = ah + 64;
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks) {
              if (ks == 0) mma_ts<0>(acc, ah, dxh, kIdescT);
              else mma_ts<1>(acc, ah + (uint32_t)(8 * ks), desc_add(dxh, 2048u * ks), kIdescT);
            }
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks)
              mma_ts<1>(acc, ah + (uint32_t)(8 * ks), desc_add(dxl, 2048u * ks), kIdescT);
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks)
              mma_ts<1>(acc, al + (uint32_t)(8 * ks), desc_add(dxh, 2048u * ks), kIdescT);
          } else {
            const uint32_t wh = sW + (uint32_t)((m - 1 - kTmemLayers) * 2) * kImg, wl = wh + kImg;
            const uint64_t dh = desc_sw128(wh), dl = desc_sw128(wl);
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks) {
              if (ks == 0) mma_ss<0>(acc, dh, dxh, kIdescT);
              else mma_ss<1>(acc, desc_add(dh, kstep_off(kH, ks)), desc_add(dxh, 2048u * ks), kIdescT);
            }
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks)
              mma_ss<1>(acc, desc_add(dh, kstep_off(kH, ks)), desc_add(dxl, 2048u * ks), kIdescT);
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks)
              mma_ss<1>(acc, desc_add(dl, kstep_off(kH, ks)), desc_add(dxh, 2048u * ks), kIdescT);
          }
          mma_commit(bar(3 + s));
        }
      }
      mma_commit(bar(5 + s));
      wait_bounded(bar(5 + s), 0, abort_flag, P.status, false);
    }
    __syncwarp();
  } else {
    const int s = warp >> 3, q = warp & 3, hh = (warp >> 2) & 1;
    const int j = 32 * q + lane;          // this thread's feature
    const uint32_t xh = sX + (uint32_t)s * 2 * kXT, xl = xh + kXT;
    const uint32_t tacc = tmem + (uint32_t)(s * kNR + 32 * hh) + ((uint32_t)(32 * q) << 16);
    const float w2x = P.w2[j][0], w2y = P.w2[j][1], wo = P.wout[j];
    const int named = 1 + 2 * s + hh;     // the four quadrant warps of these 32 rows
    uint32_t acc_ph = 0u, tok_ph = 0u;
    bool ok = true;

    // The slots take turns on the epilogue: phase n of slot 1 runs after phase n of slot
    // 0, and phase n of slot 0 after phase n - 1 of slot 1 (phase 0 after slot 1's last
    // phase of the previous tile), so that one slot's MMAs run while the other's
    // epilogue works (left alone the slots fall into step and wait for their MMAs
    // together). The turn passes when a phase's activations are computed, before they
    // are stored; the waiting slot sleeps between polls.
    auto take_turn = [&](int k, int e) {
      const bool need = (s == 1) || (e > 0 ? t_tile(k, 1) < P.n_tiles : (k > 0 && t_tile(k - 1, 1) < P.n_tiles));
      if (!need) return;
      if (ok) ok = __all_sync(0xffffffffu, wait_nap_inl(bar(7 + s), tok_ph, abort_flag, P.status));
      tok_ph ^= 1u;
    };
    auto give_turn = [&]() {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(8 - s));
    };

    // 32 activations of this feature (rows 32 hh .. + 31) -> hi and lo tiles, then signal
    auto put = [&](const float (&a)[32]) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) split2(a[8 * c + 2 * i], a[8 * c + 2 * i + 1], hi[i], lo[i]);
        const uint32_t off = xchunk(j, 4 * hh + c);
        st_shared_v4(xh + off, hi[0], hi[1], hi[2], hi[3]);
        st_shared_v4(xl + off, lo[0], lo[1], lo[2], lo[3]);
      }
      fence_proxy_async_smem();
      tc_fence_before();  // this warp's accumulator loads are ordered before the signal
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(1 + s));
    };

    for (int k = 0; t_tile(k, s) < P.n_tiles; ++k) {
      const int row0 = t_tile(k, s) * kNR + 32 * hh;
      // phase 0: first layer (Eq. 8) in FP32, B[s] + W2 x for each of the 32 rows
      take_turn(k, 0);
      if (ok) {
        // rows step through the points of a subdomain (one division per 32 rows); rows
        // past the last are computed on the last subdomain and never written
        float a[32];
        const int rps = P.g.rows_per_sub, last = P.g.n_c - 1;
        int sc = row0 / rps, pt = row0 - sc * rps;
        float b_cur = __ldg(P.B + (size_t)(sc < last ? sc : last) * kH + j);
        if (P.g.centre) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int qq = pt - kNi;
            const int px = pt < kNi ? pt : kNi / 2;
            const int py = pt < kNi ? kNi / 2 : (qq < kNi / 2 ? qq : qq + 1);
            const float x = (float)(px + 1) * (1.0f / kPts), y = (float)(py + 1) * (1.0f / kPts);
            a[i] = first_act<ACT>(fmaf(w2y, y, fmaf(w2x, x, b_cur)));
            if (++pt == rps) {
              pt = 0;
              ++sc;
              b_cur = __ldg(P.B + (size_t)(sc < last ? sc : last) * kH + j);
            }
          }
        } else {
          // full interior: x and y step by 1/32 (exact in FP32), no integer conversions
          int px = pt % kNi;
          float x = (float)(px + 1) * (1.0f / kPts), y = (float)(pt / kNi + 1) * (1.0f / kPts);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            a[i] = first_act<ACT>(fmaf(w2y, y, fmaf(w2x, x, b_cur)));
            x += 1.0f / kPts;
            if (++px == kNi) {
              px = 0;
              x = 1.0f / kPts;
              y += 1.0f / kPts;
            }
            if (++pt == rps) {
              pt = 0;
              ++sc;
              y = 1.0f / kPts;
              b_cur = __ldg(P.B + (size_t)(sc < last ? sc : last) * kH + j);
            }
          }
        }
        give_turn();
        put(a);
      } else {
        give_turn();
      }
      // hidden layers
      float usum[32];
#pragma unroll 1
      for (int m = 1; m <= NH; ++m) {
        if (ok) ok = __all_sync(0xffffffffu, wait_nap_inl(bar(3 + s), acc_ph, abort_flag, P.status));
        acc_ph ^= 1u;
        take_turn(k, m);
        if (!ok) {
          give_turn();
          continue;
        }
        tc_fence_after();
        uint32_t v[32];
        tmem_ld16(tacc, v);
        tmem_ld16(tacc + 16u, v + 16);
        tmem_wait_ld();
        float a[32];
        if constexpr (ACT == kActGelu) {
#pragma unroll
          for (int i = 0; i < 32; ++i) a[i] = act_exact<kActGelu>(__uint_as_float(v[i]) + P.bias[m - 1][j]);
        } else {
        // t = (v + b) 2 / ln 2 for two rows per packed FMA
        const float2 k2 = make_float2(kTwoLog2e, kTwoLog2e);
        const float bk = P.bias[m - 1][j] * kTwoLog2e;
        const float2 bk2 = make_float2(bk, bk);
        // the 32 values in stages (all exponentials, then all reciprocals), so that the
        // transcendental unit's latency is covered by independent work of this thread
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          float2 d[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float2 t = __ffma2_rn(make_float2(__uint_as_float(v[16 * h2 + 2 * i]), __uint_as_float(v[16 * h2 + 2 * i + 1])),
                                        k2, bk2);
            d[i] = __fadd2_rn(make_float2(ex2_fast(t.x), ex2_fast(t.y)), make_float2(1.0f, 1.0f));
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float2 r = __ffma2_rn(make_float2(rcp_fast(d[i].x), rcp_fast(d[i].y)), make_float2(-2.0f, -2.0f),
                                        make_float2(1.0f, 1.0f));
            a[16 * h2 + 2 * i] = r.x;
            a[16 * h2 + 2 * i + 1] = r.y;
          }
        }
        }
        if (m < NH) {
          give_turn();
          put(a);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) usum[i] = wo * a[i];
          give_turn();
        }
      }
      // output: reduce-scatter over the warp's 32 features (lane l keeps row l), then
      // the four quadrant warps' sums in order
      float* rbuf = red + (size_t)((s * 2 + (k & 1)) * 4) * kNR;  // [quadrant][row]
      if (ok) {
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1) {
          const bool upper = (lane & w) != 0;
#pragma unroll
          for (int i = 0; i < w; ++i) {
            // keep rows i + w (upper lanes) or i (lower lanes) of the current 2w
            const float send = upper ? usum[i] : usum[i + w];
            const float keep = upper ? usum[i + w] : usum[i];
            usum[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
          }
        }
        rbuf[q * kNR + 32 * hh + lane] = usum[0];
      }
      named_barrier_sync(named, 128);
      if (ok && q == 0) {
        const int row = row0 + lane;
        if (row < P.n_rows) {
          const float val = ((rbuf[32 * hh + lane] + rbuf[kNR + 32 * hh + lane]) +
                             (rbuf[2 * kNR + 32 * hh + lane] + rbuf[3 * kNR + 32 * hh + lane])) + P.bout;
          const RowSite site = row_site(P.g, row);
          if (P.additive)
            P.u[site.idx] += cover_weight(P.g, site.ix, site.iy) * val;
          else
            P.u[site.idx] = val;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kEpiW) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

template <int NH, int ACT>
cudaError_t launch_nh(const F32tcParams& p, cudaStream_t st) {
  static PerDevice pd;
  int grid_cap = 0;
  cudaError_t e = per_device(pd, [](int dev, int* cap, size_t*) {
    cudaError_t e1 = cudaFuncSetAttribute(mlp_f32tc_kernel<NH, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)f32tc_smem(NH));
    if (e1 != cudaSuccess) return e1;
    int sms = 0, per_sm = 0;
    e1 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e1 != cudaSuccess) return e1;
    e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_f32tc_kernel<NH, ACT>, kThreadsT, f32tc_smem(NH));
    if (e1 != cudaSuccess) return e1;
    // a CTA takes all 512 TMEM columns: one resident CTA per SM
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *cap = sms;
    return cudaSuccess;
  }, &grid_cap);
  if (e != cudaSuccess) return e;
  int grid = (p.n_tiles + kTSlots - 1) / kTSlots;
  if (grid > grid_cap) grid = grid_cap;
  if (grid < 1) return cudaSuccess;
  // shared memory above what one CTA needs keeps a second CTA (which would wait for TMEM)
  // off the SM
  int smem_sm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  size_t smem = f32tc_smem(NH);
  if (smem * 2 <= (size_t)smem_sm) {
    smem = (size_t)smem_sm / 2 + 1024;
    static PerDevice pd2;
    e = per_device(pd2, [smem](int, int*, size_t*) {
      return cudaFuncSetAttribute(mlp_f32tc_kernel<NH, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
  }
  mlp_f32tc_kernel<NH, ACT><<<grid, kThreadsT, smem, st>>>(p);
  return cudaGetLastError();
}

// F16 hi/lo images of the hidden weights: W[n][k] (FP32, row n = output unit) ->
// hi = f16(W), lo = f16(W - hi), each in the K-major 128-byte-swizzled layout
// (64-element K blocks of 128 rows x 128 bytes, 16-byte chunk c of row n at c ^ (n mod 8)).
__global__ void pack_f16_split_kernel(const float* __restrict__ WhT, int n_hidden, uint16_t* __restrict__ img) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_hidden * kH * kH) return;
  const int l = idx / (kH * kH), r = idx % (kH * kH);
  const int k = r / kH, n = r % kH;  // WhT is k-major: [l][k][n]
  const float w = WhT[idx];
  const __half hi = __float2half_rn(w);
  const __half lo = __float2half_rn(w - __half2float(hi));
  const int kb = k / 64, wk = k % 64, chunk = wk / 8, e = wk % 8;
  const size_t off = (size_t)kb * kH * 64 + (size_t)n * 64 + (size_t)((chunk ^ (n & 7)) * 8) + e;
  img[(size_t)(2 * l) * kH * kH + off] = *reinterpret_cast<const uint16_t*>(&hi);
  img[(size_t)(2 * l + 1) * kH * kH + off] = *reinterpret_cast<const uint16_t*>(&lo);
}

}  // namespace

bool f32tc_supported(const DevNet& net) {
  return net.width == kH && net.n_hidden >= 1 && net.n_hidden <= kMaxHid && net.wimg_f16 != nullptr;
}

size_t f32tc_image_bytes(int n_hidden) { return (size_t)n_hidden * 2 * kImg; }

cudaError_t f32tc_pack(const float* WhT, int n_hidden, void* img, cudaStream_t st) {
  const int n = n_hidden * kH * kH;
  pack_f16_split_kernel<<<(n + 255) / 256, 256, 0, st>>>(WhT, n_hidden, static_cast<uint16_t*>(img));
  return cudaGetLastError();
}

cudaError_t launch_mlp_f32tc(const float* B, const ColourGeom& g, const DevNet& net, float* u, int additive,
                             int* dev_status, cudaStream_t st) {
  if (g.n_c <= 0) return cudaSuccess;
  if (!f32tc_supported(net)) return cudaErrorNotSupported;
  F32tcParams p{};
  p.B = B;
  p.u = u;
  p.wimg = static_cast<const uint8_t*>(net.wimg_f16);
  p.status = dev_status;
  p.g = g;
  p.n_rows = g.n_c * g.rows_per_sub;
  p.n_tiles = (p.n_rows + kNR - 1) / kNR;
  p.additive = additive;
  p.bout = net.bout;
  for (int l = 0; l < kMaxHid; ++l)
    for (int j = 0; j < kH; ++j) p.bias[l][j] = l < net.n_hidden ? net.h_bh[l * kH + j] : 0.f;
  for (int j = 0; j < kH; ++j) {
    p.wout[j] = net.h_wout[j];
    p.w2[j][0] = net.h_W2[2 * j];
    p.w2[j][1] = net.h_W2[2 * j + 1];
  }
  if (net.act == kActGelu) {
    switch (net.n_hidden) {
      case 1: return launch_nh<1, kActGelu>(p, st);
      case 2: return launch_nh<2, kActGelu>(p, st);
      case 3: return launch_nh<3, kActGelu>(p, st);
      case 4: return launch_nh<4, kActGelu>(p, st);
      default: return launch_nh<5, kActGelu>(p, st);
    }
  }
  switch (net.n_hidden) {
    case 1: return launch_nh<1, kActTanh>(p, st);
    case 2: return launch_nh<2, kActTanh>(p, st);
    case 3: return launch_nh<3, kActTanh>(p, st);
    case 4: return launch_nh<4, kActTanh>(p, st);
    default: return launch_nh<5, kActTanh>(p, st);
  }
}

}  // namespace mf
