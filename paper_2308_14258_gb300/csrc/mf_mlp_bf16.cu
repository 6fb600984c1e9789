// K3: BF16 (or F16) SDNet over one colour on the 5th-generation tensor cores, fused with
// the scatter into the grid. The two 16-bit types differ only in the operand type of the
// MMAs, the weight images and the activation's packed form (template DT).
//
// Work: rows r = (subdomain s, interior point p) of the colour, in tiles of 128 rows
// (the M of one tcgen05.mma). Per row, the input-split first layer (Eq. 8) is
// tanh(B[s] + W2 x_p) computed on the CUDA cores from K1's FP32 B table; the hidden
// H x H layers run as tcgen05.mma (kind::f16, BF16 operands, FP32 accumulators in
// tensor memory); each epilogue reads its accumulator tile with tcgen05.ld, adds the
// bias, applies tanh and writes the BF16 activations back to shared memory as the next
// layer's A operand; the last epilogue folds w_out . h + b_out in FP32 and writes the
// prediction to its grid point.
//
// Persistent CTA per SM, 18 warps:
//   warps 0-15  epilogue: warp w serves tile slot w/8, column member (w/4) mod 2 and TMEM
//               lanes / tile rows 32(w mod 4)..+31
//   warps 16-17 lane 0 issues the MMAs of slot w-16; warp 16 also allocates TMEM and
//               loads the weights (bulk async copy)
// Shared memory: all hidden weight matrices resident (n_hidden x H x H BF16) plus one
// 128 x H BF16 activation tile per slot, in the 128-byte-swizzled K-major layout the MMA
// descriptors name. TMEM: two H-column FP32 accumulators per slot.
//
// Every mbarrier wait is bounded (about one second of %globaltimer); a wait that gives
// up records kDevErrTimeout in the status word, raises a CTA-wide abort flag so the
// other roles stop too, and the MMA lane drains its in-flight MMAs (bounded) before the
// CTA frees its tensor memory and exits.
#include <stdint.h>

#include "mf_internal.cuh"
#include "mf_tc.cuh"
#include "mf_wait.cuh"

namespace mf {

namespace {

constexpr int kMaxHidden = 5;
constexpr int kEpiWarps = 16;                     // 2 tile slots x 2 column halves x 4 row quadrants
constexpr int kThreadsBf16 = (kEpiWarps + 2) * 32;  // + one MMA-issuing warp per slot

struct Bf16Params {
  const float* B;        // [n_c][H] first-layer boundary term
  float* u;              // grid
  const uint8_t* wimg;   // BF16 weight images
  int* status;           // device status word
  ColourGeom g;
  int n_rows, n_tiles, additive;
  float bout;
  float bias[kMaxHidden][128];  // hidden-layer biases
  float wout[128];
  float w2[128][2];             // coordinate block of the first layer
  // whole-sweep launch (multi-colour kernel only): colour passes in order, each with its
  // own geometry; the kernel forms B itself (boundary gather + W1 g + b0) before each
  // pass, and passes are separated by device-wide barriers on `sync`
  int n_col;
  ColourGeom gc[4];
  int n_rows_c[4], n_tiles_c[4];
  const float* W1t;      // [128][H] boundary block of the first layer, k-major
  const float* b0;       // [H]
  unsigned int* sync;    // barrier counter, zero at launch
};

// Activation of two FP32 pre-activations, packed as a 16-bit pair of the kernel's operand
// type DT (kDtBf16 or kDtF16). tanh: the hardware tanh on the packed pair. GELU: its tanh
// form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (Hendrycks and Gimpel) with the
// FP32 hardware tanh, so that 1 + tanh keeps its accuracy for negative x; both forms cost
// one tanh per element on the MUFU unit.
constexpr int kDtBf16 = 0, kDtF16 = 1;
template <int ACT, int DT>
__device__ __forceinline__ uint32_t act16x2(float a0, float a1) {
  if constexpr (ACT == kActTanh) {
    if constexpr (DT == kDtF16) return tanh_f16x2(pack_f16x2(a0, a1));
    else return tanh_bf16x2(pack_bf16x2(a0, a1));
  } else {
    constexpr float k0 = 0.7978845608028654f;  // sqrt(2 / pi)
    constexpr float k1 = k0 * 0.044715f;
    const float t0 = tanh_approx(a0 * fmaf(k1 * a0, a0, k0));
    const float t1 = tanh_approx(a1 * fmaf(k1 * a1, a1, k0));
    const float h0 = 0.5f * a0, h1 = 0.5f * a1;
    if constexpr (DT == kDtF16) return pack_f16x2(fmaf(h0, t0, h0), fmaf(h1, t1, h1));
    else return pack_bf16x2(fmaf(h0, t0, h0), fmaf(h1, t1, h1));
  }
}
template <int DT>
__device__ __forceinline__ float lo16(uint32_t v) {
  if constexpr (DT == kDtF16) return f16_lo(v);
  else return bf16_lo(v);
}
template <int DT>
__device__ __forceinline__ float hi16(uint32_t v) {
  if constexpr (DT == kDtF16) return f16_hi(v);
  else return bf16_hi(v);
}

// ---------------------------------------------------------------- kernel
//
// Scheduling. Two tiles are in flight per SM (slots 0 and 1), each with eight epilogue
// warps and one MMA-issuing thread. The epilogue (tanh on the MUFU unit) is the
// bottleneck and each tile's layers are strictly serial (MMA -> epilogue -> MMA), so
// the slots take turns: epilogue phase n of slot 1 starts after phase n of slot 0 is
// three quarters done, and phase n of slot 0 after three quarters of phase n-1 of slot 1
// (phase 0 = first layer, phase m = hidden layer m), handed over through two token
// mbarriers. While one slot's warps own the MUFU, the other slot's MMAs run; handing
// over before the end of a phase lets the next phase start while the last warps of the
// current one finish (measured: 0.93 ms per colour launch against 1.08 with the hand-over
// at the end, 0.94 at one half, 1.06 at one quarter). Left to themselves the slots fall
// into step (fair sharing lets a lagging slot catch up) and then both wait on their MMAs
// together.
// Within a phase each warp pair first writes K half 0, signals it, then K half 1, so the
// next layer's first MMAs start before the phase ends; accumulators are therefore
// double-buffered per slot in TMEM (layer parity picks the buffer). All waits on this
// path spin inline (wait_spin_inl): a suspended wait wakes hundreds of cycles late, and
// an out-of-line call costs about as much as the wait it makes on a phase that is
// already complete.

constexpr int kSlots = 2;

template <int H, int NH>
struct Bf16Cfg {
  static constexpr int kHH = H / 2;                                 // K half
  static constexpr int kCW = H / 4;                                 // columns per warp per K half
  static constexpr int kKStepsHalf = kHH / 16;                      // K=16 steps per K half
  static constexpr uint32_t kWBytes = (uint32_t)NH * H * H * 2;     // resident hidden weights
  static constexpr uint32_t kABytes = (uint32_t)kTileRows * H * 2;  // one activation tile
  static constexpr uint32_t kTmemCols = 4 * H;                      // 2 slots x 2 buffers x H
  static constexpr uint32_t kBarBytes = 128;
  static constexpr uint32_t kSumBytes = 2 * kTileRows * 4 + 64;     // output half-sums + pair flags
  static constexpr size_t kSmem = 1024 + kWBytes + 2 * kABytes + kBarBytes + kSumBytes;
  static constexpr uint32_t kIdesc = idesc_bf16(kTileRows, H);
  static_assert(kCW % 8 == 0 && kKStepsHalf >= 1, "half geometry");
};

__device__ __forceinline__ int slot_tile(const Bf16Params& P, int round, int slot) {
  return (round * (int)gridDim.x + (int)blockIdx.x) * kSlots + slot;
}

// MMA issue for one slot (a single thread): per tile and hidden layer m, the K steps of
// K half 0 once that half of the activations is written, then K half 1, then one commit.
constexpr bool kGeluInlineIssue = false;
constexpr bool kGeluInlineEpi = false;

// How the hand-off waits are compiled, per activation (measured): inline spins for tanh;
// for GELU, whose longer epilogue the inline spins slow down, the two constants above.
// The turn-token wait of the tanh epilogue sleeps 32 ns between polls (wait_nap_inl):
// the turn passes three quarters into a phase, so a late wake-up costs nothing, and the
// eight waiting warps stop taking issue slots from the eight working ones (measured
// 0.846 against 0.852 ms per launch; a suspending try_wait gave 0.867).
template <int ACT>
struct HotWaits {
  static constexpr bool kIssue = ACT == kActTanh ? true : kGeluInlineIssue;
  static constexpr bool kEpi = ACT == kActTanh ? true : kGeluInlineEpi;
};
template <bool kInline>
__device__ __forceinline__ bool hot_spin(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  if constexpr (kInline) return wait_spin_inl(bar, parity, abort_flag, status);
  else return wait_spin(bar, parity, abort_flag, status);
}
template <bool kInline>
__device__ __forceinline__ bool hot_wait_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  if constexpr (kInline) return wait_warp_inl(bar, parity, abort_flag, status);
  else return wait_warp(bar, parity, abort_flag, status);
}

template <int H, int NH, int ACT, int DT>
__device__ __forceinline__ bool mma_issuer(const Bf16Params& P, int n_tiles, int s, uint32_t tmem, uint32_t sA,
                                           uint32_t sW, uint32_t bar_act0, uint32_t bar_act1, uint32_t bar_acc,
                                           volatile int* abort_flag, uint32_t& ph0, uint32_t& ph1) {
  using C = Bf16Cfg<H, NH>;
  const uint32_t acc0 = tmem + (uint32_t)(s * 2 * H);
  bool ok = true;
  for (int k = 0; ok && slot_tile(P, k, s) < n_tiles; ++k) {
    // rebuilt every tile (an opaque copy of the base) so the compiler does not hoist all
    // NH x H/16 descriptors out of the loop into registers
    uint32_t a_base = sA + (uint32_t)s * C::kABytes, w_base = sW;
    asm volatile("" : "+r"(a_base), "+r"(w_base));
    const uint64_t a0 = desc_sw128(a_base);
    const uint64_t w0 = desc_sw128(w_base);
#pragma unroll
    for (int m = 1; m <= NH; ++m) {
      const uint32_t acc = acc0 + (uint32_t)((m & 1) * H);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        ok = hot_spin<HotWaits<ACT>::kIssue>(h == 0 ? bar_act0 : bar_act1, h == 0 ? ph0 : ph1, abort_flag, P.status);
        if (!ok) break;
        if (h == 0) ph0 ^= 1u; else ph1 ^= 1u;
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < C::kKStepsHalf; ++kk) {
          const int ks = h * C::kKStepsHalf + kk;
          const uint64_t ad = desc_add(a0, kstep_off(kTileRows, ks));
          const uint64_t bd = desc_add(w0, (uint32_t)(m - 1) * H * H * 2 + kstep_off(H, ks));
          constexpr uint32_t kId = DT == kDtF16 ? idesc_f16(kTileRows, H) : C::kIdesc;
          if (ks == 0) mma_ss<0>(acc, ad, bd, kId);
          else mma_ss<1>(acc, ad, bd, kId);
        }
      }
      if (!ok) break;
      mma_commit(bar_acc);
    }
  }
  return ok;
}

// Epilogue of one warp: slot s, row quadrant q (TMEM lanes / tile rows 32q..32q+31),
// member JJ of the column pair (in K half h it owns columns h*H/2 + JJ*H/4 .. + H/4 - 1).
template <int H, int NH, int JJ, int ACT, bool kMulti, int DT>
__device__ __forceinline__ bool epilogue(const Bf16Params& P, const ColourGeom& geo, int n_rows, int n_tiles, int s,
                                         int q, int lane, uint32_t tmem, uint32_t sA, uint32_t bar_act0,
                                         uint32_t bar_act1, uint32_t bar_acc, uint32_t tok_wait, uint32_t tok_give,
                                         float* half_sum, volatile int* pair_ok, volatile int* abort_flag,
                                         uint32_t& acc_ph, uint32_t& tok_ph) {
  using C = Bf16Cfg<H, NH>;
  constexpr int HH = C::kHH, CW = C::kCW;
  const int rloc = 32 * q + lane;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const uint32_t a_row = sA + (uint32_t)s * C::kABytes + (uint32_t)rloc * 128u;
  const uint32_t swz = (uint32_t)(rloc & 7) << 4;
  const int named = 1 + s * 4 + q;  // named barrier of the warp pair of these rows
  bool ok = true;

  auto put = [&](int c0, const uint32_t* pk) {  // CW columns from c0 of this row
#pragma unroll
    for (int i = 0; i < CW / 8; ++i) {
      const int ch = c0 / 8 + i;  // 16-byte chunk along K
      const uint32_t addr = a_row + (uint32_t)(ch >> 3) * (kTileRows * 128u) + (((uint32_t)(ch & 7) << 4) ^ swz);
      st_shared_v4(addr, pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
    }
  };
  auto signal = [&](uint32_t b) {  // this warp's share of a K half is written
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(b);
  };
  // the other slot's turn: given three quarters into each phase (a quarter into the
  // second K half; see the scheduling note above)
  auto give_turn = [&]() {
    __syncwarp();
    if (lane == 0) mbar_arrive(tok_give);
  };
  // wait for the other slot's turn to end: slot 1 phase n needs slot 0 phase n; slot 0
  // phase n needs slot 1 phase n-1 when that phase exists
  auto take_turn = [&](int k, int e) -> bool {
    const bool need = (s == 1) || (e > 0 ? slot_tile(P, k, 1) < n_tiles
                                         : (k > 0 && slot_tile(P, k - 1, 1) < n_tiles));
    if (!need) return true;
    bool r;
    if constexpr (ACT == kActTanh) r = __all_sync(0xffffffffu, wait_nap_inl(tok_wait, tok_ph, abort_flag, P.status));
    else r = hot_wait_warp<HotWaits<ACT>::kEpi>(tok_wait, tok_ph, abort_flag, P.status);
    tok_ph ^= 1u;
    return r;
  };

  for (int k = 0; ok; ++k) {
    const int tile = slot_tile(P, k, s);
    if (tile >= n_tiles) break;
    const int row = tile * kTileRows + rloc;
    const bool valid = row < n_rows;
    const RowSite site = row_site(geo, valid ? row : n_rows - 1);
    const float x = (float)(site.px + 1) * (1.0f / kPts), y = (float)(site.py + 1) * (1.0f / kPts);
    const float* Bs = P.B + (size_t)site.s * H;

    // phase 0: first layer (Eq. 8), FP32 sum B[s] + W2 x, rounded to BF16, tanh
    {
      // B is read through L2 only when this launch wrote it (whole-sweep kernel): the
      // read-only path may hold lines from before the write
      auto ldb = [](const float* a) {
        if constexpr (kMulti) return __ldcg(reinterpret_cast<const float2*>(a));
        else return __ldg(reinterpret_cast<const float2*>(a));
      };
      float2 bb[CW / 2];  // half 0 is loaded before the turn is taken, overlapping the wait
#pragma unroll
      for (int i = 0; i < CW / 2; ++i) bb[i] = ldb(Bs + JJ * CW + 2 * i);
      ok = take_turn(k, 0);
      if (ok) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c0 = h * HH + JJ * CW;
          if (h == 1) {
#pragma unroll
            for (int i = 0; i < CW / 2; ++i) bb[i] = ldb(Bs + c0 + 2 * i);
          }
          uint32_t pk[CW / 2];
#pragma unroll
          for (int i = 0; i < CW / 2; ++i) {
            if (h == 1 && i == CW / 4) give_turn();
            const int col = c0 + 2 * i;
            const float a0 = fmaf(P.w2[col][1], y, fmaf(P.w2[col][0], x, bb[i].x));
            const float a1 = fmaf(P.w2[col + 1][1], y, fmaf(P.w2[col + 1][0], x, bb[i].y));
            pk[i] = act16x2<ACT, DT>(a0, a1);
          }
          put(c0, pk);
          signal(h == 0 ? bar_act0 : bar_act1);
        }
      }
    }

    float uacc = 0.f;
#pragma unroll
    for (int m = 1; m <= NH; ++m) {
      if (!ok) break;
      ok = hot_wait_warp<HotWaits<ACT>::kEpi>(bar_acc, acc_ph, abort_flag, P.status);
      if (!ok) break;
      acc_ph ^= 1u;
      ok = take_turn(k, m);
      if (!ok) break;
      tc_fence_after();
      const uint32_t t_buf = tmem + (uint32_t)(s * 2 * H + (m & 1) * H) + lane_off;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c0 = h * HH + JJ * CW;
        uint32_t v[CW];
        if constexpr (CW == 32) tmem_ld32(t_buf + (uint32_t)c0, *reinterpret_cast<uint32_t(*)[32]>(v));
        else tmem_ld16(t_buf + (uint32_t)c0, v);
        tmem_wait_ld();
        uint32_t pk[CW / 2];
#pragma unroll
        for (int i = 0; i < CW / 2; ++i) {
          if (h == 1 && i == CW / 4) give_turn();
          const float a0 = __uint_as_float(v[2 * i]) + P.bias[m - 1][c0 + 2 * i];
          const float a1 = __uint_as_float(v[2 * i + 1]) + P.bias[m - 1][c0 + 2 * i + 1];
          pk[i] = act16x2<ACT, DT>(a0, a1);
        }
        if (h == 1) tc_fence_before();
        if (m < NH) {
          put(c0, pk);
          signal(h == 0 ? bar_act0 : bar_act1);
        } else {
#pragma unroll
          for (int i = 0; i < CW / 2; ++i) {
            uacc = fmaf(lo16<DT>(pk[i]), P.wout[c0 + 2 * i], uacc);
            uacc = fmaf(hi16<DT>(pk[i]), P.wout[c0 + 2 * i + 1], uacc);
          }
        }
      }
    }
    // output: partner warps combine their partial sums; the continue decision is taken
    // jointly so that neither warp of the pair can leave while the other waits
    if (JJ == 1) half_sum[s * kTileRows + rloc] = uacc;
    const bool ok_warp = __all_sync(0xffffffffu, ok);
    if (lane == 0) pair_ok[(s * 4 + q) * 2 + JJ] = ok_warp ? 1 : 0;
    named_barrier_sync(named, 64);
    ok = pair_ok[(s * 4 + q) * 2 + 0] && pair_ok[(s * 4 + q) * 2 + 1];
    if (JJ == 0 && ok && valid) {
      const float val = uacc + half_sum[s * kTileRows + rloc] + P.bout;
      if (P.additive)
        P.u[site.idx] += cover_weight(geo, site.ix, site.iy) * val;
      else
        P.u[site.idx] = val;
    }
    named_barrier_sync(named, 64);
  }
  return ok;
}

// ---------------------------------------------------------------- whole-sweep launch
//
// The multi-colour kernel runs a whole multiplicative sweep in one cooperative launch:
// for each colour pass it forms the first-layer boundary term B itself (the boundary
// gather of K1 and B[s] = W1 g_s + b0, W1 staged in the activation-tile area, which is
// free between passes), waits at a device-wide barrier until every CTA has written its
// part of B, runs the colour's tiles exactly as the single-colour kernel does, and
// waits at a second barrier until every prediction of the colour is in the grid before
// the next pass gathers. Only the 16 epilogue warps take part in the barriers; the MMA
// issuers simply wait for the next pass's activations. Every wait is bounded.

constexpr int kEpiAllBar = 9;  // named barrier of all epilogue warps (ids 1..8 pair the warps)

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned int* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Device-wide barrier of the epilogue warps: true when every CTA has arrived `target`
// times in all; false (the same answer in every warp of the CTA) once the CTA aborts or
// the bounded wait gives up.
__device__ __forceinline__ bool epi_grid_sync(const Bf16Params& P, unsigned target, volatile int* abort_flag,
                                              volatile int* go) {
  named_barrier_sync(kEpiAllBar, kEpiWarps * 32);
  if (threadIdx.x == 0) {
    bool ok = *abort_flag == 0;
    if (ok) {
      __threadfence();
      atomicAdd(P.sync, 1u);
      const unsigned long long t0 = globaltimer();
      while (ld_acquire_gpu(P.sync) < target) {
        if (*abort_flag) {
          ok = false;
          break;
        }
        if (globaltimer() - t0 > kWaitLimitNs) {
          *abort_flag = 1;
          atomicExch(P.status, kDevErrTimeout);
          ok = false;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    *go = ok ? 1 : 0;
  }
  named_barrier_sync(kEpiAllBar, kEpiWarps * 32);
  return *go != 0;
}

// K1 inside the whole-sweep kernel: B[s][:] = W1 g_s + b0 for the colour's subdomains,
// one warp per subdomain (subdomains dealt to the CTAs' warps round robin). Lane l holds
// boundary values l, 32 + l, 64 + l, 96 + l (the CCW order of K1) and H/32 consecutive
// outputs; W1 (k-major, [128][H] FP32) is read from its staged copy in shared memory.
template <int H>
__device__ __forceinline__ void gather_pass(const Bf16Params& P, const ColourGeom& geo, const float* W1s, int warp,
                                            int lane) {
  constexpr int kJ = H / 32;
  for (int sub = (int)blockIdx.x * kEpiWarps + warp; sub < geo.n_c; sub += (int)gridDim.x * kEpiWarps) {
    const size_t nx = sub_stride(geo, sub);
    const float* o = P.u + sub_point(geo, sub, 0, 0);
    // the grid was written earlier in this launch: read through L2
    float gv[4];
    gv[0] = __ldcg(o + lane);                                    // (lane, 0)
    gv[1] = __ldcg(o + (size_t)lane * nx + kPts);                // (32, lane)
    gv[2] = __ldcg(o + (size_t)kPts * nx + (kPts - lane));       // (32 - lane, 32)
    gv[3] = __ldcg(o + (size_t)(kPts - lane) * nx);              // (0, 32 - lane)
    float acc[kJ];
#pragma unroll
    for (int i = 0; i < kJ; ++i) acc[i] = 0.f;
#pragma unroll
    for (int seg = 0; seg < 4; ++seg) {
#pragma unroll 8
      for (int t = 0; t < 32; ++t) {
        const int k = seg * 32 + t;
        const float gk = __shfl_sync(0xffffffffu, gv[seg], t);
        const float* w = W1s + k * H + lane * kJ;
        if constexpr (kJ == 4) {
          const float4 v = *reinterpret_cast<const float4*>(w);
          acc[0] = fmaf(v.x, gk, acc[0]);
          acc[1] = fmaf(v.y, gk, acc[1]);
          acc[2] = fmaf(v.z, gk, acc[2]);
          acc[3] = fmaf(v.w, gk, acc[3]);
        } else {
          const float2 v = *reinterpret_cast<const float2*>(w);
          acc[0] = fmaf(v.x, gk, acc[0]);
          acc[1] = fmaf(v.y, gk, acc[1]);
        }
      }
    }
    float* Bo = const_cast<float*>(P.B) + (size_t)sub * H + lane * kJ;
#pragma unroll
    for (int i = 0; i < kJ; ++i) Bo[i] = acc[i] + __ldg(P.b0 + lane * kJ + i);
  }
}

template <int H, int NH, int ACT, bool kMulti, int DT>
__global__ void __launch_bounds__(kThreadsBf16, 1) mlp_bf16_kernel(const __grid_constant__ Bf16Params P) {
  using C = Bf16Cfg<H, NH>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen = smem_raw + (base - raw);
  const uint32_t sW = base;
  const uint32_t sA = base + C::kWBytes;
  const uint32_t sBar = sA + 2 * C::kABytes;
  // barriers: 0 weights loaded; 1 + 2s + h: K half h of slot s's activations written
  // (8 warp arrivals); 5 + s: slot s's accumulator ready; 7 + s: MMA drain of slot s's
  // issuer; 9 + s: slot s may run its next epilogue phase (8 arrivals of the other slot)
  auto bar = [&](int i) { return sBar + 8u * (uint32_t)i; };
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gen + C::kWBytes + 2 * C::kABytes + 96);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gen + C::kWBytes + 2 * C::kABytes + 104);
  float* half_sum = reinterpret_cast<float*>(gen + C::kWBytes + 2 * C::kABytes + C::kBarBytes);  // [2][128]
  volatile int* pair_ok = reinterpret_cast<volatile int*>(half_sum + 2 * kTileRows);             // [2][4][2]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(bar(0), 1);
    for (int i = 1; i <= 4; ++i) mbar_init(bar(i), 8);
    for (int i = 5; i <= 8; ++i) mbar_init(bar(i), 1);
    for (int i = 9; i <= 10; ++i) mbar_init(bar(i), 8);
    if constexpr (kMulti) mbar_init(bar(11), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == kEpiWarps) {
    tmem_alloc(smem_addr(tmem_holder), C::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp >= kEpiWarps) {
    if (lane == 0) {
      const int s = warp - kEpiWarps;  // the slot this lane issues MMAs for
      if (s == 0) {
        // weights: one bulk async copy per layer, completion counted in bytes
        mbar_arrive_expect_tx(bar(0), C::kWBytes);
#pragma unroll
        for (int l = 0; l < NH; ++l)
          bulk_g2s(sW + (uint32_t)l * H * H * 2, P.wimg + (size_t)l * H * H * 2, H * H * 2, bar(0));
      }
      if (wait_bounded(bar(0), 0, abort_flag, P.status, true)) {
        uint32_t ph0 = 0u, ph1 = 0u;
        if constexpr (kMulti) {
          bool ok = true;
          for (int c = 0; ok && c < P.n_col; ++c)
            ok = mma_issuer<H, NH, ACT, DT>(P, P.n_tiles_c[c], s, tmem, sA, sW, bar(1 + 2 * s), bar(2 + 2 * s),
                                        bar(5 + s), abort_flag, ph0, ph1);
        } else {
          mma_issuer<H, NH, ACT, DT>(P, P.n_tiles, s, tmem, sA, sW, bar(1 + 2 * s), bar(2 + 2 * s), bar(5 + s),
                                 abort_flag, ph0, ph1);
        }
      }
      // drain: every MMA this thread issued has completed before TMEM is released
      mma_commit(bar(7 + s));
      wait_bounded(bar(7 + s), 0, abort_flag, P.status, false);
    }
    __syncwarp();
  } else {
    const int s = warp >> 3, jj = (warp >> 2) & 1, q = warp & 3;
    uint32_t acc_ph = 0u, tok_ph = 0u;
    auto run = [&](const ColourGeom& geo, int n_rows, int n_tiles) {
      if (jj == 0)
        epilogue<H, NH, 0, ACT, kMulti, DT>(P, geo, n_rows, n_tiles, s, q, lane, tmem, sA, bar(1 + 2 * s), bar(2 + 2 * s),
                                        bar(5 + s), bar(9 + s), bar(10 - s), half_sum, pair_ok, abort_flag, acc_ph,
                                        tok_ph);
      else
        epilogue<H, NH, 1, ACT, kMulti, DT>(P, geo, n_rows, n_tiles, s, q, lane, tmem, sA, bar(1 + 2 * s), bar(2 + 2 * s),
                                        bar(5 + s), bar(9 + s), bar(10 - s), half_sum, pair_ok, abort_flag, acc_ph,
                                        tok_ph);
    };
    if constexpr (kMulti) {
      volatile int* go = reinterpret_cast<volatile int*>(gen + C::kWBytes + 2 * C::kABytes + 112);
      const float* W1s = reinterpret_cast<const float*>(gen + C::kWBytes);  // the activation-tile area
      uint32_t w1_ph = 0u;
      unsigned target = 0u;
      for (int c = 0; c < P.n_col; ++c) {
        // stage W1 over the (now idle) activation tiles; earlier generic writes there
        // are ordered before the asynchronous copy
        fence_proxy_async_smem();
        named_barrier_sync(kEpiAllBar, kEpiWarps * 32);
        if (threadIdx.x == 0) {
          mbar_arrive_expect_tx(bar(11), 128u * H * 4u);
          bulk_g2s(sA, P.W1t, 128u * H * 4u, bar(11));
        }
        if (hot_wait_warp<false>(bar(11), w1_ph, abort_flag, P.status)) gather_pass<H>(P, P.gc[c], W1s, warp, lane);
        w1_ph ^= 1u;
        target += gridDim.x;
        if (!epi_grid_sync(P, target, abort_flag, go)) break;  // B of the pass complete everywhere
        run(P.gc[c], P.n_rows_c[c], P.n_tiles_c[c]);
        if (c + 1 == P.n_col) break;
        // the turn tokens may hold phases nobody waited for (a slot with one tile more
        // than the other): start the next pass from fresh token barriers
        named_barrier_sync(kEpiAllBar, kEpiWarps * 32);
        if (threadIdx.x == 0) {
          for (int i = 9; i <= 10; ++i) {
            mbar_inval(bar(i));
            mbar_init(bar(i), 8);
          }
          fence_barrier_init();
        }
        tok_ph = 0u;
        target += gridDim.x;
        if (!epi_grid_sync(P, target, abort_flag, go)) break;  // the pass's predictions are in the grid
      }
    } else {
      run(P.g, P.n_rows, P.n_tiles);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kEpiWarps) {
    tc_fence_after();
    tmem_dealloc(tmem, C::kTmemCols);
  }
}

template <int H, int NH, int ACT, bool kMulti, int DT>
cudaError_t launch_t(const Bf16Params& p, cudaStream_t st) {
  using C = Bf16Cfg<H, NH>;
  // per device: the dynamic shared memory to request and the grid cap (resident CTAs)
  static PerDevice pd;
  int grid_cap = 0;
  size_t smem_bytes = 0;
  cudaError_t e0 = per_device(pd, [](int dev, int* cap, size_t* smem) {
    cudaError_t e = cudaFuncSetAttribute(mlp_bf16_kernel<H, NH, ACT, kMulti, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::kSmem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_bf16_kernel<H, NH, ACT, kMulti, DT>, kThreadsBf16, C::kSmem);
    if (e != cudaSuccess) return e;
    // every resident CTA must be able to hold its tensor memory at once (512 columns):
    // if shared memory alone would admit more CTAs per SM, request more of it
    const int tmem_cap = 512 / (int)C::kTmemCols;
    *smem = C::kSmem;
    if (per_sm > tmem_cap) {
      int smem_sm = 0;
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      *smem = (size_t)smem_sm / (size_t)(tmem_cap + 1) + 1024;
      e = cudaFuncSetAttribute(mlp_bf16_kernel<H, NH, ACT, kMulti, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_bf16_kernel<H, NH, ACT, kMulti, DT>, kThreadsBf16, *smem);
      if (e != cudaSuccess) return e;
    }
    if (per_sm > tmem_cap || per_sm < 1) return cudaErrorInvalidConfiguration;
    *cap = sms * per_sm;
    return cudaSuccess;
  }, &grid_cap, &smem_bytes);
  if (e0 != cudaSuccess) return e0;
  if constexpr (kMulti) {
    // every CTA takes part in every device-wide barrier, so all must be resident at
    // once: a cooperative launch of at most the resident-CTA count
    int most = 0;
    for (int c = 0; c < p.n_col; ++c) most = p.n_tiles_c[c] > most ? p.n_tiles_c[c] : most;
    int grid = (most + kSlots - 1) / kSlots;
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) grid = 1;
    cudaError_t e = cudaMemsetAsync(p.sync, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<Bf16Params*>(&p)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&mlp_bf16_kernel<H, NH, ACT, true, DT>),
                                       dim3(grid), dim3(kThreadsBf16), args, smem_bytes, st);
  } else {
    int grid = (p.n_tiles + kSlots - 1) / kSlots;
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) return cudaSuccess;
    mlp_bf16_kernel<H, NH, ACT, false, DT><<<grid, kThreadsBf16, smem_bytes, st>>>(p);
    return cudaGetLastError();
  }
}

template <int ACT, bool kMulti, int DT>
cudaError_t dispatch(const DevNet& net, const Bf16Params& p, cudaStream_t st) {
  if (net.width == 128) {
    switch (net.n_hidden) {
      case 1: return launch_t<128, 1, ACT, kMulti, DT>(p, st);
      case 2: return launch_t<128, 2, ACT, kMulti, DT>(p, st);
      case 3: return launch_t<128, 3, ACT, kMulti, DT>(p, st);
      case 4: return launch_t<128, 4, ACT, kMulti, DT>(p, st);
      default: return launch_t<128, 5, ACT, kMulti, DT>(p, st);
    }
  }
  switch (net.n_hidden) {
    case 1: return launch_t<64, 1, ACT, kMulti, DT>(p, st);
    case 2: return launch_t<64, 2, ACT, kMulti, DT>(p, st);
    case 3: return launch_t<64, 3, ACT, kMulti, DT>(p, st);
    case 4: return launch_t<64, 4, ACT, kMulti, DT>(p, st);
    default: return launch_t<64, 5, ACT, kMulti, DT>(p, st);
  }
}

void fill_net(const DevNet& net, Bf16Params& p) {
  p.wimg = static_cast<const uint8_t*>(net.wimg_bf16);
  p.bout = net.bout;
  for (int l = 0; l < kMaxHidden; ++l)
    for (int j = 0; j < 128; ++j) p.bias[l][j] = (l < net.n_hidden && j < net.width) ? net.h_bh[l * net.width + j] : 0.f;
  for (int j = 0; j < 128; ++j) {
    p.wout[j] = j < net.width ? net.h_wout[j] : 0.f;
    p.w2[j][0] = j < net.width ? net.h_W2[2 * j] : 0.f;
    p.w2[j][1] = j < net.width ? net.h_W2[2 * j + 1] : 0.f;
  }
}

}  // namespace

bool bf16_supported(const DevNet& net) {
  return (net.width == 64 || net.width == 128) && net.n_hidden >= 1 && net.n_hidden <= kMaxHidden;
}

bool f16_supported(const DevNet& net) { return bf16_supported(net) && net.wimg_f16s != nullptr; }

cudaError_t launch_mlp_bf16(const float* B, const ColourGeom& g, const DevNet& net, float* u, int additive,
                            int* dev_status, cudaStream_t st, bool f16) {
  if (g.n_c <= 0) return cudaSuccess;
  if (!bf16_supported(net) || (f16 && !f16_supported(net))) return cudaErrorNotSupported;
  Bf16Params p{};
  p.B = B;
  p.u = u;
  p.status = dev_status;
  p.g = g;
  p.n_rows = g.n_c * g.rows_per_sub;
  p.n_tiles = (p.n_rows + kTileRows - 1) / kTileRows;
  p.additive = additive;
  fill_net(net, p);
  if (f16) {
    p.wimg = static_cast<const uint8_t*>(net.wimg_f16s);
    if (net.act == kActGelu) return dispatch<kActGelu, false, kDtF16>(net, p, st);
    return dispatch<kActTanh, false, kDtF16>(net, p, st);
  }
  if (net.act == kActGelu) return dispatch<kActGelu, false, kDtBf16>(net, p, st);
  return dispatch<kActTanh, false, kDtBf16>(net, p, st);
}

bool bf16_sweep_supported(const DevNet& net) { return bf16_supported(net) && net.embed_c == 0; }

cudaError_t launch_mlp_bf16_sweep(const ColourGeom* gc, int n_col, const DevNet& net, float* u, float* B,
                                  unsigned int* sync, int* dev_status, cudaStream_t st) {
  if (n_col < 1 || n_col > 4) return cudaErrorInvalidValue;
  if (!bf16_sweep_supported(net)) return cudaErrorNotSupported;
  Bf16Params p{};
  p.B = B;
  p.u = u;
  p.status = dev_status;
  p.additive = 0;
  p.n_col = n_col;
  for (int c = 0; c < n_col; ++c) {
    p.gc[c] = gc[c];
    p.n_rows_c[c] = gc[c].n_c * gc[c].rows_per_sub;
    p.n_tiles_c[c] = (p.n_rows_c[c] + kTileRows - 1) / kTileRows;
  }
  p.W1t = net.W1t;
  p.b0 = net.b0;
  p.sync = sync;
  fill_net(net, p);
  if (net.act == kActGelu) return dispatch<kActGelu, true, kDtBf16>(net, p, st);
  return dispatch<kActTanh, true, kDtBf16>(net, p, st);
}

}  // namespace mf
