// K3: BF16 SDNet over one colour on the 5th-generation tensor cores, fused with the
// scatter into the grid.
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
//   warps 0-15 epilogue: warp w owns TMEM lanes / tile rows 32(w mod 4)..+31 and output
//              columns (w/4)*H/4..+H/4-1, and serves the two tile slots in alternation
//   warp 16    TMEM allocation; lane 0 loads the weights (bulk async copy) and issues
//              the MMAs of slot 0
//   warp 17    lane 0 issues the MMAs of slot 1
// Each issuing lane blocks on its own slot's barriers, and its tcgen05.commit tracks
// exactly its slot's MMAs, so the two slots run independently and one slot's epilogue
// overlaps the other slot's MMAs.
// Shared memory: all hidden weight matrices resident (n_hidden x H x H BF16) plus one
// 128 x H BF16 activation tile per slot, all in the 128-byte-swizzled K-major layout
// the MMA descriptors name. TMEM: H FP32 columns per slot.
//
// Every mbarrier wait is bounded (about one second of %globaltimer); a wait that gives
// up records kDevErrTimeout in the status word, raises a CTA-wide abort flag so the
// other roles stop too, and the MMA lane drains its in-flight MMAs (bounded) before the
// CTA frees its tensor memory and exits.
#include <stdint.h>

#include "mf_internal.cuh"

namespace mf {

namespace {

constexpr int kMaxHidden = 5;
constexpr int kEpiWarps = 16;                     // 4 row quadrants x 4 column quarters
constexpr int kThreadsBf16 = (kEpiWarps + 2) * 32;  // + one MMA-issuing warp per slot
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

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
};

// ---------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t x) {
  uint32_t d;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(d) : "r"(x));
  return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ void named_barrier_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle layout:
// 8-row groups of 128-byte rows, groups 1024 bytes apart (SBO); descriptor version 1;
// swizzle mode 2 (128B). The leading-byte offset is unused for this layout.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Bounded wait on an mbarrier phase; false once the CTA is aborting or after the limit.
__device__ __noinline__ bool wait_bounded(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          bool honour_abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (honour_abort && *abort_flag) return false;
    if (globaltimer() - t0 > kWaitLimitNs) {
      *abort_flag = 1;
      atomicExch(status, kDevErrTimeout);
      return false;
    }
  }
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Spinning bounded wait: polls the phase without suspending (a suspended try_wait wakes
// a few hundred cycles after the phase completes, which sits on the critical path);
// the abort flag and the time limit are checked every 64 polls.
__device__ __noinline__ bool wait_spin(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 63u) == 0u) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > kWaitLimitNs) {
        *abort_flag = 1;
        atomicExch(status, kDevErrTimeout);
        return false;
      }
    }
  }
}

// Warp-uniform form: every lane waits, and the warp continues only if all lanes saw
// the phase complete (the .sync.aligned tcgen05 loads that follow need the whole warp).
__device__ __forceinline__ bool wait_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  const bool ok = wait_spin(bar, parity, abort_flag, status);
  return __all_sync(0xffffffffu, ok);
}

// ---------------------------------------------------------------- kernel
//
// Scheduling. The 16 epilogue warps serve one tile slot at a time and alternate:
// epilogue phase m of slot 0, then phase m of slot 1, then phase m+1 of slot 0, ...
// (phase 0 is the first layer, phase m the output of hidden layer m). Warp w owns TMEM
// lanes / tile rows 32(w mod 4)..+31 and columns (w/4)*H/4 .. +H/4-1, so each SM
// sub-partition runs four warps of the current phase. A slot's MMAs for layer m+1 are
// issued as soon as its phase m has written the activations and run while the warps
// work on the other slot, so the tensor core and the MUFU (tanh) unit overlap without
// any cross-slot signal: the alternation is just program order. Accumulators are
// double-buffered per slot in TMEM (layer parity picks the buffer) because the MMAs of
// layer m+1 start on the first column quarter while other warps still read layer m.

constexpr int kQuarters = 4;

template <int H, int NH>
struct Bf16Cfg {
  static constexpr int kGW = H / kQuarters;                         // columns per warp (one K quarter)
  static constexpr int kKStepsGroup = kGW / 16;                     // K=16 steps per quarter
  static constexpr uint32_t kWBytes = (uint32_t)NH * H * H * 2;     // resident hidden weights
  static constexpr uint32_t kABytes = (uint32_t)kTileRows * H * 2;  // one activation tile
  static constexpr uint32_t kTmemCols = 4 * H;                      // 2 slots x 2 buffers x H
  static constexpr uint32_t kBarBytes = 192;
  static constexpr uint32_t kSumBytes = 3 * kTileRows * 4 + 64;     // output partial sums + flags
  static constexpr size_t kSmem = 1024 + kWBytes + 2 * kABytes + kBarBytes + kSumBytes;
  static constexpr uint32_t kIdesc = idesc_bf16(kTileRows, H);
  static_assert(kKStepsGroup >= 1 && kGW % 8 == 0, "quarter geometry");
};

// Byte offset, within a K-major SW128 operand of `rows` rows, of K step `ks` (16 elements).
__host__ __device__ constexpr uint32_t kstep_off(int rows, int ks) {
  return (uint32_t)(ks >> 2) * (uint32_t)(rows * 128) + (uint32_t)(ks & 3) * 32u;
}

// Descriptor whose start address is advanced by `bytes` (the start field is the low 14
// bits of the low word and stays below 2^14, so a 32-bit add on the low word suffices).
__device__ __forceinline__ uint64_t desc_add(uint64_t d, uint32_t bytes) {
  const uint32_t lo = (uint32_t)d + (bytes >> 4), hi = (uint32_t)(d >> 32);
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}

template <uint32_t ACC>
__device__ __forceinline__ void mma_bf16_c(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "n"(ACC)
      : "memory");
}

__device__ __forceinline__ bool slot_has_tile(const Bf16Params& P, int round, int slot) {
  return ((round * (int)gridDim.x + (int)blockIdx.x) * 2 + slot) < P.n_tiles;
}

// MMA issue for one slot (a single thread): per tile and hidden layer m, for each K
// quarter the quarter's K steps once its activations are written, then one commit for
// the whole accumulator. Every descriptor is a base plus a compile-time offset.
template <int H, int NH>
__device__ __forceinline__ void mma_issuer(const Bf16Params& P, int s, uint32_t tmem, uint32_t sA, uint32_t sW,
                                           uint32_t bar_act, uint32_t bar_acc, volatile int* abort_flag) {
  using C = Bf16Cfg<H, NH>;
  const uint32_t acc0 = tmem + (uint32_t)(s * 2 * H);
  uint32_t ph = 0u;  // bit g: phase parity of quarter g's barrier
  bool ok = true;
  for (int k = 0; ok && slot_has_tile(P, k, s); ++k) {
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
      for (int g = 0; g < kQuarters; ++g) {
        ok = wait_spin(bar_act + 8u * (uint32_t)g, (ph >> g) & 1u, abort_flag, P.status);
        if (!ok) break;
        ph ^= 1u << g;
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < C::kKStepsGroup; ++kk) {
          const int ks = g * C::kKStepsGroup + kk;
          const uint64_t ad = desc_add(a0, kstep_off(kTileRows, ks));
          const uint64_t bd = desc_add(w0, (uint32_t)(m - 1) * H * H * 2 + kstep_off(H, ks));
          if (ks == 0) mma_bf16_c<0>(acc, ad, bd, C::kIdesc);
          else mma_bf16_c<1>(acc, ad, bd, C::kIdesc);
        }
      }
      if (!ok) break;
      mma_commit(bar_acc);
    }
  }
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t* v) {
  if constexpr (N == 32) tmem_ld32(taddr, *reinterpret_cast<uint32_t(*)[32]>(v));
  else if constexpr (N == 16) tmem_ld16(taddr, v);
  else tmem_ld8(taddr, v);
}

// Epilogue of warp (row quadrant q, column quarter G): TMEM lanes 32q..32q+31, columns
// G*H/4 .. G*H/4 + H/4 - 1, for both tile slots in alternation.
template <int H, int NH, int G>
__device__ __forceinline__ void epilogue(const Bf16Params& P, int q, int lane, uint32_t tmem, uint32_t sA,
                                         uint32_t bar_act_base, uint32_t bar_acc_base, float* part,
                                         volatile int* quad_ok, volatile int* abort_flag) {
  using C = Bf16Cfg<H, NH>;
  constexpr int GW = C::kGW;
  constexpr int c0 = G * GW;  // first column of this warp
  const int rloc = 32 * q + lane;
  const uint32_t swz = (uint32_t)(rloc & 7) << 4;
  const int named = 1 + q;    // named barrier of the four column-quarter warps of these rows
  uint32_t acc_ph = 0u;       // bit s: phase parity of slot s's accumulator barrier
  bool ok = true;

  auto a_row = [&](int s) { return sA + (uint32_t)s * C::kABytes + (uint32_t)rloc * 128u; };
  auto st_cols = [&](int s, const uint32_t* pk) {  // this warp's GW columns of row rloc
#pragma unroll
    for (int i = 0; i < GW / 8; ++i) {
      const int c = c0 / 8 + i;
      const uint32_t addr = a_row(s) + (uint32_t)(c >> 3) * (kTileRows * 128u) + (((uint32_t)(c & 7) << 4) ^ swz);
      st_shared_v4(addr, pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
    }
  };
  auto signal = [&](int s) {  // this warp's quarter of slot s's activations is written
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(bar_act_base + 8u * (uint32_t)(kQuarters * s + G));
  };

  for (int k = 0; ok && slot_has_tile(P, k, 0); ++k) {
    const int nslots = slot_has_tile(P, k, 1) ? 2 : 1;
    float uacc[2] = {0.f, 0.f};
    // row of slot s in this round (clamped to the last row for the ragged tail)
    auto row_of = [&](int s) { return ((k * (int)gridDim.x + (int)blockIdx.x) * 2 + s) * kTileRows + rloc; };

    // phase 0 (first layer, Eq. 8): FP32 sum B[s] + W2 x, rounded to BF16, tanh
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (s >= nslots) break;
      const RowSite site = row_site(P.g, min(row_of(s), P.n_rows - 1));
      const float x = (float)(site.px + 1) * (1.0f / kPts), y = (float)(site.py + 1) * (1.0f / kPts);
      const float2* Bs = reinterpret_cast<const float2*>(P.B + (size_t)site.s * H + c0);
      float2 bb[GW / 2];
#pragma unroll
      for (int i = 0; i < GW / 2; ++i) bb[i] = __ldg(Bs + i);
      uint32_t pk[GW / 2];
#pragma unroll
      for (int i = 0; i < GW / 2; ++i) {
        const int col = c0 + 2 * i;
        const float a0 = fmaf(P.w2[col][1], y, fmaf(P.w2[col][0], x, bb[i].x));
        const float a1 = fmaf(P.w2[col + 1][1], y, fmaf(P.w2[col + 1][0], x, bb[i].y));
        pk[i] = tanh_bf16x2(pack_bf16x2(a0, a1));
      }
      st_cols(s, pk);
      signal(s);
    }

    // phases 1..NH
#pragma unroll
    for (int m = 1; m <= NH; ++m) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (s >= nslots || !ok) break;
        ok = wait_warp(bar_acc_base + 8u * (uint32_t)s, (acc_ph >> s) & 1u, abort_flag, P.status);
        if (!ok) break;
        acc_ph ^= 1u << s;
        tc_fence_after();
        uint32_t pk[GW / 2];
        const uint32_t taddr = tmem + (uint32_t)(s * 2 * H + (m & 1) * H + c0) + ((uint32_t)(32 * q) << 16);
#pragma unroll
        for (int h = 0; h < GW / 16 || h == 0; ++h) {  // 16-column pieces keep registers low
          constexpr int PW = GW < 16 ? GW : 16;
          uint32_t v[PW];
          tmem_ld<PW>(taddr + (uint32_t)(h * PW), v);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < PW / 2; ++i) {
            const int col = c0 + h * PW + 2 * i;
            const float a0 = __uint_as_float(v[2 * i]) + P.bias[m - 1][col];
            const float a1 = __uint_as_float(v[2 * i + 1]) + P.bias[m - 1][col + 1];
            pk[h * PW / 2 + i] = tanh_bf16x2(pack_bf16x2(a0, a1));
          }
        }
        tc_fence_before();
        if (m < NH) {
          st_cols(s, pk);
          signal(s);
        } else {
          float u = 0.f;
#pragma unroll
          for (int i = 0; i < GW / 2; ++i) {
            u = fmaf(bf16_lo(pk[i]), P.wout[c0 + 2 * i], u);
            u = fmaf(bf16_hi(pk[i]), P.wout[c0 + 2 * i + 1], u);
          }
          uacc[s] = u;
        }
      }
    }

    // output: the four column-quarter warps of these rows add their partial sums (in a
    // fixed order) and agree on whether to continue, so no warp leaves while the others
    // wait at the named barrier
    const bool ok_warp = __all_sync(0xffffffffu, ok);
    if (lane == 0) quad_ok[q * 4 + G] = ok_warp ? 1 : 0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (G > 0) part[(G - 1) * kTileRows + rloc] = uacc[s];
      named_barrier_sync(named, 128);
      const bool ok_all = quad_ok[q * 4 + 0] && quad_ok[q * 4 + 1] && quad_ok[q * 4 + 2] && quad_ok[q * 4 + 3];
      const int row = row_of(s);
      if (G == 0 && ok_all && s < nslots && row < P.n_rows) {
        const RowSite site = row_site(P.g, row);
        const float val = ((uacc[s] + part[rloc]) + part[kTileRows + rloc]) + part[2 * kTileRows + rloc] + P.bout;
        if (P.additive)
          P.u[site.idx] += cover_weight(P.g, site.ix, site.iy) * val;
        else
          P.u[site.idx] = val;
      }
      named_barrier_sync(named, 128);
      ok = ok_all;
    }
  }
}

template <int H, int NH>
__global__ void __launch_bounds__(kThreadsBf16, 1) mlp_bf16_kernel(const __grid_constant__ Bf16Params P) {
  using C = Bf16Cfg<H, NH>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen = smem_raw + (base - raw);
  const uint32_t sW = base;
  const uint32_t sA = base + C::kWBytes;
  const uint32_t sBar = sA + 2 * C::kABytes;
  // barriers: 0 weights loaded; 1 + 4*slot + g: quarter g of the slot's activations
  // written (4 warp arrivals); 9 + slot: accumulator of the slot ready; 11 + slot: MMA
  // drain of that slot's issuer
  auto bar = [&](int i) { return sBar + 8u * (uint32_t)i; };
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gen + C::kWBytes + 2 * C::kABytes + 160);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gen + C::kWBytes + 2 * C::kABytes + 168);
  float* part = reinterpret_cast<float*>(gen + C::kWBytes + 2 * C::kABytes + C::kBarBytes);  // [3][128]
  volatile int* quad_ok = reinterpret_cast<volatile int*>(part + 3 * kTileRows);              // [4][4]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(bar(0), 1);
    for (int i = 1; i <= 8; ++i) mbar_init(bar(i), 4);
    for (int i = 9; i <= 12; ++i) mbar_init(bar(i), 1);
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
      if (wait_bounded(bar(0), 0, abort_flag, P.status, true))
        mma_issuer<H, NH>(P, s, tmem, sA, sW, bar(1 + 4 * s), bar(9 + s), abort_flag);
      // drain: every MMA this thread issued has completed before TMEM is released
      mma_commit(bar(11 + s));
      wait_bounded(bar(11 + s), 0, abort_flag, P.status, false);
    }
    __syncwarp();
  } else {
    const int q = warp & 3, g = warp >> 2;
    switch (g) {
      case 0: epilogue<H, NH, 0>(P, q, lane, tmem, sA, bar(1), bar(9), part, quad_ok, abort_flag); break;
      case 1: epilogue<H, NH, 1>(P, q, lane, tmem, sA, bar(1), bar(9), part, quad_ok, abort_flag); break;
      case 2: epilogue<H, NH, 2>(P, q, lane, tmem, sA, bar(1), bar(9), part, quad_ok, abort_flag); break;
      default: epilogue<H, NH, 3>(P, q, lane, tmem, sA, bar(1), bar(9), part, quad_ok, abort_flag); break;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kEpiWarps) {
    tc_fence_after();
    tmem_dealloc(tmem, C::kTmemCols);
  }
}

template <int H, int NH>
cudaError_t launch_t(const Bf16Params& p, cudaStream_t st) {
  using C = Bf16Cfg<H, NH>;
  static int grid_cap = 0;
  static size_t smem_bytes = 0;
  if (grid_cap == 0) {
    cudaError_t e = cudaFuncSetAttribute(mlp_bf16_kernel<H, NH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::kSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_bf16_kernel<H, NH>, kThreadsBf16, C::kSmem);
    if (e != cudaSuccess) return e;
    // every resident CTA must be able to hold its tensor memory at once (512 columns):
    // if shared memory alone would admit more CTAs per SM, request more of it
    const int tmem_cap = 512 / (int)C::kTmemCols;
    smem_bytes = C::kSmem;
    if (per_sm > tmem_cap) {
      int smem_sm = 0;
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      smem_bytes = (size_t)smem_sm / (size_t)(tmem_cap + 1) + 1024;
      e = cudaFuncSetAttribute(mlp_bf16_kernel<H, NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_bf16_kernel<H, NH>, kThreadsBf16, smem_bytes);
      if (e != cudaSuccess) return e;
    }
    if (per_sm > tmem_cap || per_sm < 1) return cudaErrorInvalidConfiguration;
    grid_cap = sms * per_sm;
  }
  int grid = (p.n_tiles + 1) / 2;
  if (grid > grid_cap) grid = grid_cap;
  if (grid < 1) return cudaSuccess;
  mlp_bf16_kernel<H, NH><<<grid, kThreadsBf16, smem_bytes, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

bool bf16_supported(const DevNet& net) {
  return (net.width == 64 || net.width == 128) && net.n_hidden >= 1 && net.n_hidden <= kMaxHidden;
}

cudaError_t launch_mlp_bf16(const float* B, const ColourGeom& g, const DevNet& net, float* u, int additive,
                            int* dev_status, cudaStream_t st) {
  if (g.n_c <= 0) return cudaSuccess;
  if (!bf16_supported(net)) return cudaErrorNotSupported;
  Bf16Params p;
  p.B = B;
  p.u = u;
  p.wimg = static_cast<const uint8_t*>(net.wimg_bf16);
  p.status = dev_status;
  p.g = g;
  p.n_rows = g.n_c * kNint;
  p.n_tiles = (p.n_rows + kTileRows - 1) / kTileRows;
  p.additive = additive;
  p.bout = net.bout;
  for (int l = 0; l < kMaxHidden; ++l)
    for (int j = 0; j < 128; ++j) p.bias[l][j] = (l < net.n_hidden && j < net.width) ? net.h_bh[l * net.width + j] : 0.f;
  for (int j = 0; j < 128; ++j) {
    p.wout[j] = j < net.width ? net.h_wout[j] : 0.f;
    p.w2[j][0] = j < net.width ? net.h_W2[2 * j] : 0.f;
    p.w2[j][1] = j < net.width ? net.h_W2[2 * j + 1] : 0.f;
  }
  if (net.width == 128) {
    switch (net.n_hidden) {
      case 1: return launch_t<128, 1>(p, st);
      case 2: return launch_t<128, 2>(p, st);
      case 3: return launch_t<128, 3>(p, st);
      case 4: return launch_t<128, 4>(p, st);
      default: return launch_t<128, 5>(p, st);
    }
  }
  switch (net.n_hidden) {
    case 1: return launch_t<64, 1>(p, st);
    case 2: return launch_t<64, 2>(p, st);
    case 3: return launch_t<64, 3>(p, st);
    case 4: return launch_t<64, 4>(p, st);
    default: return launch_t<64, 5>(p, st);
  }
}

}  // namespace mf
