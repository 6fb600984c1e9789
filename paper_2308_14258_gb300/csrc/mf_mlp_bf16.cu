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
// Persistent CTA per SM, 9 warps:
//   warps 0-3  epilogue of tile slot 0 (warp w owns TMEM lanes / tile rows 32(w%4)..+31)
//   warps 4-7  epilogue of tile slot 1
//   warp 8     TMEM allocation; one lane loads the weights (bulk async copy) and issues
//              the MMAs, alternating slots so that one slot's epilogue overlaps the
//              other slot's MMAs.
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
constexpr int kThreadsBf16 = 288;
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
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
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

// Byte offset of the 16-byte chunk `chunk` (8 BF16 along K) of row `row` of a K-major
// 128B-swizzled operand with `rows` rows: K blocks of 64 elements are rows*128 bytes
// apart; the chunk index is XORed with row mod 8.
__device__ __forceinline__ uint32_t sw128_offset(int rows, int row, int kchunk) {
  const int kb = kchunk >> 3, c = kchunk & 7;
  return (uint32_t)(kb * rows * 128 + row * 128 + ((c ^ (row & 7)) << 4));
}

// Warp-uniform form: every lane waits, and the warp continues only if all lanes saw
// the phase complete (the .sync.aligned tcgen05 loads that follow need the whole warp).
__device__ __forceinline__ bool wait_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
  const bool ok = wait_bounded(bar, parity, abort_flag, status, true);
  return __all_sync(0xffffffffu, ok);
}

// ---------------------------------------------------------------- kernel

template <int H, int NH>
struct Bf16Cfg {
  static constexpr uint32_t kWBytes = (uint32_t)NH * H * H * 2;     // resident hidden weights
  static constexpr uint32_t kABytes = (uint32_t)kTileRows * H * 2;  // one activation tile
  static constexpr uint32_t kTmemCols = 2 * H;                      // H FP32 columns per slot
  static constexpr uint32_t kBarBytes = 128;
  static constexpr size_t kSmem = 1024 + kWBytes + 2 * kABytes + kBarBytes;
  static constexpr uint32_t kIdesc = idesc_bf16(kTileRows, H);
};

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
  // barriers: 0 weights loaded, 1-2 activations ready (per slot), 3-4 accumulator
  // ready (per slot), 5 MMA drain
  auto bar = [&](int i) { return sBar + 8u * (uint32_t)i; };
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gen + C::kWBytes + 2 * C::kABytes + 64);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gen + C::kWBytes + 2 * C::kABytes + 72);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(bar(0), 1);
    mbar_init(bar(1), 128);
    mbar_init(bar(2), 128);
    mbar_init(bar(3), 1);
    mbar_init(bar(4), 1);
    mbar_init(bar(5), 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 8) {
    tmem_alloc(smem_addr(tmem_holder), C::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 8) {
    if (lane == 0) {
      // ---- weights: one bulk async copy per layer, completion counted in bytes
      mbar_arrive_expect_tx(bar(0), C::kWBytes);
#pragma unroll
      for (int l = 0; l < NH; ++l)
        bulk_g2s(sW + (uint32_t)l * H * H * 2, P.wimg + (size_t)l * H * H * 2, H * H * 2, bar(0));
      bool ok = wait_bounded(bar(0), 0, abort_flag, P.status, true);
      uint32_t act_phase[2] = {0u, 0u};
      for (int k = 0; ok; ++k) {
        const int t0 = (k * (int)gridDim.x + (int)blockIdx.x) * 2;
        if (t0 >= P.n_tiles) break;
        const int nslots = (t0 + 1 < P.n_tiles) ? 2 : 1;
        for (int l = 0; l < NH && ok; ++l) {
          for (int slot = 0; slot < nslots; ++slot) {
            ok = wait_bounded(bar(1 + slot), act_phase[slot], abort_flag, P.status, true);
            if (!ok) break;
            act_phase[slot] ^= 1u;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(slot * H);
            const uint32_t a0 = sA + (uint32_t)slot * C::kABytes;
            const uint32_t b0 = sW + (uint32_t)l * H * H * 2;
#pragma unroll
            for (int kk = 0; kk < H / 16; ++kk) {
              const uint32_t koff_a = (uint32_t)(kk >> 2) * (kTileRows * 128) + (uint32_t)(kk & 3) * 32;
              const uint32_t koff_b = (uint32_t)(kk >> 2) * (H * 128) + (uint32_t)(kk & 3) * 32;
              mma_bf16(d, desc_sw128(a0 + koff_a), desc_sw128(b0 + koff_b), C::kIdesc, kk > 0 ? 1u : 0u);
            }
            mma_commit(bar(3 + slot));
          }
        }
      }
      // ---- drain: every MMA issued above has completed before TMEM is released
      mma_commit(bar(5));
      wait_bounded(bar(5), 0, abort_flag, P.status, false);
    }
    __syncwarp();
  } else {
    // ---- epilogue roles
    const int slot = warp >> 2, q = warp & 3;
    const int rloc = 32 * q + lane;  // tile row = TMEM lane
    const uint32_t a_tile = sA + (uint32_t)slot * C::kABytes;
    const uint32_t t_row = tmem + (uint32_t)(slot * H) + ((uint32_t)(32 * q) << 16);
    uint32_t acc_phase = 0u;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int tile = (k * (int)gridDim.x + (int)blockIdx.x) * 2 + slot;
      if (tile >= P.n_tiles) break;
      const int row = tile * kTileRows + rloc;
      const bool valid = row < P.n_rows;
      const RowSite site = row_site(P.g, valid ? row : P.n_rows - 1);
      const float x = (float)(site.px + 1) * (1.0f / kPts), y = (float)(site.py + 1) * (1.0f / kPts);
      const float* Bs = P.B + (size_t)site.s * H;

      // first layer (Eq. 8), FP32 sum, rounded to BF16, tanh
#pragma unroll
      for (int c = 0; c < H / 32; ++c) {
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = 32 * c + 2 * j;
          const float2 bb = __ldg(reinterpret_cast<const float2*>(Bs + col));
          const float a0 = fmaf(P.w2[col][1], y, fmaf(P.w2[col][0], x, bb.x));
          const float a1 = fmaf(P.w2[col + 1][1], y, fmaf(P.w2[col + 1][0], x, bb.y));
          pk[j] = tanh_bf16x2(pack_bf16x2(a0, a1));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          st_shared_v4(a_tile + sw128_offset(kTileRows, rloc, 4 * c + i), pk[4 * i], pk[4 * i + 1],
                       pk[4 * i + 2], pk[4 * i + 3]);
      }
      fence_proxy_async_smem();
      mbar_arrive(bar(1 + slot));

      float uacc = 0.f;
#pragma unroll
      for (int l = 0; l < NH; ++l) {
        ok = wait_warp(bar(3 + slot), acc_phase, abort_flag, P.status);
        if (!ok) break;
        acc_phase ^= 1u;
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < H / 32; ++c) {
          uint32_t v[32];
          tmem_ld32(t_row + (uint32_t)(32 * c), v);
          tmem_wait_ld();
          uint32_t pk[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = 32 * c + 2 * j;
            const float a0 = __uint_as_float(v[2 * j]) + P.bias[l][col];
            const float a1 = __uint_as_float(v[2 * j + 1]) + P.bias[l][col + 1];
            pk[j] = tanh_bf16x2(pack_bf16x2(a0, a1));
          }
          if (l + 1 < NH) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              st_shared_v4(a_tile + sw128_offset(kTileRows, rloc, 4 * c + i), pk[4 * i], pk[4 * i + 1],
                           pk[4 * i + 2], pk[4 * i + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              uacc = fmaf(bf16_lo(pk[j]), P.wout[32 * c + 2 * j], uacc);
              uacc = fmaf(bf16_hi(pk[j]), P.wout[32 * c + 2 * j + 1], uacc);
            }
          }
        }
        tc_fence_before();
        if (l + 1 < NH) {
          fence_proxy_async_smem();
          mbar_arrive(bar(1 + slot));
        }
      }
      if (ok && valid) {
        const float val = uacc + P.bout;
        if (P.additive)
          P.u[site.idx] += cover_weight(P.g, site.ix, site.iy) * val;
        else
          P.u[site.idx] = val;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    tmem_dealloc(tmem, C::kTmemCols);
  }
}

template <int H, int NH>
cudaError_t launch_t(const Bf16Params& p, cudaStream_t st) {
  using C = Bf16Cfg<H, NH>;
  static int grid_cap = 0;
  if (grid_cap == 0) {
    cudaError_t e = cudaFuncSetAttribute(mlp_bf16_kernel<H, NH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::kSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_bf16_kernel<H, NH>, kThreadsBf16, C::kSmem);
    if (e != cudaSuccess) return e;
    // every resident CTA must be able to hold its tensor memory at once (512 columns)
    const int tmem_cap = 512 / (int)C::kTmemCols;
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid_cap = sms * per_sm;
  }
  int grid = (p.n_tiles + 1) / 2;
  if (grid > grid_cap) grid = grid_cap;
  if (grid < 1) return cudaSuccess;
  mlp_bf16_kernel<H, NH><<<grid, kThreadsBf16, C::kSmem, st>>>(p);
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
