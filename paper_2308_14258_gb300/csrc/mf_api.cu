// C ABI of the Mosaic Flow sweep engine: handles, validation, weight packing and the
// sweep driver (Section 2.4, Section 4.1, Algorithm 2). All arithmetic of the sweep
// runs in the kernels of this library; this file only validates, allocates, packs and
// enqueues.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mosaicflow.h"
#include "mf_internal.cuh"

struct mf_sdnet {
  int device = 0;
  mf::DevNet d{};
  void* dmem = nullptr;           // one device allocation for every weight array
  std::vector<float> h_bh, h_wout, h_W2;
};

struct mf_grid {
  int device = 0;
  int lx = 0, ly = 0, nx = 0, ny = 0;
  float* u = nullptr;       // current grid
  float* prev = nullptr;    // grid before the sweep (delta, additive reads)
  float* B = nullptr;       // [max colour subdomains][128] first-layer term
  double* partial = nullptr;
  double* out = nullptr;    // 16 doubles: [0..4] sweep reduction + delta, [8..12] residual
  int* status = nullptr;    // kernel status word
  unsigned int* sync = nullptr;  // barrier counter of the whole-sweep launch
  double* h_out = nullptr;  // pinned host mirror of out (16 doubles)
  int* h_status = nullptr;  // pinned host mirror of status
  std::vector<cudaEvent_t> events;  // profiling events, grown on demand
};

namespace {

thread_local std::string g_err;

mf_status fail(mf_status code, const std::string& msg) {
  g_err = msg;
  return code;
}

mf_status cuda_fail(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(e == cudaErrorMemoryAllocation ? MF_ERR_OUT_OF_MEMORY : MF_ERR_CUDA, m);
}

#define MF_CUDA(call, what)                     \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Make the handle's device current for the rest of the enclosing call.
#define MF_ON_DEVICE(dev, what)                  \
  mf::DeviceGuard guard_((dev));                 \
  if (guard_.err != cudaSuccess) return cuda_fail(guard_.err, what)

uint16_t bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40u);  // NaN
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// BF16 image of one H x H matrix W[n][k] (row n = output unit) as the B operand of
// tcgen05.mma: K-major, 128-byte swizzle: K blocks of 64 elements, each block holds
// H rows of 128 bytes, 16-byte chunk c of row n stored at chunk c ^ (n mod 8).
// f16: F16 elements (round to nearest even) instead of BF16.
void pack_sw128(const float* W, int H, uint16_t* img, bool f16 = false) {
  for (int n = 0; n < H; ++n)
    for (int k = 0; k < H; ++k) {
      const int kb = k / 64, w = k % 64, chunk = w / 8, e = w % 8;
      const size_t off = (size_t)kb * H * 64 + (size_t)n * 64 + (size_t)((chunk ^ (n & 7)) * 8) + e;
      const float x = W[(size_t)n * H + k];
      if (f16) {
        const __half h = __float2half_rn(x);
        std::memcpy(&img[off], &h, sizeof(uint16_t));
      } else {
        img[off] = bf16_rne(x);
      }
    }
}

mf::ColourGeom colour_geom(const mf_grid* g, int c) {
  mf::ColourGeom cg{};
  cg.nx = g->nx;
  cg.ca = c & 1;
  cg.cb = c >> 1;
  cg.nsx = 2 * g->lx - 1;
  cg.nsy = 2 * g->ly - 1;
  const int n_a = (cg.nsx - cg.ca + 1) / 2;
  const int n_b = (cg.nsy - cg.cb + 1) / 2;
  cg.n_a = n_a;
  cg.n_c = n_a * n_b;
  cg.centre = 0;
  cg.rows_per_sub = mf::kNint;
  cg.table = nullptr;
  return cg;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Phase timer: consecutive events on the launching stream; each interval is charged to
// the phase named when its closing event was recorded.
struct PhaseTimer {
  mf_grid* g;
  cudaStream_t st;
  bool on;
  size_t n = 0;
  std::vector<int> phase;  // phase of interval i (between event i and i+1)
  cudaError_t mark(int next_phase_of_previous) {
    if (!on) return cudaSuccess;
    if (n == g->events.size()) {
      cudaEvent_t ev;
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return e;
      g->events.push_back(ev);
    }
    if (n > 0) phase.push_back(next_phase_of_previous);
    return cudaEventRecord(g->events[n++], st);
  }
  cudaError_t totals(double ms[3]) {
    ms[0] = ms[1] = ms[2] = 0.0;
    if (!on) return cudaSuccess;
    for (size_t i = 0; i + 1 < n; ++i) {
      float t = 0.f;
      cudaError_t e = cudaEventElapsedTime(&t, g->events[i], g->events[i + 1]);
      if (e != cudaSuccess) return e;
      ms[phase[i]] += t;
    }
    return cudaSuccess;
  }
};
enum { kPhaseGather = 0, kPhaseMlp = 1, kPhaseReduce = 2 };

}  // namespace

namespace mf {
// Internal accessors used by the allocation-free sweep (mf_noalloc.cu).
const DevNet* devnet_of(const mf_sdnet* net, int* device) {
  if (device) *device = net->device;
  return &net->d;
}
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace mf

extern "C" {

const char* mf_last_error(void) { return g_err.c_str(); }

int mf_version(void) { return 300; }

mf_status mf_ctx_create(int device, mf_ctx** out) {
  if (!out) return fail(MF_ERR_INVALID_ARG, "mf_ctx_create: null argument");
  *out = nullptr;
  if (device < 0 || device >= mf::kMaxDevices) return fail(MF_ERR_INVALID_ARG, "mf_ctx_create: bad device index");
  int count = 0;
  MF_CUDA(cudaGetDeviceCount(&count), "mf_ctx_create: cudaGetDeviceCount");
  if (device >= count) return fail(MF_ERR_INVALID_ARG, "mf_ctx_create: no such device");
  MF_ON_DEVICE(device, "mf_ctx_create: cudaSetDevice");
  MF_CUDA(cudaFree(nullptr), "mf_ctx_create: context initialisation");
  int major = 0, minor = 0, sms = 0;
  MF_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device), "mf_ctx_create: attribute");
  MF_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device), "mf_ctx_create: attribute");
  MF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "mf_ctx_create: attribute");
  if (major != 10 || minor != 3)
    return fail(MF_ERR_UNSUPPORTED, "mf_ctx_create: the library carries sm_103a code only; device has compute "
                                    "capability " + std::to_string(major) + "." + std::to_string(minor));
  mf_ctx* c = new mf_ctx();
  c->device = device;
  c->sms = sms;
  *out = c;
  return MF_OK;
}

mf_status mf_ctx_destroy(mf_ctx* ctx) {
  delete ctx;
  return MF_OK;
}

mf_status mf_ctx_device(const mf_ctx* ctx, int* device, int* sm_count) {
  if (!ctx) return fail(MF_ERR_INVALID_ARG, "mf_ctx_device: null context");
  if (device) *device = ctx->device;
  if (sm_count) *sm_count = ctx->sms;
  return MF_OK;
}

mf_status mf_load_sdnet(mf_ctx* ctx, const mf_sdnet_desc* desc, const float* w, mf_sdnet** out) {
  if (!desc) return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: null argument");
  const mf_sdnet_desc_ex ex{desc->width, desc->depth, MF_ACT_TANH, 0, 0};
  return mf_load_sdnet_ex(ctx, &ex, w, out);
}

mf_status mf_load_sdnet_ex(mf_ctx* ctx, const mf_sdnet_desc_ex* desc, const float* w, mf_sdnet** out) {
  if (!desc || !w || !out) return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: null argument");
  *out = nullptr;
  const int H = desc->width, D = desc->depth;
  if (H != 64 && H != 128) return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: width must be 64 or 128");
  if (D < 2 || D > 6) return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: depth must be in 2..6");
  if (desc->activation != MF_ACT_TANH && desc->activation != MF_ACT_GELU)
    return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: activation must be MF_ACT_TANH or MF_ACT_GELU");
  const int C = desc->embed_channels, K = desc->embed_kernel;
  if (C < 0 || C > mf::kMaxEmbedC) return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: embed_channels must be in 0..16");
  if (C > 0 && (K < 1 || K > mf::kMaxEmbedK || K % 2 == 0))
    return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: embed_kernel must be odd, 1..9");
  const int NH = D - 1;
  const int n_in = C > 0 ? C * 64 : 128;
  const size_t n_conv = C > 0 ? (size_t)C * K + C + (size_t)C * C * K + C : 0;
  const size_t n_all = n_conv + (size_t)H * (n_in + 2) + H + (size_t)NH * (H * H + H) + H + 1;
  for (size_t i = 0; i < n_all; ++i)
    if (!std::isfinite(w[i])) return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: non-finite weight");

  // unpack [conv1 W, b, conv2 W, b], W0[H][n_in+2], b0, {W[H][H], b}, w_out, b_out
  const float* p = w;
  const float* cw1 = p;  p += (size_t)C * K;
  const float* cb1 = p;  p += C;
  const float* cw2 = p;  p += (size_t)C * C * K;
  const float* cb2 = p;  p += C;
  const float* W0 = p;  p += (size_t)H * (n_in + 2);
  const float* b0 = p;  p += H;
  std::vector<float> W1t((size_t)n_in * H), W2((size_t)H * 2), WhT((size_t)NH * H * H), bh((size_t)NH * H);
  for (int j = 0; j < H; ++j) {
    for (int k = 0; k < n_in; ++k) W1t[(size_t)k * H + j] = W0[(size_t)j * (n_in + 2) + k];
    W2[2 * j] = W0[(size_t)j * (n_in + 2) + n_in];
    W2[2 * j + 1] = W0[(size_t)j * (n_in + 2) + n_in + 1];
  }
  std::vector<uint16_t> img((size_t)NH * H * H), img16((size_t)NH * H * H);
  bool f16s_ok = true;  // every hidden weight within the F16 range: the F16 sweep is offered
  for (int l = 0; l < NH; ++l) {
    const float* Wl = p;  p += (size_t)H * H;
    const float* bl = p;  p += H;
    for (int n = 0; n < H; ++n)
      for (int k = 0; k < H; ++k) WhT[(size_t)l * H * H + (size_t)k * H + n] = Wl[(size_t)n * H + k];
    std::memcpy(&bh[(size_t)l * H], bl, sizeof(float) * H);
    pack_sw128(Wl, H, &img[(size_t)l * H * H]);
    for (size_t i = 0; i < (size_t)H * H; ++i) f16s_ok = f16s_ok && std::fabs(Wl[i]) < 65504.0f;
    if (f16s_ok) pack_sw128(Wl, H, &img16[(size_t)l * H * H], true);
  }
  const float* wout = p;  p += H;
  const float bout = *p;

  if (!ctx) return fail(MF_ERR_INVALID_ARG, "mf_load_sdnet: null context");
  MF_ON_DEVICE(ctx->device, "mf_load_sdnet: cudaSetDevice");
  mf_sdnet* net = new mf_sdnet();
  net->device = ctx->device;
  // one allocation: W1t | W2 | b0 | WhT | bh | wout | BF16 images | conv | F16 split images |
  // F16 images (each 256-byte aligned)
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t sz_W1t = up(W1t.size() * 4), sz_W2 = up(W2.size() * 4), sz_b0 = up((size_t)H * 4),
               sz_WhT = up(WhT.size() * 4), sz_bh = up(bh.size() * 4), sz_wout = up((size_t)H * 4),
               sz_img = up(img.size() * 2), sz_conv = up(n_conv * 4 + 4);
  // F16 hi/lo images for the FP32 tensor-core kernel: width 128, and every hidden
  // weight within the F16 range (else that kernel is not offered for this SDNet)
  bool f16_ok = H == 128;
  for (size_t i = 0; f16_ok && i < WhT.size(); ++i) f16_ok = std::fabs(WhT[i]) < 65504.0f;
  const size_t sz_f16 = f16_ok ? up(mf::f32tc_image_bytes(NH)) : 0;
  const size_t sz_img16 = f16s_ok ? sz_img : 0;
  const size_t total = sz_W1t + sz_W2 + sz_b0 + sz_WhT + sz_bh + sz_wout + sz_img + sz_conv + sz_f16 + sz_img16;
  cudaError_t e = cudaMalloc(&net->dmem, total);
  if (e != cudaSuccess) {
    delete net;
    return cuda_fail(e, "mf_load_sdnet: cudaMalloc");
  }
  char* base = static_cast<char*>(net->dmem);
  size_t o = 0;
  auto place = [&](const void* src, size_t bytes, size_t slot) -> void* {
    void* dst = base + o;
    o += slot;
    if (bytes && cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    return dst;
  };
  net->d.W1t = (const float*)place(W1t.data(), W1t.size() * 4, sz_W1t);
  net->d.W2 = (const float*)place(W2.data(), W2.size() * 4, sz_W2);
  net->d.b0 = (const float*)place(b0, (size_t)H * 4, sz_b0);
  net->d.WhT = (const float*)place(WhT.data(), WhT.size() * 4, sz_WhT);
  net->d.bh = (const float*)place(bh.data(), bh.size() * 4, sz_bh);
  net->d.wout = (const float*)place(wout, (size_t)H * 4, sz_wout);
  net->d.wimg_bf16 = place(img.data(), img.size() * 2, sz_img);
  const float* conv = (const float*)place(w, n_conv * 4, sz_conv);  // cw1 | cb1 | cw2 | cb2, as packed
  void* f16img = f16_ok ? place(nullptr, 0, sz_f16) : nullptr;
  const void* img16_d = f16s_ok ? place(img16.data(), img16.size() * 2, sz_img16) : nullptr;
  if (!net->d.W1t || !net->d.W2 || !net->d.b0 || !net->d.WhT || !net->d.bh || !net->d.wout || !net->d.wimg_bf16 ||
      !conv || (f16s_ok && !img16_d)) {
    cudaError_t err = cudaGetLastError();
    cudaFree(net->dmem);
    delete net;
    return cuda_fail(err == cudaSuccess ? cudaErrorUnknown : err, "mf_load_sdnet: upload");
  }
  net->d.width = H;
  net->d.depth = D;
  net->d.n_hidden = NH;
  net->d.act = desc->activation == MF_ACT_GELU ? mf::kActGelu : mf::kActTanh;
  net->d.embed_c = C;
  net->d.embed_k = C > 0 ? K : 0;
  net->d.n_in = n_in;
  net->d.cw1 = C > 0 ? conv + (cw1 - w) : nullptr;
  net->d.cb1 = C > 0 ? conv + (cb1 - w) : nullptr;
  net->d.cw2 = C > 0 ? conv + (cw2 - w) : nullptr;
  net->d.cb2 = C > 0 ? conv + (cb2 - w) : nullptr;
  net->d.bout = bout;
  net->d.wimg_bytes = img.size() * 2;
  net->d.wimg_f16 = nullptr;
  net->d.wimg_f16s = img16_d;
  if (f16img) {
    cudaError_t pe = mf::f32tc_pack(net->d.WhT, NH, f16img, nullptr);
    if (pe == cudaSuccess) pe = cudaDeviceSynchronize();
    if (pe != cudaSuccess) {
      cudaFree(net->dmem);
      delete net;
      return cuda_fail(pe, "mf_load_sdnet: F16 images");
    }
    net->d.wimg_f16 = f16img;
  }
  net->h_bh = bh;
  net->h_wout.assign(wout, wout + H);
  net->h_W2 = W2;
  net->d.h_bh = net->h_bh.data();
  net->d.h_wout = net->h_wout.data();
  net->d.h_W2 = net->h_W2.data();
  *out = net;
  return MF_OK;
}

mf_status mf_free_sdnet(mf_sdnet* net) {
  if (!net) return MF_OK;
  mf::DeviceGuard guard(net->device);
  cudaFree(net->dmem);
  delete net;
  return MF_OK;
}

mf_status mf_destroy_grid(mf_grid* g) {
  if (!g) return MF_OK;
  mf::DeviceGuard guard(g->device);
  cudaFree(g->u);
  cudaFree(g->prev);
  cudaFree(g->B);
  cudaFree(g->partial);
  cudaFree(g->out);
  cudaFree(g->status);
  cudaFree(g->sync);
  cudaFreeHost(g->h_out);
  cudaFreeHost(g->h_status);
  for (cudaEvent_t ev : g->events) cudaEventDestroy(ev);
  delete g;
  return MF_OK;
}

mf_status mf_create_grid(mf_ctx* ctx, const mf_grid_desc* desc, const double* bc, mf_grid** out) {
  if (!desc || !bc || !out) return fail(MF_ERR_INVALID_ARG, "mf_create_grid: null argument");
  *out = nullptr;
  if (desc->lx < 1 || desc->lx > 128 || desc->ly < 1 || desc->ly > 128)
    return fail(MF_ERR_INVALID_ARG, "mf_create_grid: lx and ly must be in 1..128");
  if (!ctx) return fail(MF_ERR_INVALID_ARG, "mf_create_grid: null context");
  MF_ON_DEVICE(ctx->device, "mf_create_grid: cudaSetDevice");
  mf_grid* g = new mf_grid();
  g->device = ctx->device;
  g->lx = desc->lx;
  g->ly = desc->ly;
  g->nx = mf::kPts * g->lx + 1;
  g->ny = mf::kPts * g->ly + 1;
  const size_t npts = (size_t)g->nx * g->ny;
  const size_t nbc = 2 * (size_t)(g->nx - 1) + 2 * (size_t)(g->ny - 1);
  const size_t max_colour = (size_t)g->lx * g->ly;  // colour (0,0) is the largest
  double* dbc = nullptr;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&g->u, npts * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&g->prev, npts * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&g->B, max_colour * 128 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&g->partial, mf::kReduceBlocks * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&g->out, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&g->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&g->sync, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMallocHost(&g->h_out, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&g->h_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&dbc, nbc * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(dbc, bc, nbc * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mf::launch_init_grid(g->u, g->nx, g->ny, dbc, nullptr);
  if (e == cudaSuccess) e = cudaMemset(g->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->out, 0, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (dbc) cudaFree(dbc);
  if (e != cudaSuccess) {
    mf_destroy_grid(g);
    return cuda_fail(e, "mf_create_grid");
  }
  *out = g;
  return MF_OK;
}

mf_status mf_grid_dims(const mf_grid* g, int* nx, int* ny) {
  if (!g) return fail(MF_ERR_INVALID_ARG, "mf_grid_dims: null grid");
  if (nx) *nx = g->nx;
  if (ny) *ny = g->ny;
  return MF_OK;
}

mf_status mf_grid_upload(mf_grid* g, const float* src, int on_device, void* stream) {
  if (!g || !src) return fail(MF_ERR_INVALID_ARG, "mf_grid_upload: null argument");
  MF_ON_DEVICE(g->device, "mf_grid_upload: cudaSetDevice");
  MF_CUDA(cudaMemcpyAsync(g->u, src, (size_t)g->nx * g->ny * sizeof(float),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, as_stream(stream)),
          "mf_grid_upload: cudaMemcpyAsync");
  return MF_OK;
}

mf_status mf_grid_download(const mf_grid* g, float* dst, int on_device, void* stream) {
  if (!g || !dst) return fail(MF_ERR_INVALID_ARG, "mf_grid_download: null argument");
  MF_ON_DEVICE(g->device, "mf_grid_download: cudaSetDevice");
  MF_CUDA(cudaMemcpyAsync(dst, g->u, (size_t)g->nx * g->ny * sizeof(float),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, as_stream(stream)),
          "mf_grid_download: cudaMemcpyAsync");
  return MF_OK;
}

}  // extern "C"

namespace {

mf_status sweep_impl(mf_grid* g, const mf_sdnet* net, const mf_sweep_opts* o, mf_sweep_result* res,
                     void* stream) {
  if (!g || !net || !o) return fail(MF_ERR_INVALID_ARG, "mf_sweep: null argument");
  if (o->n_sweeps < 0) return fail(MF_ERR_INVALID_ARG, "mf_sweep: n_sweeps < 0");
  if (o->schedule != MF_SCHEDULE_MULTIPLICATIVE && o->schedule != MF_SCHEDULE_ADDITIVE)
    return fail(MF_ERR_INVALID_ARG, "mf_sweep: unknown schedule");
  if (o->precision != MF_PREC_FP32 && o->precision != MF_PREC_BF16 && o->precision != MF_PREC_MIXED &&
      o->precision != MF_PREC_FP32_SIMT && o->precision != MF_PREC_F16)
    return fail(MF_ERR_INVALID_ARG, "mf_sweep: unknown precision");
  if (o->precision == MF_PREC_MIXED && !(o->eps_coarse > 0.0 && std::isfinite(o->eps_coarse)))
    return fail(MF_ERR_INVALID_ARG, "mf_sweep: MF_PREC_MIXED needs eps_coarse > 0");
  if (o->colours < 0 || o->colours > 15) return fail(MF_ERR_INVALID_ARG, "mf_sweep: colours must be a 4-bit mask");
  if (o->check_every < 1) return fail(MF_ERR_INVALID_ARG, "mf_sweep: check_every must be >= 1");
  if (o->query != MF_QUERY_FULL && o->query != MF_QUERY_CENTRE)
    return fail(MF_ERR_INVALID_ARG, "mf_sweep: unknown query");
  if (o->query == MF_QUERY_CENTRE && o->schedule == MF_SCHEDULE_ADDITIVE)
    return fail(MF_ERR_INVALID_ARG, "mf_sweep: centre-line sweeps use the multiplicative schedule");
  if (!std::isfinite(o->eps)) return fail(MF_ERR_INVALID_ARG, "mf_sweep: eps must be finite");
  if ((o->precision == MF_PREC_BF16 || o->precision == MF_PREC_MIXED) && !mf::bf16_supported(net->d))
    return fail(MF_ERR_UNSUPPORTED, "mf_sweep: BF16 path needs 1..5 hidden layers");
  if (o->precision == MF_PREC_F16 && !mf::f16_supported(net->d))
    return fail(MF_ERR_UNSUPPORTED, "mf_sweep: F16 path needs 1..5 hidden layers and weights within the F16 range");
  if (o->launch_mode != MF_LAUNCH_PER_COLOUR && o->launch_mode != MF_LAUNCH_SWEEP)
    return fail(MF_ERR_INVALID_ARG, "mf_sweep: launch_mode must be MF_LAUNCH_PER_COLOUR or MF_LAUNCH_SWEEP");
  const bool sweep_launch = o->launch_mode == MF_LAUNCH_SWEEP;
  if (sweep_launch && (o->schedule != MF_SCHEDULE_MULTIPLICATIVE || (o->colours != 0 && o->colours != 15) ||
                       o->precision == MF_PREC_FP32 || o->precision == MF_PREC_FP32_SIMT ||
                       o->precision == MF_PREC_F16 || !mf::bf16_sweep_supported(net->d)))
    return fail(MF_ERR_UNSUPPORTED, "mf_sweep: MF_LAUNCH_SWEEP runs BF16 multiplicative sweeps of all colours "
                                    "with an SDNet without a boundary embedding");
  if (net->device != g->device) return fail(MF_ERR_INVALID_ARG, "mf_sweep: grid and SDNet on different devices");
  if (res) *res = mf_sweep_result{0, -1.0, 0, 0, 0.0, 0.0, 0.0, 0, 0, MF_OK, o->launch_mode, 16};
  MF_ON_DEVICE(g->device, "mf_sweep: cudaSetDevice");
  cudaStream_t st = as_stream(stream);
  const int mask = o->colours == 0 ? 15 : o->colours;
  const bool additive = o->schedule == MF_SCHEDULE_ADDITIVE;
  const size_t bytes = (size_t)g->nx * g->ny * sizeof(float);
  PhaseTimer pt{g, st, o->profile != 0};
  int launches = 0, mlp_launches = 0;
  MF_CUDA(cudaMemsetAsync(g->status, 0, sizeof(int), st), "mf_sweep: reset status");
  MF_CUDA(pt.mark(kPhaseReduce), "mf_sweep: event");

  int done = 0, done_bf16 = 0;
  bool checked = false;
  const bool mixed = o->precision == MF_PREC_MIXED;
  bool coarse = mixed;  // mixed precision: still in the BF16 phase
  double d_prev = INFINITY;  // delta of the previous BF16 sweep
  for (int k = 0; k < o->n_sweeps; ++k) {
    const bool check = coarse || ((k + 1) % o->check_every == 0) || (k + 1 == o->n_sweeps);
    const bool bf16 = mixed ? coarse : (o->precision == MF_PREC_BF16);
    const bool f16 = o->precision == MF_PREC_F16;
    if (check || additive)
      MF_CUDA(cudaMemcpyAsync(g->prev, g->u, bytes, cudaMemcpyDeviceToDevice, st), "mf_sweep: snapshot");
    if (additive) {
      MF_CUDA(mf::launch_zero_interior(g->u, g->nx, g->ny, st), "mf_sweep: zero interior");
      ++launches;
    }
    MF_CUDA(pt.mark(kPhaseReduce), "mf_sweep: event");
    if (bf16 && sweep_launch) {
      // the whole sweep in one cooperative launch (gathers included)
      mf::ColourGeom gc[4];
      int n_col = 0;
      for (int c = 0; c < 4; ++c) {
        mf::ColourGeom cg = colour_geom(g, c);
        if (cg.n_c == 0) continue;
        if (o->query == MF_QUERY_CENTRE) {
          cg.centre = 1;
          cg.rows_per_sub = mf::kNcross;
        }
        gc[n_col++] = cg;
      }
      MF_CUDA(mf::launch_mlp_bf16_sweep(gc, n_col, net->d, g->u, g->B, g->sync, g->status, st),
              "mf_sweep: whole-sweep launch");
      MF_CUDA(pt.mark(kPhaseMlp), "mf_sweep: event");
      launches += 1;
      mlp_launches += 1;
    }
    for (int c = 0; c < 4 && !(bf16 && sweep_launch); ++c) {
      if (!((mask >> c) & 1)) continue;
      mf::ColourGeom cg = colour_geom(g, c);
      if (cg.n_c == 0) continue;
      if (o->query == MF_QUERY_CENTRE) {
        cg.centre = 1;
        cg.rows_per_sub = mf::kNcross;
      }
      MF_CUDA(mf::launch_gather_boundary(additive ? g->prev : g->u, cg, net->d, g->B, st), "mf_sweep: gather");
      MF_CUDA(pt.mark(kPhaseGather), "mf_sweep: event");
      if (bf16)
        MF_CUDA(mf::launch_mlp_bf16(g->B, cg, net->d, g->u, additive ? 1 : 0, g->status, st), "mf_sweep: bf16 mlp");
      else if (f16)
        MF_CUDA(mf::launch_mlp_bf16(g->B, cg, net->d, g->u, additive ? 1 : 0, g->status, st, true),
                "mf_sweep: f16 mlp");
      else
        MF_CUDA(mf::launch_mlp_fp32_path(g->B, cg, net->d, g->u, additive ? 1 : 0, g->status,
                                         o->precision == MF_PREC_FP32_SIMT, st),
                "mf_sweep: fp32 mlp");
      MF_CUDA(pt.mark(kPhaseMlp), "mf_sweep: event");
      launches += 2;
      mlp_launches += 1;
    }
    done = k + 1;
    if (bf16) done_bf16 = k + 1;
    if (check) {
      MF_CUDA(mf::launch_reduce(g->u, g->prev, g->nx, g->ny, g->partial, g->out, st), "mf_sweep: reduce");
      MF_CUDA(pt.mark(kPhaseReduce), "mf_sweep: event");
      launches += 2;
      checked = true;
      if (o->eps > 0.0 || coarse) {
        MF_CUDA(cudaMemcpyAsync(g->h_out, g->out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "mf_sweep: read delta");
        MF_CUDA(cudaMemcpyAsync(g->h_status, g->status, sizeof(int), cudaMemcpyDeviceToHost, st), "mf_sweep: read status");
        MF_CUDA(cudaStreamSynchronize(st), "mf_sweep: synchronize");
        if (*g->h_status != mf::kDevErrNone) return fail(MF_ERR_TIMEOUT, "mf_sweep: a kernel wait timed out");
        const double d = g->h_out[4];
        if (res) { res->sweeps_done = done; res->delta = d; res->sweeps_bf16 = done_bf16; }
        if (!std::isfinite(d)) return fail(MF_ERR_DIVERGED, "mf_sweep: delta is not finite");
        if (coarse) {
          // switch to FP32 refinement once delta is small enough, or once a BF16 sweep
          // no longer reduces it (the BF16 iteration has reached its rounding floor)
          if (d < o->eps_coarse || d >= d_prev) coarse = false;
          d_prev = d;
        } else if (d < o->eps) {
          break;
        }
      }
    }
  }
  MF_CUDA(cudaMemcpyAsync(g->h_out, g->out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "mf_sweep: read delta");
  MF_CUDA(cudaMemcpyAsync(g->h_status, g->status, sizeof(int), cudaMemcpyDeviceToHost, st), "mf_sweep: read status");
  MF_CUDA(cudaStreamSynchronize(st), "mf_sweep: synchronize");
  if (*g->h_status != mf::kDevErrNone) return fail(MF_ERR_TIMEOUT, "mf_sweep: a kernel wait timed out");
  double ms[3];
  MF_CUDA(pt.totals(ms), "mf_sweep: event timing");
  if (res) {
    res->sweeps_done = done;
    res->delta = checked ? g->h_out[4] : -1.0;
    res->kernel_launches = launches;
    res->mlp_launches = mlp_launches;
    res->ms_gather = ms[kPhaseGather];
    res->ms_mlp = ms[kPhaseMlp];
    res->ms_reduce = ms[kPhaseReduce];
    res->sweeps_bf16 = done_bf16;
  }
  if (checked && !std::isfinite(g->h_out[4])) return fail(MF_ERR_DIVERGED, "mf_sweep: delta is not finite");
  return MF_OK;
}

}  // namespace

extern "C" {

mf_status mf_sweep(mf_grid* g, const mf_sdnet* net, const mf_sweep_opts* o, mf_sweep_result* res,
                   void* stream) {
  const mf_status st = sweep_impl(g, net, o, res, stream);
  if (res) res->status = st;
  return st;
}

mf_status mf_synchronize(void* stream) {
  MF_CUDA(cudaStreamSynchronize(as_stream(stream)), "mf_synchronize");
  return MF_OK;
}

mf_status mf_residual(const mf_grid* g, double* max_abs, double* rms, void* stream) {
  if (!g) return fail(MF_ERR_INVALID_ARG, "mf_residual: null grid");
  MF_ON_DEVICE(g->device, "mf_residual: cudaSetDevice");
  cudaStream_t st = as_stream(stream);
  MF_CUDA(mf::launch_reduce(g->u, nullptr, g->nx, g->ny, g->partial, g->out + 8, st), "mf_residual: reduce");
  MF_CUDA(cudaMemcpyAsync(g->h_out + 8, g->out + 8, 5 * sizeof(double), cudaMemcpyDeviceToHost, st),
          "mf_residual: read");
  MF_CUDA(cudaStreamSynchronize(st), "mf_residual: synchronize");
  const double n_int = (double)(g->nx - 2) * (double)(g->ny - 2);
  if (max_abs) *max_abs = g->h_out[10];
  if (rms) *rms = std::sqrt(g->h_out[11] / n_int);
  return MF_OK;
}

}  // extern "C"
