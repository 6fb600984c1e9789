// mf_sweep_noalloc: the multiplicative sweep for callers that must not allocate device
// memory during the call.
//
// Who needs it: code that runs inside a host framework whose caching allocator owns
// the device memory budget (a stray cudaMalloc there can fail once the pool has taken
// the memory, or fragment it), and latency-critical loops where a cudaMalloc/cudaFree
// pair would implicitly synchronise the device in the middle of a stream of work. Such
// a caller owns the grid buffer itself and only needs the library not to allocate.
//
// How: all scratch of the sweep (the per-subdomain first-layer table, the snapshot of
// the grid used for delta, the reduction partials and the kernel status word) lives in
// one file-scope __device__ array of fixed size, so every GPU that loads this library
// holds about 4.7 MB for it until the process exits. The existing kernels run on
// pointers into that array; nothing here calls cudaMalloc, cudaFree or any allocating
// library routine.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mosaicflow.h"
#include "mf_internal.cuh"

namespace mf {
// Defined in mf_api.cu: the device-side view of a loaded SDNet and its device.
const DevNet* devnet_of(const mf_sdnet* net, int* device);
void set_last_error(const std::string& msg);
}  // namespace mf

namespace {

constexpr int kMaxSide = 32;                                   // lx, ly <= 32 units
constexpr size_t kMaxPoints = (size_t)(32 * kMaxSide + 1) * (32 * kMaxSide + 1);
constexpr size_t kMaxColour = (size_t)kMaxSide * kMaxSide;     // subdomains in the largest colour
constexpr size_t kAlign = 256;
constexpr size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffB = 0;                                                   // float [kMaxColour][128]
constexpr size_t kOffPrev = kOffB + up(kMaxColour * 128 * sizeof(float));     // float [kMaxPoints]
constexpr size_t kOffPartial = kOffPrev + up(kMaxPoints * sizeof(float));     // double [kReduceBlocks][4]
constexpr size_t kOffOut = kOffPartial + up((size_t)mf::kReduceBlocks * 4 * sizeof(double));  // double [16]
constexpr size_t kOffStatus = kOffOut + up(16 * sizeof(double));              // int
constexpr size_t kScratchBytes = kOffStatus + up(sizeof(int));

// The scratch itself. Host code must not take its address with & (that is a host-side
// stand-in); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
cudaError_t scratch_on(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[device]);
  return cudaSuccess;
}

mf::ColourGeom geom(int lx, int ly, int c) {
  mf::ColourGeom g{};
  g.nx = 32 * lx + 1;
  g.ca = c & 1;
  g.cb = c >> 1;
  g.nsx = 2 * lx - 1;
  g.nsy = 2 * ly - 1;
  g.n_a = (g.nsx - g.ca + 1) / 2;
  g.n_c = g.n_a * ((g.nsy - g.cb + 1) / 2);
  g.centre = 0;
  g.rows_per_sub = mf::kNint;
  g.table = nullptr;
  return g;
}

mf_status fail(mf_status code, const std::string& msg) {
  mf::set_last_error(msg);
  return code;
}

mf_status cuda_fail(cudaError_t e, const char* what) {
  return fail(MF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define NA_CUDA(call, what)                              \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
  } while (0)

}  // namespace

extern "C" mf_status mf_sweep_noalloc(float* u, int lx, int ly, const mf_sdnet* net, int precision, int n_sweeps,
                                      double* delta, void* stream) {
  if (!u || !net) return fail(MF_ERR_INVALID_ARG, "mf_sweep_noalloc: null grid or SDNet");
  if (lx < 1 || ly < 1 || lx > kMaxSide || ly > kMaxSide)
    return fail(MF_ERR_INVALID_ARG, "mf_sweep_noalloc: lx and ly must be in 1..32 (the static scratch is sized "
                                    "for domains up to 32 x 32 units); use mf_sweep for larger grids");
  if (n_sweeps < 0) return fail(MF_ERR_INVALID_ARG, "mf_sweep_noalloc: n_sweeps < 0");
  if (precision != MF_PREC_FP32 && precision != MF_PREC_BF16)
    return fail(MF_ERR_INVALID_ARG, "mf_sweep_noalloc: unknown precision");
  int net_device = 0;
  const mf::DevNet* d = mf::devnet_of(net, &net_device);
  if (precision == MF_PREC_BF16 && !mf::bf16_supported(*d))
    return fail(MF_ERR_UNSUPPORTED, "mf_sweep_noalloc: BF16 path needs 1..5 hidden layers");
  int device = 0;
  NA_CUDA(cudaGetDevice(&device), "mf_sweep_noalloc: cudaGetDevice");
  if (device != net_device) return fail(MF_ERR_INVALID_ARG, "mf_sweep_noalloc: SDNet was loaded on another device");
  if (device < 0 || device >= kMaxDevices) return fail(MF_ERR_UNSUPPORTED, "mf_sweep_noalloc: device index too large");
  if (delta) *delta = -1.0;

  unsigned char* base = nullptr;
  NA_CUDA(scratch_on(device, &base), "mf_sweep_noalloc: cudaGetSymbolAddress");
  float* B = reinterpret_cast<float*>(base + kOffB);
  float* prev = reinterpret_cast<float*>(base + kOffPrev);
  double* partial = reinterpret_cast<double*>(base + kOffPartial);
  double* out = reinterpret_cast<double*>(base + kOffOut);
  int* status = reinterpret_cast<int*>(base + kOffStatus);

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nx = 32 * lx + 1, ny = 32 * ly + 1;
  // the status word keeps the previous call's value: it must start at zero
  NA_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st), "mf_sweep_noalloc: clear status");
  for (int k = 0; k < n_sweeps; ++k) {
    if (k + 1 == n_sweeps)
      NA_CUDA(cudaMemcpyAsync(prev, u, (size_t)nx * ny * sizeof(float), cudaMemcpyDeviceToDevice, st),
              "mf_sweep_noalloc: snapshot");
    for (int c = 0; c < 4; ++c) {
      const mf::ColourGeom g = geom(lx, ly, c);
      if (g.n_c == 0) continue;
      NA_CUDA(mf::launch_gather_boundary(u, g, *d, B, st), "mf_sweep_noalloc: gather");
      if (precision == MF_PREC_BF16)
        NA_CUDA(mf::launch_mlp_bf16(B, g, *d, u, 0, status, st), "mf_sweep_noalloc: bf16 mlp");
      else
        NA_CUDA(mf::launch_mlp_fp32(B, g, *d, u, 0, st), "mf_sweep_noalloc: fp32 mlp");
    }
  }
  double h_out[5] = {0, 0, 0, 0, 0};
  int h_status = 0;
  if (n_sweeps > 0) {
    NA_CUDA(mf::launch_reduce(u, prev, nx, ny, partial, out, st), "mf_sweep_noalloc: reduce");
    NA_CUDA(cudaMemcpyAsync(h_out, out, sizeof(h_out), cudaMemcpyDeviceToHost, st), "mf_sweep_noalloc: read delta");
  }
  NA_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st), "mf_sweep_noalloc: read status");
  NA_CUDA(cudaStreamSynchronize(st), "mf_sweep_noalloc: synchronize");
  if (h_status != mf::kDevErrNone) return fail(MF_ERR_TIMEOUT, "mf_sweep_noalloc: a kernel wait timed out");
  if (n_sweeps > 0) {
    if (delta) *delta = h_out[4];
    if (!std::isfinite(h_out[4])) return fail(MF_ERR_DIVERGED, "mf_sweep_noalloc: delta is not finite");
  }
  return MF_OK;
}
