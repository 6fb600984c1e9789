// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

// An execution context (the ABI's mf_ctx): one CUDA device and what the library knows
// about it. Handles created under it copy the device index and keep no pointer to it.
struct mf_ctx {
  int device = 0;
  int sms = 0;
};

namespace mf {

// ---- devices ----------------------------------------------------------------------
// Handles record the device they were created on; every call that works on a handle
// makes that device current for its duration and gives the caller's selection back.
constexpr int kMaxDevices = 64;

struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int device) {
    err = cudaGetDevice(&prev);
    if (err != cudaSuccess) {
      prev = -1;
      return;
    }
    if (prev != device) err = cudaSetDevice(device);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// One-time launch set-up per device. A cudaFuncSetAttribute call, an occupancy query
// and the SM count all belong to the device that is current when they run, so each
// launcher keeps one record per device, filled under a lock the first time that
// device launches it.
struct PerDevice {
  std::mutex lock;
  bool ready[kMaxDevices] = {};
  int ival[kMaxDevices] = {};
  size_t zval[kMaxDevices] = {};
};

inline cudaError_t current_device(int* dev) {
  const cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return e;
  return (*dev < 0 || *dev >= kMaxDevices) ? cudaErrorInvalidDevice : cudaSuccess;
}

// Runs init(device, ival, zval) once per device for the record `pd`; returns its
// error, and the stored values through ival/zval.
template <class F>
cudaError_t per_device(PerDevice& pd, F&& init, int* ival = nullptr, size_t* zval = nullptr) {
  int dev = 0;
  cudaError_t e = current_device(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(pd.lock);
  if (!pd.ready[dev]) {
    int iv = 0;
    size_t zv = 0;
    e = init(dev, &iv, &zv);
    if (e != cudaSuccess) return e;
    pd.ival[dev] = iv;
    pd.zval[dev] = zv;
    pd.ready[dev] = true;
  }
  if (ival) *ival = pd.ival[dev];
  if (zval) *zval = pd.zval[dev];
  return cudaSuccess;
}

// SM count of the current device (cached per device).
inline cudaError_t device_sms(int* sms) {
  static PerDevice pd;
  return per_device(pd, [](int dev, int* iv, size_t*) {
    return cudaDeviceGetAttribute(iv, cudaDevAttrMultiProcessorCount, dev);
  }, sms);
}

// Geometry of the unit subdomain: 32 intervals per side, lattice spacing 16 points.
constexpr int kPts = 32;        // intervals per unit length
constexpr int kHalf = 16;       // spacing of subdomain origins (1/2 unit)
constexpr int kNi = 31;         // interior points per side
constexpr int kNint = 961;      // interior points per subdomain
constexpr int kNbdry = 128;     // boundary values per subdomain
constexpr int kTileRows = 128;  // rows (subdomain, point) per MLP tile

// Activations of the SDNet layers.
constexpr int kActTanh = 0;
constexpr int kActGelu = 1;
constexpr int kMaxEmbedC = 16;  // boundary-embedding channels
constexpr int kMaxEmbedK = 9;   // boundary-embedding kernel size (odd)

// Activation in FP32 with CUDA's accurate functions: tanh, or GELU x Phi(x) =
// x (1 + erf(x / sqrt 2)) / 2 (the FP32 kernels, and the boundary embedding).
template <int ACT>
__device__ __forceinline__ float act_exact(float x) {
  if constexpr (ACT == kActTanh) return tanhf(x);
  else return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

// Device error codes written to the status word by kernels whose bounded waits give up.
constexpr int kDevErrNone = 0;
constexpr int kDevErrTimeout = 1;

// A subdomain of a batch of problems: where its corner (local (0,0)) sits in the
// batch's grid buffer and the row stride of its problem's grid.
struct SubRef {
  unsigned long long origin;
  int nx;
  int pad;
};

// One colour of one problem (or of a batch of problems, through `table`), as seen by
// the kernels.
struct ColourGeom {
  int nx;           // grid row length (points)
  int ca, cb;       // colour parity in x and y
  int n_a;          // subdomains of this colour along x
  int n_c;          // subdomains of this colour
  int nsx, nsy;     // subdomains along x and y (all colours)
  int centre;       // 1: predict only each subdomain's centre cross (61 points)
  int rows_per_sub; // kNint (961) or kNcross (61)
  const SubRef* table; // batch: the colour's subdomains (then ca, cb, n_a, nsx, nsy unused)
};

// Grid offset of local point (i, j) of colour-local subdomain s.
__device__ __forceinline__ size_t sub_point(const ColourGeom& g, int s, int i, int j) {
  if (g.table) {
    const SubRef r = g.table[s];
    return (size_t)r.origin + (size_t)j * (size_t)r.nx + (size_t)i;
  }
  const int a = g.ca + 2 * (s % g.n_a);
  const int b = g.cb + 2 * (s / g.n_a);
  return (size_t)(kHalf * b + j) * (size_t)g.nx + (size_t)(kHalf * a + i);
}
__device__ __forceinline__ size_t sub_stride(const ColourGeom& g, int s) {
  return g.table ? (size_t)g.table[s].nx : (size_t)g.nx;
}
constexpr int kNcross = 61;  // centre row (31 points) + centre column without its middle (30)

// SDNet weights resident on the device (plus host copies of the small vectors that
// the tensor-core kernel takes as launch parameters).
struct DevNet {
  int width, depth;      // H and number of activation layers
  int n_hidden;          // depth - 1 hidden H x H layers
  int act;               // kActTanh or kActGelu (first and hidden layers)
  int embed_c, embed_k;  // boundary embedding: channels C (0 = none) and kernel size K
  int n_in;              // boundary input width of the first layer: 128, or C x 64
  const float* cw1;      // [C][K] first conv1d layer (1 -> C), stride 1
  const float* cb1;      // [C]
  const float* cw2;      // [C][C][K] second conv1d layer (C -> C), stride 2
  const float* cb2;      // [C]
  const float* W1t;      // [n_in][H] boundary block of W0, transposed (k-major)
  const float* W2;       // [H][2] coordinate block of W0
  const float* b0;       // [H]
  const float* WhT;      // [n_hidden][H(k)][H(n)] hidden weights, transposed (k-major)
  const float* bh;       // [n_hidden][H]
  const float* wout;     // [H]
  float bout;
  const void* wimg_bf16; // [n_hidden] BF16 images in the tensor-core shared-memory layout
  size_t wimg_bytes;     // bytes of all images
  const void* wimg_f16;  // [n_hidden][hi, lo] F16 split images (width 128), or null
  const void* wimg_f16s; // [n_hidden] F16 images (the F16 sweep's B operands), or null
  const float* h_bh;     // host copies: hidden biases [n_hidden][H]
  const float* h_wout;   // [H]
  const float* h_W2;     // [H][2]
};

// K1: gather the boundary of every subdomain of the colour from `u` and form the
// per-subdomain first-layer term B[s][:] = W1 z_s + b0 (Eq. 8, left operand), with z_s
// the boundary g_s itself or, for the embedding variant, its conv1d embedding.
// subs_per_block: subdomains per block of the plain gather (4, 8 or 16).
cudaError_t launch_gather_boundary(const float* u, const ColourGeom& g, const DevNet& net,
                                   float* B, cudaStream_t st, int subs_per_block = 16);

// K3f: FP32 SDNet on every interior point of every subdomain of the colour, fused with
// the scatter into `u` (store, or weighted add for the additive schedule).
cudaError_t launch_mlp_fp32(const float* B, const ColourGeom& g, const DevNet& net,
                            float* u, int additive, cudaStream_t st);

// K3: BF16 tcgen05 SDNet with TMEM accumulators, same contract as launch_mlp_fp32;
// f16: F16 operands and activations instead (needs the F16 weight images).
cudaError_t launch_mlp_bf16(const float* B, const ColourGeom& g, const DevNet& net,
                            float* u, int additive, int* dev_status, cudaStream_t st, bool f16 = false);
bool bf16_supported(const DevNet& net);
bool f16_supported(const DevNet& net);

// K3t: the FP32 SDNet on the tensor cores, each hidden product split in three F16
// products with FP32 accumulation (width 128, tanh or GELU); same contract as
// launch_mlp_fp32.
cudaError_t launch_mlp_f32tc(const float* B, const ColourGeom& g, const DevNet& net, float* u, int additive,
                             int* dev_status, cudaStream_t st);
bool f32tc_supported(const DevNet& net);
size_t f32tc_image_bytes(int n_hidden);
// hi/lo F16 images of the hidden weights (WhT: [n_hidden][k][n] FP32) into img
cudaError_t f32tc_pack(const float* WhT, int n_hidden, void* img, cudaStream_t st);

// The FP32-accuracy SDNet launch of a sweep: the tensor-core kernel where the SDNet
// allows it and simt is false, else the SIMT kernel.
inline cudaError_t launch_mlp_fp32_path(const float* B, const ColourGeom& g, const DevNet& net, float* u,
                                        int additive, int* dev_status, bool simt, cudaStream_t st) {
  if (!simt && f32tc_supported(net)) return launch_mlp_f32tc(B, g, net, u, additive, dev_status, st);
  return launch_mlp_fp32(B, g, net, u, additive, st);
}

// K3 over a whole multiplicative sweep in one cooperative launch: for each of the n_col
// colour passes gc[0..n_col-1] in order, the boundary gather and B = W1 g + b0 (into B,
// which must hold the largest pass's n_c x H floats), then the SDNet with the scatter
// into `u`, with device-wide barriers between the steps (`sync`: one word of device
// memory, zeroed by the call before the launch). The multiplicative schedule only; not
// for SDNets with a boundary embedding.
cudaError_t launch_mlp_bf16_sweep(const ColourGeom* gc, int n_col, const DevNet& net, float* u, float* B,
                                  unsigned int* sync, int* dev_status, cudaStream_t st);
bool bf16_sweep_supported(const DevNet& net);

// K5: FP64 reductions over the grid. partial must hold kReduceBlocks * 4 doubles and
// out 5 doubles: {sum (u-prev)^2, sum prev^2, max |r|, sum r^2, delta}.
constexpr int kReduceBlocks = 512;
cudaError_t launch_reduce(const float* u, const float* prev, int nx, int ny, double* partial,
                          double* out, cudaStream_t st, bool residual = true);

// K0 grid set-up: boundary from the FP64 counter-clockwise list `bc` (device), interior 0.
cudaError_t launch_init_grid(float* u, int nx, int ny, const double* bc, cudaStream_t st);
cudaError_t launch_zero_interior(float* u, int nx, int ny, cudaStream_t st);

}  // namespace mf

namespace mf {

// Row r of a colour's batch is point p = r mod R of subdomain s = r / R (colour-local
// index, row-major over the colour's subdomains), R = 961 interior points, or R = 61
// centre-cross points (p < 31: centre row px = p; else the centre column, py = 0..30
// without 15) when only the interfaces are predicted.
struct RowSite {
  int s;      // colour-local subdomain index
  size_t idx; // grid offset of the point
  int px, py; // local interior indices 0..30
  int ix, iy; // global grid indices
};

__device__ __forceinline__ RowSite row_site(const ColourGeom& g, int row) {
  RowSite r;
  r.s = row / g.rows_per_sub;
  const int p = row - r.s * g.rows_per_sub;
  if (g.centre) {
    const int mid = kNi / 2;  // 15
    const int q = p - kNi;
    r.px = p < kNi ? p : mid;
    r.py = p < kNi ? mid : (q < mid ? q : q + 1);
  } else {
    r.py = p / kNi;
    r.px = p - r.py * kNi;
  }
  if (g.table) {
    const SubRef t = g.table[r.s];
    r.ix = r.iy = 0;  // (only the additive schedule needs them; batches are multiplicative)
    r.idx = (size_t)t.origin + (size_t)(1 + r.py) * (size_t)t.nx + (size_t)(1 + r.px);
    return r;
  }
  const int a = g.ca + 2 * (r.s % g.n_a);
  const int b = g.cb + 2 * (r.s / g.n_a);
  r.ix = kHalf * a + 1 + r.px;
  r.iy = kHalf * b + 1 + r.py;
  r.idx = (size_t)r.iy * (size_t)g.nx + (size_t)r.ix;
  return r;
}

// Number of subdomains along one axis whose open interior holds grid coordinate i.
__device__ __forceinline__ int axis_cover(int i, int n_sub) {
  int c = 0;
  const int a1 = (i - 1) / kHalf;  // largest origin index with 16a < i
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const int a = a1 - d;
    if (a >= 0 && a < n_sub && kHalf * a < i && i < kHalf * a + kPts) ++c;
  }
  return c;
}

// Additive schedule: weight 1/cover of the point (exact in FP32: 1, 1/2 or 1/4).
__device__ __forceinline__ float cover_weight(const ColourGeom& g, int ix, int iy) {
  return 1.0f / (float)(axis_cover(ix, g.nsx) * axis_cover(iy, g.nsy));
}

}  // namespace mf
