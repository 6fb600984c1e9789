// Batches of independent Mosaic Flow problems of different sizes.
//
// All grids of a batch live in one device buffer, problem after problem. For each
// colour a table lists every subdomain of that colour across the batch (its corner's
// offset in the buffer and its problem's row stride), so one gather launch and one
// SDNet launch per colour serve the whole batch, however uneven the problems are: the
// kernels flatten (subdomain, point) rows across problems exactly as they do within one
// problem (Section 4.1 batches a problem's atomic subdomains; here the batch also spans
// problems). A sweep is launched in one of three ways: per colour one gather launch and
// one SDNet launch; the same launches replayed from a CUDA graph (sweeps without a
// convergence check); or one cooperative launch per sweep that gathers, evaluates and
// scatters every colour with device-wide barriers between them (BF16). An autotuner
// times these modes and the gather block size on a scratch copy of the batch and keeps
// the fastest per SDNet, precision and query.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mosaicflow.h"
#include "mf_internal.cuh"

namespace mf {
const DevNet* devnet_of(const mf_sdnet* net, int* device);
void set_last_error(const std::string& msg);
}  // namespace mf

struct mf_batch {
  int device = 0;
  int n = 0;
  std::vector<int> lx, ly, nx, ny;
  std::vector<size_t> offset;  // float offset of each problem's grid
  size_t total = 0;            // floats, padded to a multiple of kRow
  float* u = nullptr;
  float* prev = nullptr;
  mf::SubRef* table[4] = {nullptr, nullptr, nullptr, nullptr};
  int n_c[4] = {0, 0, 0, 0};
  float* B = nullptr;
  double* partial = nullptr;
  double* out = nullptr;
  int* status = nullptr;
  double* h_out = nullptr;
  int* h_status = nullptr;
  unsigned int* sync = nullptr;  // barrier counter of the whole-sweep launch
  // captured sweep
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  const mf_sdnet* g_net = nullptr;
  int g_prec = -1, g_query = -1, g_gather = -1;
  bool warmed = false;
  // autotuner choices: (SDNet, precision, query) -> (launch mode, gather block)
  struct Choice {
    const mf_sdnet* net;
    int prec, query, mode, gather;
  };
  std::vector<Choice> tuned;
};

namespace {

constexpr size_t kRow = 4096;  // the buffer is viewed as rows of this length for delta

mf_status fail(mf_status code, const std::string& msg) {
  mf::set_last_error(msg);
  return code;
}
mf_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? MF_ERR_OUT_OF_MEMORY : MF_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}
#define BT_CUDA(call, what)                            \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)
#define BT_ON_DEVICE(dev, what)   \
  mf::DeviceGuard guard_((dev));  \
  if (guard_.err != cudaSuccess) return cuda_fail(guard_.err, what)

mf::ColourGeom batch_geom(const mf_batch* b, int c, int query) {
  mf::ColourGeom g{};
  g.n_c = b->n_c[c];
  g.table = b->table[c];
  g.centre = query == MF_QUERY_CENTRE ? 1 : 0;
  g.rows_per_sub = g.centre ? mf::kNcross : mf::kNint;
  return g;
}

// One sweep's launches (gather + SDNet for colours 0..3) over the grids at `u` (the
// batch's own, or a scratch copy of the same layout) on stream st.
cudaError_t enqueue_sweep(mf_batch* b, const mf::DevNet& net, int prec, int query, int gather, float* u,
                          cudaStream_t st) {
  for (int c = 0; c < 4; ++c) {
    const mf::ColourGeom g = batch_geom(b, c, query);
    if (g.n_c == 0) continue;
    cudaError_t e = mf::launch_gather_boundary(u, g, net, b->B, st, gather);
    if (e != cudaSuccess) return e;
    e = (prec == MF_PREC_BF16 || prec == MF_PREC_F16)
            ? mf::launch_mlp_bf16(b->B, g, net, u, 0, b->status, st, prec == MF_PREC_F16)
            : mf::launch_mlp_fp32_path(b->B, g, net, u, 0, b->status, prec == MF_PREC_FP32_SIMT, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One sweep as a single cooperative launch (BF16).
cudaError_t enqueue_sweep_whole(mf_batch* b, const mf::DevNet& net, int query, float* u, cudaStream_t st) {
  mf::ColourGeom gc[4];
  int n_col = 0;
  for (int c = 0; c < 4; ++c) {
    const mf::ColourGeom g = batch_geom(b, c, query);
    if (g.n_c > 0) gc[n_col++] = g;
  }
  return mf::launch_mlp_bf16_sweep(gc, n_col, net, u, b->B, b->sync, b->status, st);
}

void drop_graph(mf_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->g_net = nullptr;
  b->g_prec = b->g_query = b->g_gather = -1;
}

// Capture one sweep's per-colour launches over the grids at `u` into an executable graph.
cudaError_t capture_sweep(mf_batch* b, const mf::DevNet& net, int prec, int query, int gather, float* u,
                          cudaGraphExec_t* out) {
  if (!b->cap_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t e1 = enqueue_sweep(b, net, prec, query, gather, u, b->cap_stream);
  const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return e1 != cudaSuccess ? e1 : e2;
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

// The autotuner: time every applicable (mode, gather block) on a scratch copy of the
// grids (the `prev` buffer, which every checked sweep overwrites anyway) and return the
// fastest. Each candidate runs one untimed sweep, then kTimed timed sweeps.
cudaError_t autotune(mf_batch* b, const mf::DevNet& net, int prec, int query, cudaStream_t st, int* mode,
                     int* gather) {
  constexpr int kTimed = 3;
  float* scratch = b->prev;
  cudaError_t e = cudaMemcpyAsync(scratch, b->u, b->total * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  std::vector<std::tuple<int, int>> cand;
  for (int gs : {4, 8, 16}) cand.emplace_back(MF_LAUNCH_PER_COLOUR, gs);
  if (prec == MF_PREC_BF16 && mf::bf16_sweep_supported(net)) cand.emplace_back(MF_LAUNCH_SWEEP, 16);
  float best = 3.4e38f;
  int best_mode = MF_LAUNCH_PER_COLOUR, best_gather = 16;
  for (const auto& c : cand) {
    const int md = std::get<0>(c), gs = std::get<1>(c);
    auto one = [&]() {
      return md == MF_LAUNCH_SWEEP ? enqueue_sweep_whole(b, net, query, scratch, st)
                                   : enqueue_sweep(b, net, prec, query, gs, scratch, st);
    };
    if ((e = one()) != cudaSuccess) break;
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
    for (int k = 0; k < kTimed && e == cudaSuccess; ++k) e = one();
    if (e != cudaSuccess || (e = cudaEventRecord(e1, st)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (ms < best) {
      best = ms;
      best_mode = md;
      best_gather = gs;
    }
  }
  // the graph of the best per-colour configuration, replayed
  if (e == cudaSuccess) {
    int gs = best_mode == MF_LAUNCH_PER_COLOUR ? best_gather : 16;
    cudaGraphExec_t ge = nullptr;
    e = capture_sweep(b, net, prec, query, gs, scratch, &ge);
    if (e == cudaSuccess) {
      e = cudaGraphLaunch(ge, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int k = 0; k < kTimed && e == cudaSuccess; ++k) e = cudaGraphLaunch(ge, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_mode = MF_LAUNCH_GRAPH;
        best_gather = gs;
      }
      cudaGraphExecDestroy(ge);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *mode = best_mode;
  *gather = best_gather;
  return e;
}

}  // namespace

extern "C" {

mf_status mf_destroy_batch(mf_batch* b) {
  if (!b) return MF_OK;
  mf::DeviceGuard guard(b->device);
  drop_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFree(b->u);
  cudaFree(b->prev);
  for (int c = 0; c < 4; ++c) cudaFree(b->table[c]);
  cudaFree(b->B);
  cudaFree(b->partial);
  cudaFree(b->out);
  cudaFree(b->status);
  cudaFree(b->sync);
  cudaFreeHost(b->h_out);
  cudaFreeHost(b->h_status);
  delete b;
  return MF_OK;
}

mf_status mf_create_batch(mf_ctx* ctx, int n, const mf_grid_desc* descs, const double* bc_all, mf_batch** out) {
  if (!descs || !bc_all || !out || n < 1) return fail(MF_ERR_INVALID_ARG, "mf_create_batch: null argument or n < 1");
  *out = nullptr;
  for (int q = 0; q < n; ++q)
    if (descs[q].lx < 1 || descs[q].lx > 128 || descs[q].ly < 1 || descs[q].ly > 128)
      return fail(MF_ERR_INVALID_ARG, "mf_create_batch: lx and ly must be in 1..128");
  if (!ctx) return fail(MF_ERR_INVALID_ARG, "mf_create_batch: null context");
  BT_ON_DEVICE(ctx->device, "mf_create_batch: cudaSetDevice");
  mf_batch* b = new mf_batch();
  b->device = ctx->device;
  b->n = n;
  size_t off = 0, nbc = 0;
  std::vector<size_t> bc_off(n);
  for (int q = 0; q < n; ++q) {
    b->lx.push_back(descs[q].lx);
    b->ly.push_back(descs[q].ly);
    b->nx.push_back(32 * descs[q].lx + 1);
    b->ny.push_back(32 * descs[q].ly + 1);
    b->offset.push_back(off);
    off += ((size_t)b->nx[q] * b->ny[q] + 31) / 32 * 32;  // keep each grid 128-byte aligned
    bc_off[q] = nbc;
    nbc += 2 * (size_t)(b->nx[q] - 1) + 2 * (size_t)(b->ny[q] - 1);
  }
  b->total = (off + kRow - 1) / kRow * kRow;
  // colour tables
  std::vector<mf::SubRef> tab[4];
  for (int q = 0; q < n; ++q) {
    const int nsx = 2 * b->lx[q] - 1, nsy = 2 * b->ly[q] - 1;
    for (int c = 0; c < 4; ++c)
      for (int sb = c >> 1; sb < nsy; sb += 2)
        for (int sa = c & 1; sa < nsx; sa += 2)
          tab[c].push_back(mf::SubRef{(unsigned long long)(b->offset[q] + (size_t)(16 * sb) * b->nx[q] + 16 * sa),
                                      b->nx[q], 0});
  }
  int max_c = 1;
  for (int c = 0; c < 4; ++c) {
    b->n_c[c] = (int)tab[c].size();
    if (b->n_c[c] > max_c) max_c = b->n_c[c];
  }
  cudaError_t e = cudaSuccess;
  double* dbc = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&b->u, b->total * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b->prev, b->total * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(b->u, 0, b->total * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(b->prev, 0, b->total * sizeof(float));
  for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
    if (tab[c].empty()) continue;
    e = cudaMalloc(&b->table[c], tab[c].size() * sizeof(mf::SubRef));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->table[c], tab[c].data(), tab[c].size() * sizeof(mf::SubRef), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->B, (size_t)max_c * 128 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b->partial, mf::kReduceBlocks * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->out, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->sync, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_out, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&dbc, nbc * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(dbc, bc_all, nbc * sizeof(double), cudaMemcpyHostToDevice);
  for (int q = 0; q < n && e == cudaSuccess; ++q)
    e = mf::launch_init_grid(b->u + b->offset[q], b->nx[q], b->ny[q], dbc + bc_off[q], nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (dbc) cudaFree(dbc);
  if (e != cudaSuccess) {
    mf_destroy_batch(b);
    return cuda_fail(e, "mf_create_batch");
  }
  *out = b;
  return MF_OK;
}

mf_status mf_batch_info(const mf_batch* b, int problem, int* nx, int* ny, long long* offset) {
  if (!b || problem < 0 || problem >= b->n) return fail(MF_ERR_INVALID_ARG, "mf_batch_info: bad batch or problem");
  if (nx) *nx = b->nx[problem];
  if (ny) *ny = b->ny[problem];
  if (offset) *offset = (long long)b->offset[problem];
  return MF_OK;
}

mf_status mf_batch_upload(mf_batch* b, int problem, const float* src, int on_device, void* stream) {
  if (!b || !src || problem < 0 || problem >= b->n) return fail(MF_ERR_INVALID_ARG, "mf_batch_upload: bad argument");
  BT_ON_DEVICE(b->device, "mf_batch_upload: cudaSetDevice");
  BT_CUDA(cudaMemcpyAsync(b->u + b->offset[problem], src, (size_t)b->nx[problem] * b->ny[problem] * sizeof(float),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          reinterpret_cast<cudaStream_t>(stream)),
          "mf_batch_upload: cudaMemcpyAsync");
  return MF_OK;
}

mf_status mf_batch_download(const mf_batch* b, int problem, float* dst, int on_device, void* stream) {
  if (!b || !dst || problem < 0 || problem >= b->n) return fail(MF_ERR_INVALID_ARG, "mf_batch_download: bad argument");
  BT_ON_DEVICE(b->device, "mf_batch_download: cudaSetDevice");
  BT_CUDA(cudaMemcpyAsync(dst, b->u + b->offset[problem], (size_t)b->nx[problem] * b->ny[problem] * sizeof(float),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          reinterpret_cast<cudaStream_t>(stream)),
          "mf_batch_download: cudaMemcpyAsync");
  return MF_OK;
}

mf_status mf_batch_residual(const mf_batch* b, int problem, double* max_abs, double* rms, void* stream) {
  if (!b || problem < 0 || problem >= b->n) return fail(MF_ERR_INVALID_ARG, "mf_batch_residual: bad argument");
  BT_ON_DEVICE(b->device, "mf_batch_residual: cudaSetDevice");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nx = b->nx[problem], ny = b->ny[problem];
  BT_CUDA(mf::launch_reduce(b->u + b->offset[problem], nullptr, nx, ny, b->partial, b->out + 8, st),
          "mf_batch_residual: reduce");
  BT_CUDA(cudaMemcpyAsync(b->h_out + 8, b->out + 8, 5 * sizeof(double), cudaMemcpyDeviceToHost, st),
          "mf_batch_residual: read");
  BT_CUDA(cudaStreamSynchronize(st), "mf_batch_residual: synchronize");
  if (max_abs) *max_abs = b->h_out[10];
  if (rms) *rms = std::sqrt(b->h_out[11] / ((double)(nx - 2) * (double)(ny - 2)));
  return MF_OK;
}

}  // extern "C"

namespace {

mf_status batch_sweep_impl(mf_batch* b, const mf_sdnet* net, const mf_sweep_opts* o, mf_sweep_result* res,
                           void* stream) {
  if (!b || !net || !o) return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: null argument");
  if (o->n_sweeps < 0) return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: n_sweeps < 0");
  if (o->schedule != MF_SCHEDULE_MULTIPLICATIVE)
    return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: batches use the multiplicative schedule");
  if (o->precision != MF_PREC_FP32 && o->precision != MF_PREC_BF16 && o->precision != MF_PREC_FP32_SIMT &&
      o->precision != MF_PREC_F16)
    return fail(MF_ERR_INVALID_ARG,
                "mf_batch_sweep: precision must be MF_PREC_FP32, MF_PREC_FP32_SIMT, MF_PREC_BF16 or MF_PREC_F16");
  if (o->query != MF_QUERY_FULL && o->query != MF_QUERY_CENTRE)
    return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: unknown query");
  if (o->colours != 0 && o->colours != 15) return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: colours must be 0 (all)");
  if (o->check_every < 1) return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: check_every must be >= 1");
  if (!std::isfinite(o->eps)) return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: eps must be finite");
  int net_device = 0;
  const mf::DevNet* d = mf::devnet_of(net, &net_device);
  if (net_device != b->device) return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: batch and SDNet on different devices");
  if (o->precision == MF_PREC_BF16 && !mf::bf16_supported(*d))
    return fail(MF_ERR_UNSUPPORTED, "mf_batch_sweep: BF16 path needs 1..5 hidden layers");
  if (o->precision == MF_PREC_F16 && !mf::f16_supported(*d))
    return fail(MF_ERR_UNSUPPORTED, "mf_batch_sweep: F16 path needs 1..5 hidden layers and weights in the F16 range");
  if (o->launch_mode < MF_LAUNCH_PER_COLOUR || o->launch_mode > MF_LAUNCH_AUTO)
    return fail(MF_ERR_INVALID_ARG, "mf_batch_sweep: unknown launch_mode");
  if (o->launch_mode == MF_LAUNCH_SWEEP && (o->precision != MF_PREC_BF16 || !mf::bf16_sweep_supported(*d)))
    return fail(MF_ERR_UNSUPPORTED, "mf_batch_sweep: MF_LAUNCH_SWEEP runs BF16 sweeps with an SDNet without a "
                                    "boundary embedding");
  BT_ON_DEVICE(b->device, "mf_batch_sweep: cudaSetDevice");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  BT_CUDA(cudaMemsetAsync(b->status, 0, sizeof(int), st), "mf_batch_sweep: reset status");

  int mode = o->launch_mode, gather = 16;
  if (mode == MF_LAUNCH_AUTO) {
    bool found = false;
    for (const auto& c : b->tuned)
      if (c.net == net && c.prec == o->precision && c.query == o->query) {
        mode = c.mode;
        gather = c.gather;
        found = true;
      }
    if (!found) {
      BT_CUDA(autotune(b, *d, o->precision, o->query, st, &mode, &gather), "mf_batch_sweep: autotune");
      b->tuned.push_back(mf_batch::Choice{net, o->precision, o->query, mode, gather});
    }
  }
  if (res) *res = mf_sweep_result{0, -1.0, 0, 0, 0.0, 0.0, 0.0, 0, 0, MF_OK, mode, gather};

  // graph of one unchecked sweep, captured once the kernels have run uncaptured
  const bool use_graph = mode == MF_LAUNCH_GRAPH;
  if (use_graph && b->warmed &&
      (b->g_net != net || b->g_prec != o->precision || b->g_query != o->query || b->g_gather != gather || !b->graph)) {
    drop_graph(b);
    BT_CUDA(capture_sweep(b, *d, o->precision, o->query, gather, b->u, &b->graph), "mf_batch_sweep: capture");
    b->g_net = net;
    b->g_prec = o->precision;
    b->g_query = o->query;
    b->g_gather = gather;
  }

  int done = 0, launches = 0, graph_sweeps = 0;
  bool checked = false;
  const size_t bytes = b->total * sizeof(float);
  for (int k = 0; k < o->n_sweeps; ++k) {
    const bool check = ((k + 1) % o->check_every == 0) || (k + 1 == o->n_sweeps);
    if (check)
      BT_CUDA(cudaMemcpyAsync(b->prev, b->u, bytes, cudaMemcpyDeviceToDevice, st), "mf_batch_sweep: snapshot");
    if (use_graph && b->graph) {
      BT_CUDA(cudaGraphLaunch(b->graph, st), "mf_batch_sweep: graph launch");
      ++graph_sweeps;
      launches += 8;
    } else if (mode == MF_LAUNCH_SWEEP) {
      BT_CUDA(enqueue_sweep_whole(b, *d, o->query, b->u, st), "mf_batch_sweep: whole-sweep launch");
      launches += 1;
    } else {
      BT_CUDA(enqueue_sweep(b, *d, o->precision, o->query, gather, b->u, st), "mf_batch_sweep: sweep");
      b->warmed = true;
      launches += 8;
    }
    done = k + 1;
    if (check) {
      BT_CUDA(mf::launch_reduce(b->u, b->prev, (int)kRow, (int)(b->total / kRow), b->partial, b->out, st, false),
              "mf_batch_sweep: reduce");
      launches += 2;
      checked = true;
      if (o->eps > 0.0) {
        BT_CUDA(cudaMemcpyAsync(b->h_out, b->out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "mf_batch_sweep: read");
        BT_CUDA(cudaMemcpyAsync(b->h_status, b->status, sizeof(int), cudaMemcpyDeviceToHost, st), "mf_batch_sweep: read");
        BT_CUDA(cudaStreamSynchronize(st), "mf_batch_sweep: synchronize");
        if (*b->h_status != mf::kDevErrNone) return fail(MF_ERR_TIMEOUT, "mf_batch_sweep: a kernel wait timed out");
        if (!std::isfinite(b->h_out[4])) return fail(MF_ERR_DIVERGED, "mf_batch_sweep: delta is not finite");
        if (b->h_out[4] < o->eps) break;
      }
    }
  }
  BT_CUDA(cudaMemcpyAsync(b->h_out, b->out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "mf_batch_sweep: read");
  BT_CUDA(cudaMemcpyAsync(b->h_status, b->status, sizeof(int), cudaMemcpyDeviceToHost, st), "mf_batch_sweep: read");
  BT_CUDA(cudaStreamSynchronize(st), "mf_batch_sweep: synchronize");
  if (*b->h_status != mf::kDevErrNone) return fail(MF_ERR_TIMEOUT, "mf_batch_sweep: a kernel wait timed out");
  if (res) {
    res->sweeps_done = done;
    res->delta = checked ? b->h_out[4] : -1.0;
    res->kernel_launches = launches;
    res->mlp_launches = mode == MF_LAUNCH_SWEEP ? done : 4 * done;
    res->sweeps_bf16 = o->precision == MF_PREC_BF16 ? done : 0;
    res->graph_sweeps = graph_sweeps;
  }
  if (checked && !std::isfinite(b->h_out[4])) return fail(MF_ERR_DIVERGED, "mf_batch_sweep: delta is not finite");
  return MF_OK;
}

}  // namespace

extern "C" {

mf_status mf_batch_sweep(mf_batch* b, const mf_sdnet* net, const mf_sweep_opts* o, mf_sweep_result* res,
                         void* stream) {
  const mf_status st = batch_sweep_impl(b, net, o, res, stream);
  if (res) res->status = st;
  return st;
}

}  // extern "C"
