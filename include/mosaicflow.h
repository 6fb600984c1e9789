/*
 * mosaicflow.h -- C ABI of the GB300 Mosaic Flow sweep engine.
 *
 * Mosaic Flow (Feeney, Li, Bostanabad, Chandramowlishwaran, SC '23) solves the 2-D
 * Laplace equation with Dirichlet data (Section 2.1, Eq. 2) on a large domain by
 * iterating a pre-trained subdomain network (SDNet, Section 2.4 and Section 3) over
 * overlapping unit subdomains (Section 2.4, Figure 3), batching the non-overlapping
 * ("atomic") subdomains of one iteration (Section 4.1) and stopping on the relative
 * change of the boundary values (Algorithm 2).
 *
 * Conventions shared by every call:
 *  - Domain [0, lx] x [0, ly] in units of the subdomain side; 32 grid intervals per
 *    unit, so the grid has nx = 32 lx + 1 columns and ny = 32 ly + 1 rows, stored
 *    row-major as FP32, element (iy, ix) at offset iy * nx + ix, x = ix / 32.
 *  - Subdomain (a, b), a in [0, 2lx-2], b in [0, 2ly-2], covers grid points
 *    [16a, 16a+32] x [16b, 16b+32] (lattice spacing 1/2, Section 4.2). Its 128
 *    boundary values are read counter-clockwise from its corner (16a, 16b): bottom
 *    (i = 0..31), right (j = 0..31), top (i = 32..1), left (j = 32..1). Its 961
 *    interior points p = py * 31 + px have local coordinates ((px+1)/32, (py+1)/32).
 *  - Colour c = (a mod 2) + 2 (b mod 2); subdomains of one colour have disjoint
 *    interiors and are predicted as one batch.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls enqueue their GPU work on it and return; calls that hand a host scalar
 *    back synchronise that stream first, as stated per call.
 *  - Every call returns an mf_status; nothing throws across the ABI. A call that
 *    fails validation returns MF_ERR_INVALID_ARG before any GPU work is enqueued.
 *    mf_last_error() gives a message for the calling thread's last failure.
 *  - The library owns the device memory behind handles; the caller owns host
 *    buffers and streams. There is no CPU fallback: without a usable CUDA device
 *    every call that needs one returns MF_ERR_CUDA.
 *  - Every handle is created under an mf_ctx, which names one CUDA device, and lives
 *    on that device. A call on a handle makes the handle's device current while it
 *    runs and restores the caller's current device before it returns. Streams passed
 *    with a handle must belong to the handle's device.
 */
#ifndef MOSAICFLOW_H
#define MOSAICFLOW_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int mf_status;
#define MF_OK 0
#define MF_ERR_INVALID_ARG (-1)  /* bad pointer, size, shape or option */
#define MF_ERR_CUDA (-2)         /* a CUDA runtime call failed (message has the CUDA error) */
#define MF_ERR_OUT_OF_MEMORY (-3)
#define MF_ERR_DIVERGED (-4)     /* delta became NaN or infinite */
#define MF_ERR_TIMEOUT (-5)      /* a bounded wait inside a kernel gave up; results invalid */
#define MF_ERR_UNSUPPORTED (-6)  /* valid request this build or device cannot serve */

#define MF_PREC_FP32 0  /* FP32 accuracy: width-128 SDNets (tanh or GELU) on the tensor cores, each hidden
                           product split in three F16 products with FP32 accumulation; other SDNets as
                           MF_PREC_FP32_SIMT */
#define MF_PREC_BF16 1  /* BF16 weights/activations on tcgen05 tensor cores, FP32 accumulate */
#define MF_PREC_MIXED 2 /* BF16 sweeps until delta < eps_coarse or stalls, then FP32 refinement */
#define MF_PREC_FP32_SIMT 3 /* FP32 weights and activations on the CUDA cores (FMA), accurate tanh */
#define MF_PREC_F16 4   /* F16 weights/activations on the tcgen05 tensor cores, FP32 accumulate: the BF16
                           kernel with the other 16-bit type (three more mantissa bits, the same speed);
                           per-colour launches; SDNets whose hidden weights lie within the F16 range */

#define MF_SCHEDULE_MULTIPLICATIVE 0 /* colours 0..3 in turn, each reads the latest grid */
#define MF_SCHEDULE_ADDITIVE 1       /* all colours read the old grid; overlaps averaged */

#define MF_QUERY_FULL 0   /* predict all 961 interior points of every subdomain */
#define MF_QUERY_CENTRE 1 /* predict only the 61 centre-cross points (interfaces) */

/* How a multiplicative sweep is launched (mf_sweep_opts.launch_mode). */
#define MF_LAUNCH_PER_COLOUR 0 /* per colour one boundary-gather launch and one SDNet launch */
#define MF_LAUNCH_GRAPH 1      /* mf_batch_sweep: the same launches, unchecked sweeps replayed from a CUDA graph */
#define MF_LAUNCH_SWEEP 2      /* one cooperative launch per sweep: gather, SDNet and scatter of every colour,
                                  colours separated by device-wide barriers (BF16 sweeps; SDNets without a
                                  boundary embedding) */
#define MF_LAUNCH_AUTO 3       /* mf_batch_sweep: time the launch modes and gather block sizes on a copy of
                                  the batch at the first call for this SDNet, precision and query; keep the
                                  fastest */

typedef struct mf_ctx mf_ctx;     /* one CUDA device and the library's set-up on it */
typedef struct mf_sdnet mf_sdnet; /* device-resident SDNet weights (both precisions) */
typedef struct mf_grid mf_grid;   /* device grid of one problem plus its sweep scratch */
typedef struct mf_batch mf_batch; /* device grids of many independent problems */

typedef struct {
  int width; /* hidden width H: 64 or 128 */
  int depth; /* number of tanh layers (first layer + depth-1 hidden H x H layers), 2..6 */
} mf_sdnet_desc;

typedef struct {
  int lx; /* domain width in unit subdomain lengths, 1..128 */
  int ly; /* domain height, 1..128 */
} mf_grid_desc;

typedef struct {
  int n_sweeps;    /* maximum number of sweeps, >= 0 */
  int schedule;    /* MF_SCHEDULE_* */
  int precision;   /* MF_PREC_* */
  int colours;     /* bitmask of colours applied each sweep, in order 0..3; 0 means all */
  double eps;      /* stop once delta < eps (eps <= 0: run all n_sweeps, no mid-run sync) */
  int check_every; /* delta computed after every check_every-th sweep and the last (>= 1) */
  int profile;     /* nonzero: time each phase with CUDA events recorded on `stream` */
  double eps_coarse; /* MF_PREC_MIXED: switch from BF16 to FP32 once delta < eps_coarse (> 0) */
  int query;         /* MF_QUERY_FULL, or MF_QUERY_CENTRE (multiplicative schedule only) */
  int launch_mode;   /* MF_LAUNCH_*; mf_sweep takes MF_LAUNCH_PER_COLOUR or MF_LAUNCH_SWEEP */
} mf_sweep_opts;

typedef struct {
  int sweeps_done;     /* sweeps applied */
  double delta;        /* delta of the last checked sweep (Algorithm 2), -1 if none checked */
  int kernel_launches; /* kernels this call launched */
  int mlp_launches;    /* of which SDNet (gather-fed MLP + scatter) kernels */
  double ms_gather;    /* profile only: summed event time of the boundary-gather kernels */
  double ms_mlp;       /* profile only: summed event time of the SDNet + scatter kernels */
  double ms_reduce;    /* profile only: summed event time of snapshot copies and reductions */
  int sweeps_bf16;     /* of sweeps_done, sweeps run on the BF16 path */
  int graph_sweeps;    /* mf_batch_sweep: sweeps replayed from the captured graph */
  mf_status status;    /* the call's own return value (MF_OK, MF_ERR_DIVERGED, ...) */
  int launch_mode;     /* the MF_LAUNCH_* mode that ran (the autotuner's choice under MF_LAUNCH_AUTO) */
  int gather_block;    /* subdomains per block of the boundary-gather launches (4, 8 or 16) */
} mf_sweep_result;

#define MF_ACT_TANH 0 /* tanh activations (the default network) */
#define MF_ACT_GELU 1 /* GELU activations, x Phi(x) (Section 3.1) */

typedef struct {
  int width;          /* hidden width H: 64 or 128 */
  int depth;          /* activation layers (first + depth-1 hidden H x H layers), 2..6 */
  int activation;     /* MF_ACT_TANH or MF_ACT_GELU, for the first and hidden layers */
  int embed_channels; /* 0: the first layer reads the 128 boundary values; C in 1..16: it
                         reads their conv1d embedding of C x 64 values (see mf_load_sdnet_ex) */
  int embed_kernel;   /* with embed_channels > 0: odd kernel size K of both conv layers, 1..9 */
} mf_sdnet_desc_ex;

/* Message describing the calling thread's most recent failed call ("" if none). */
const char* mf_last_error(void);

/* Library version as major*10000 + minor*100 + patch (0.3.0: MF_PREC_F16). */
int mf_version(void);

/* mf_ctx_create -- the execution context of the Laplace problems of Section 2.1 (Eq. 2)
 * on one device: it binds the library to CUDA device `device` (0-based, as numbered by
 * the CUDA runtime under CUDA_VISIBLE_DEVICES), initialises the CUDA context there,
 * checks that the device can run this build (compute capability 10.3, the sm_103a
 * code the library carries) and records its SM count. The paper has no such object;
 * it runs one process per GPU and leaves the device implicit.
 * Grids, batches, SDNets and trainers are created under a context and stay on its
 * device. The context owns no device memory; destroying it does not free the handles
 * created under it, which stay valid and are freed by their own calls. It is safe to
 * create several contexts for one device. The caller's current device is unchanged.
 * Errors: MF_ERR_INVALID_ARG (null `out`, device < 0 or not present), MF_ERR_UNSUPPORTED
 * (a device of another compute capability), MF_ERR_CUDA (no CUDA device or driver).
 * Synchronous. */
mf_status mf_ctx_create(int device, mf_ctx** out);
mf_status mf_ctx_destroy(mf_ctx* ctx);

/* The device index of a context, and its SM count (either pointer may be NULL). */
mf_status mf_ctx_device(const mf_ctx* ctx, int* device, int* sm_count);

/* mf_load_sdnet -- copy an SDNet to the context's device (Section 3.1-3.2).
 * `weights` is a host array of FP32 values packed as
 *   W0[H][130], b0[H], { W_l[H][H], b_l[H] } for l = 1..depth-1, w_out[H], b_out
 * where columns 0..127 of W0 are the boundary block W1 and columns 128..129 the
 * coordinate block W2 of the input-split first layer (Eq. 7-8); rows are output
 * units. The array is read during the call and not retained. The handle keeps an
 * FP32 copy and a BF16 (round-to-nearest-even) copy laid out for the tensor cores.
 * Both copies are kept, so one handle serves every precision of mf_sweep; the
 * precision is chosen per sweep, not at load time.
 * Errors: MF_ERR_INVALID_ARG for a null pointer or unsupported width/depth,
 * MF_ERR_OUT_OF_MEMORY / MF_ERR_CUDA from the device. Synchronous. */
mf_status mf_load_sdnet(mf_ctx* ctx, const mf_sdnet_desc* desc, const float* weights, mf_sdnet** out);

/* mf_load_sdnet_ex -- mf_load_sdnet for the SDNet variants of Section 3.1: GELU
 * activations and/or a boundary embedding by 1-D convolutions, the boundary taken as a
 * closed curve (the paper gives no sizes; channels and kernel size are parameters).
 * With embed_channels = C > 0 the 128 CCW boundary values g pass through
 *   h1[c][i] = act(cb1[c] + sum_t cw1[c][t] g[(i + t - K/2) mod 128]),      i < 128
 *   h2[c][i] = act(cb2[c] + sum_{c',t} cw2[c][c'][t] h1[c'][(2i + t - K/2) mod 128]), i < 64
 * (act = the network's activation) and z[c * 64 + i] = h2[c][i] replaces g as the first
 * layer's boundary input; the first layer stays input-split (Eq. 8), evaluated once per
 * subdomain. `weights` then begins with cw1[C][1][K], cb1[C], cw2[C][C][K], cb2[C], and
 * W0 is [H][C*64 + 2]; the rest of the packing is that of mf_load_sdnet.
 * MF_ACT_GELU is x Phi(x): exact (erf) on the FP32 path; on the BF16 path its tanh form
 * 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (Hendrycks and Gimpel), whose error is
 * far below the BF16 rounding. Errors and synchronisation as mf_load_sdnet. */
mf_status mf_load_sdnet_ex(mf_ctx* ctx, const mf_sdnet_desc_ex* desc, const float* weights, mf_sdnet** out);
mf_status mf_free_sdnet(mf_sdnet* net);

/* mf_create_grid -- allocate the global grid of one Laplace problem (Eq. 2) on the
 * context's device and set it up: boundary from `bc_ccw`, interior zero.
 * `bc_ccw` is a host array of 2(nx-1) + 2(ny-1) FP64 Dirichlet values in
 * counter-clockwise order from (0,0): bottom ix = 0..nx-2, right iy = 0..ny-2,
 * top ix = nx-1..1, left iy = ny-1..1. Values are rounded to FP32. Synchronous.
 * Errors: MF_ERR_INVALID_ARG (null pointer, lx or ly outside 1..128),
 * MF_ERR_OUT_OF_MEMORY, MF_ERR_CUDA. */
mf_status mf_create_grid(mf_ctx* ctx, const mf_grid_desc* desc, const double* bc_ccw, mf_grid** out);
mf_status mf_destroy_grid(mf_grid* grid);

/* Grid dimensions (points): *nx = 32 lx + 1, *ny = 32 ly + 1. */
mf_status mf_grid_dims(const mf_grid* grid, int* nx, int* ny);

/* Overwrite the whole grid (ny x nx FP32, boundary included) from `src`, a host
 * (src_on_device = 0) or device (1) pointer. Asynchronous on `stream`; a host
 * source should be pinned for the copy to overlap, and must stay valid until the
 * stream reaches the copy. */
mf_status mf_grid_upload(mf_grid* grid, const float* src, int src_on_device, void* stream);

/* Copy the whole grid to `dst` (host or device). Asynchronous like mf_grid_upload. */
mf_status mf_grid_download(const mf_grid* grid, float* dst, int dst_on_device, void* stream);

/* mf_sweep -- run Mosaic Flow predictor sweeps on the grid (Section 2.4, Section 4.1,
 * Algorithm 2). Each sweep, for each selected colour in order 0..3: gather the 128
 * boundary values of every subdomain of the colour, evaluate the SDNet at its 961
 * interior points with the input-split first layer (Eq. 8), and write the
 * predictions into the grid. MF_SCHEDULE_MULTIPLICATIVE writes them directly, so
 * later colours see earlier colours' results. MF_SCHEDULE_ADDITIVE makes every
 * colour read the grid as it was before the sweep and sets each interior point to
 * the average of the predictions of the subdomains that contain it.
 * After each checked sweep, delta = ||u_k - u_{k-1}||_2 / ||u_{k-1}||_2 over all grid
 * points is computed with FP64 accumulation (0/0 = 0). With eps > 0 the call
 * synchronises `stream` after each checked sweep and stops once delta < eps. The call
 * always synchronises `stream` before returning to fill `result` (which may be NULL).
 * MF_PREC_MIXED is iterative refinement of the converged field: BF16 sweeps (checked
 * every sweep) until delta < eps_coarse or until a BF16 sweep fails to reduce delta
 * (delta_k >= delta_{k-1}: the BF16 iteration has reached the floor its rounding
 * allows), then FP32 sweeps until delta < eps, all within the n_sweeps budget.
 * Launch modes: MF_LAUNCH_PER_COLOUR, or MF_LAUNCH_SWEEP (one cooperative launch per
 * BF16 sweep of all colours; the multiplicative schedule with all colours, SDNets
 * without a boundary embedding, else MF_ERR_UNSUPPORTED; FP32 sweeps of MF_PREC_MIXED
 * keep the per-colour launches); other modes return MF_ERR_INVALID_ARG.
 * MF_QUERY_CENTRE is the interface-only iteration of Algorithm 2: a subdomain's only
 * interior points that other subdomains read are its centre lines (x or y on the
 * 1/2 lattice), so each sweep predicts just those 61 points and leaves the others as
 * they are; the lattice-line values evolve exactly as with MF_QUERY_FULL. Algorithm 2's
 * final full prediction averaged over overlaps is then one MF_SCHEDULE_ADDITIVE sweep
 * with MF_QUERY_FULL.
 * Errors: MF_ERR_INVALID_ARG (null handle/opts, bad option), MF_ERR_DIVERGED (delta
 * not finite; the grid holds the diverged state), MF_ERR_TIMEOUT, MF_ERR_CUDA. */
mf_status mf_sweep(mf_grid* grid, const mf_sdnet* net, const mf_sweep_opts* opts,
                   mf_sweep_result* result, void* stream);

/* Block the calling host thread until all work enqueued on `stream` has finished. */
mf_status mf_synchronize(void* stream);

/* mf_residual -- 5-point Laplace residual r = u_E + u_W + u_N + u_S - 4u over the
 * interior points (grid units, no 1/h^2), accumulated in FP64 in a fixed order (the
 * result does not depend on timing). Writes max |r| and the root mean square of r
 * to the host doubles; synchronises `stream`. Either output pointer may be NULL. */
mf_status mf_residual(const mf_grid* grid, double* max_abs, double* rms, void* stream);

/* mf_create_batch -- n independent Laplace problems (Eq. 2) of sizes descs[q] in one
 * device buffer, each set up like mf_create_grid. `bc_all` holds the problems' CCW
 * Dirichlet lists (as in mf_create_grid) one after another. Sweeps over a batch treat
 * the atomic subdomains of one colour of all problems as one batch (Section 4.1
 * applied across problems). Synchronous. Errors as mf_create_grid. */
mf_status mf_create_batch(mf_ctx* ctx, int n, const mf_grid_desc* descs, const double* bc_all, mf_batch** out);
mf_status mf_destroy_batch(mf_batch* batch);

/* Grid dimensions of one problem and its offset (in floats) inside the batch buffer. */
mf_status mf_batch_info(const mf_batch* batch, int problem, int* nx, int* ny, long long* offset);

/* Copy one problem's grid in or out (host or device pointer), asynchronously on stream. */
mf_status mf_batch_upload(mf_batch* batch, int problem, const float* src, int src_on_device, void* stream);
mf_status mf_batch_download(const mf_batch* batch, int problem, float* dst, int dst_on_device, void* stream);

/* mf_batch_sweep -- multiplicative sweeps (all four colours) of every problem of the
 * batch at once (Section 4.1's batching of atomic subdomains, applied across problems):
 * each colour of all problems is one batch. Options as mf_sweep (precision MF_PREC_FP32,
 * MF_PREC_FP32_SIMT, MF_PREC_BF16 or MF_PREC_F16; MF_QUERY_FULL or MF_QUERY_CENTRE;
 * colours must be 0). delta is taken
 * over all problems' grid points together. Launch modes (opts->launch_mode):
 *  - MF_LAUNCH_PER_COLOUR: per colour one gather launch and one SDNet launch;
 *  - MF_LAUNCH_GRAPH: sweeps after the first are replayed from a CUDA graph of one
 *    sweep (re-captured when the SDNet, precision or query changes);
 *  - MF_LAUNCH_SWEEP: one cooperative launch per sweep (BF16 only, else
 *    MF_ERR_UNSUPPORTED);
 *  - MF_LAUNCH_AUTO: at the first call for an SDNet, precision and query, every
 *    applicable mode and gather block size (4, 8, 16 subdomains) is timed over a few
 *    sweeps of a scratch copy of the grids (the batch's own grids are not touched) and
 *    the fastest is kept for later calls with the same SDNet, precision and query.
 * result->launch_mode and result->gather_block report what ran. Synchronises `stream`
 * before returning. Errors as mf_sweep. */
mf_status mf_batch_sweep(mf_batch* batch, const mf_sdnet* net, const mf_sweep_opts* opts,
                         mf_sweep_result* result, void* stream);

/* 5-point residual of one problem of the batch, as mf_residual. */
mf_status mf_batch_residual(const mf_batch* batch, int problem, double* max_abs, double* rms, void* stream);

/* mf_sweep_noalloc -- the multiplicative sweep of mf_sweep (n_sweeps sweeps, all four
 * colours, no early stop) for callers that must not allocate device memory during the
 * call: code whose device memory belongs to another allocator's pool, and loops that
 * cannot afford the device synchronisation a cudaMalloc/cudaFree implies. The paper
 * has no counterpart; this is an interface convenience of this library.
 * `u` is the caller's device grid (ny x nx FP32, row-major, boundary included), read
 * and updated in place; `net` was loaded earlier with mf_load_sdnet under a context of
 * the current device (the call does not switch devices; another device returns
 * MF_ERR_INVALID_ARG); `precision` is MF_PREC_FP32 (here always the CUDA-core FP32
 * kernel of MF_PREC_FP32_SIMT) or MF_PREC_BF16. If `delta` is not
 * NULL it receives delta of the last sweep (-1 when n_sweeps is 0). The call is
 * synchronous: it waits for its work on `stream` to finish, then returns.
 * Memory: nothing is allocated. All scratch lives in one fixed array of about 4.7 MB
 * that every GPU using this library holds until the process exits; grids are limited
 * to 1 <= lx, ly <= 32 (larger sizes return MF_ERR_INVALID_ARG). The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and keeps it for
 * later calls. All calls share the one array, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must not be issued.
 * Errors: as mf_sweep. */
mf_status mf_sweep_noalloc(float* u, int lx, int ly, const mf_sdnet* net, int precision, int n_sweeps,
                           double* delta, void* stream);

/* mf_check_wait_timeout -- failure-detection self-test of the bounded device waits.
 * Launches one CTA whose 64 threads wait, through the same bounded-wait routines as the
 * tensor-core SDNet kernel, on an mbarrier phase that nothing completes, with a limit of
 * limit_ms milliseconds (0 < limit_ms <= 1000). Every wait must give up, record the
 * timeout in the device status word and return; the call then reads that word as
 * mf_sweep does. Returns MF_ERR_TIMEOUT when the status word recorded the timeout (the
 * designed outcome), MF_OK if it did not (a defect), MF_ERR_INVALID_ARG for a bad limit,
 * MF_ERR_CUDA on a CUDA error. *waits_gave_up (may be NULL) receives how many of the 64
 * waits returned without the phase completing (64 by design). Synchronous; the device
 * context stays usable. The paper has no counterpart: this checks this library's
 * failure handling. */
mf_status mf_check_wait_timeout(double limit_ms, int* waits_gave_up);

/* ---- Physics-informed SDNet training (Section 3.3, Eq. 3, Algorithm 1) ---- */

#define MF_OPT_SGD 0  /* w -= lr g */
#define MF_OPT_LAMB 1 /* LAMB (You et al., ICLR 2020): Adam moments, trust ratio ||w||/||r|| per tensor */

#define MF_TRAIN_ENGINE_AUTO 0 /* fused tensor-core layer kernels for BF16 at width 128, else GEMM */
#define MF_TRAIN_ENGINE_GEMM 1 /* layer GEMMs and elementwise steps as separate kernels (any width/precision) */

typedef struct mf_trainer mf_trainer; /* device weights, optimiser state and training scratch */

typedef struct {
  int width;         /* hidden width H: 64 or 128 */
  int depth;         /* tanh layers, 2..6, as mf_sdnet_desc */
  int precision;     /* MF_PREC_FP32, or MF_PREC_BF16: BF16 operands of the H x H layer GEMMs */
  int optimizer;     /* MF_OPT_SGD or MF_OPT_LAMB */
  int max_functions; /* functions per chunk (>= 1); a call with more functions runs in chunks */
  int max_points;    /* largest Nc or Nb of any call: a multiple of 64 */
  float beta1, beta2, eps, weight_decay; /* LAMB hyper-parameters (ignored by SGD) */
  int engine;        /* MF_TRAIN_ENGINE_AUTO or MF_TRAIN_ENGINE_GEMM (same results to rounding) */
} mf_train_desc;

/* mf_create_trainer -- device state for training one SDNet on the context's device.
 * `weights`: host FP32 parameters in the mf_load_sdnet packing, copied during the call.
 * Device memory grows with max_functions * max_points * width * depth (about 20 GB at
 * 1024 x 1024 x 128 x 6 in BF16 with the GEMM engine, 8 GB with the fused engine): a
 * chunk of functions is processed at a time, so max_functions bounds memory without
 * bounding the batch. The fused engine (BF16, width 128) runs each layer as one
 * tensor-core kernel that recomputes pre-activations in the backward pass instead of
 * storing them; the GEMM engine stores them and runs each layer GEMM as a separate
 * FP32-accumulating kernel.
 * Errors: MF_ERR_INVALID_ARG (null pointer, unsupported option, non-finite weight,
 * 4 * max_functions * max_points above 2^31 - 1), MF_ERR_OUT_OF_MEMORY, MF_ERR_CUDA.
 * Synchronous. */
mf_status mf_create_trainer(mf_ctx* ctx, const mf_train_desc* desc, const float* weights, mf_trainer** out);
mf_status mf_destroy_trainer(mf_trainer* trainer);

/* Replace the weights from a host (src_on_device = 0) or device (1) FP32 array in the
 * packing above; optimiser moments are kept. Asynchronous on `stream`. */
mf_status mf_trainer_set_weights(mf_trainer* trainer, const float* src, int src_on_device, void* stream);

/* Copy the current weights, or the gradient of the last mf_train_grad / mf_train_step,
 * to a host or device FP32 array in the packing above. Asynchronous on `stream`. */
mf_status mf_trainer_get_weights(const mf_trainer* trainer, float* dst, int dst_on_device, void* stream);
mf_status mf_trainer_get_grads(const mf_trainer* trainer, float* dst, int dst_on_device, void* stream);

/* mf_train_grad -- loss and gradient of one training iteration (Algorithm 1 on one
 * device, where the gradient allreduce is the identity):
 *   L = L_data + L_pde,  L_data = mean over the F * Nb data points of (N(x, g_f) - y)^2,
 *   L_pde = mean over the F * Nc collocation points of (Delta_x N(x, g_f))^2   (Eq. 3),
 * with N the SDNet of Eq. 7-8 and Delta_x its Laplacian in the query coordinate.
 * Device arrays (FP32, row-major, read only): G [F][128] boundary values of each
 * function (CCW from the corner, as in a subdomain), Xc [F][Nc][2] collocation points,
 * Xb [F][Nb][2] data points, Yb [F][Nb] their targets, each starting on a 16-byte
 * boundary (the kernels read them 16 bytes at a time). Nc and Nb must be multiples of 64
 * and at most max_points; F >= 1. The gradient stays on the device (mf_trainer_get_grads).
 * If loss3 is not NULL it receives (L, L_data, L_pde) in that order. Synchronises `stream`.
 * Errors: MF_ERR_INVALID_ARG, MF_ERR_DIVERGED (a loss term is not finite),
 * MF_ERR_TIMEOUT (a bounded wait in a fused kernel gave up), MF_ERR_CUDA. */
mf_status mf_train_grad(mf_trainer* trainer, int F, int Nc, int Nb, const float* G, const float* Xc,
                        const float* Xb, const float* Yb, double* loss3, void* stream);

/* mf_train_step -- mf_train_grad followed by the optimiser update with learning rate lr
 * (Algorithm 1, step 4; LAMB as used for SDNet training in Section 5.2). Arguments and
 * errors as mf_train_grad. The update is enqueued behind the gradient pass and reads
 * its outcome on the device: when a loss term is not finite or a wait gave up, the
 * weights, the optimiser moments and the step count stay as they were. Synchronises
 * `stream` once. */
mf_status mf_train_step(mf_trainer* trainer, int F, int Nc, int Nb, const float* G, const float* Xc,
                        const float* Xb, const float* Yb, float lr, double* loss3, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MOSAICFLOW_H */
