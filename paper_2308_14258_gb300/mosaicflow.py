"""ctypes binding of libmosaicflow.so: the mf_* calls with Python argument marshalling.

Every step of the sweep and of the training step runs in the library's own sm_103a
kernels (no other CUDA library is linked); this module only
converts arguments (NumPy arrays, torch tensors, streams) to the C ABI and raises
MFError on a non-zero status. There is no CPU fallback: if the library is missing or cannot be
loaded, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MF_OK = 0
MF_ERR_INVALID_ARG = -1
MF_ERR_CUDA = -2
MF_ERR_OUT_OF_MEMORY = -3
MF_ERR_DIVERGED = -4
MF_ERR_TIMEOUT = -5
MF_ERR_UNSUPPORTED = -6

PREC = {"fp32": 0, "bf16": 1, "mixed": 2, "fp32_simt": 3, "f16": 4}
SCHEDULE = {"M": 0, "multiplicative": 0, "A": 1, "additive": 1}
QUERY = {"full": 0, "centre": 1, "center": 1}
OPTIMIZER = {"sgd": 0, "lamb": 1}
ENGINE = {"auto": 0, "gemm": 1}
ACTIVATION = {"tanh": 0, "gelu": 1}
LAUNCH = {"per_colour": 0, "graph": 1, "sweep": 2, "auto": 3}
LAUNCH_NAMES = {v: k for k, v in LAUNCH.items()}

# Every exported symbol the header declares (checked by the CPU test suite).
EXPORTS = ["mf_last_error", "mf_version", "mf_ctx_create", "mf_ctx_destroy", "mf_ctx_device", "mf_load_sdnet", "mf_load_sdnet_ex", "mf_free_sdnet", "mf_create_grid",
           "mf_destroy_grid", "mf_grid_dims", "mf_grid_upload", "mf_grid_download", "mf_sweep",
           "mf_residual", "mf_synchronize", "mf_sweep_noalloc", "mf_create_batch", "mf_destroy_batch",
           "mf_batch_info", "mf_batch_upload", "mf_batch_download", "mf_batch_sweep", "mf_batch_residual",
           "mf_create_trainer", "mf_destroy_trainer", "mf_trainer_set_weights", "mf_trainer_get_weights",
           "mf_trainer_get_grads", "mf_train_grad", "mf_train_step", "mf_check_wait_timeout"]


class MFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mosaicflow status {status}: {msg}")
        self.status = status


class SDNetDesc(C.Structure):
    _fields_ = [("width", C.c_int), ("depth", C.c_int)]


class SDNetDescEx(C.Structure):
    _fields_ = [("width", C.c_int), ("depth", C.c_int), ("activation", C.c_int),
                ("embed_channels", C.c_int), ("embed_kernel", C.c_int)]


class GridDesc(C.Structure):
    _fields_ = [("lx", C.c_int), ("ly", C.c_int)]


class SweepOpts(C.Structure):
    _fields_ = [("n_sweeps", C.c_int), ("schedule", C.c_int), ("precision", C.c_int),
                ("colours", C.c_int), ("eps", C.c_double), ("check_every", C.c_int),
                ("profile", C.c_int), ("eps_coarse", C.c_double), ("query", C.c_int), ("launch_mode", C.c_int)]


class SweepResult(C.Structure):
    _fields_ = [("sweeps_done", C.c_int), ("delta", C.c_double), ("kernel_launches", C.c_int),
                ("mlp_launches", C.c_int), ("ms_gather", C.c_double), ("ms_mlp", C.c_double),
                ("ms_reduce", C.c_double), ("sweeps_bf16", C.c_int), ("graph_sweeps", C.c_int),
                ("status", C.c_int), ("launch_mode", C.c_int), ("gather_block", C.c_int)]


class TrainDesc(C.Structure):
    _fields_ = [("width", C.c_int), ("depth", C.c_int), ("precision", C.c_int), ("optimizer", C.c_int),
                ("max_functions", C.c_int), ("max_points", C.c_int), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("weight_decay", C.c_float), ("engine", C.c_int)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> C.CDLL:
    """Load the library (once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libmosaicflow.so not found at {path}; run __graft_entry__.build() first")
    lib = C.CDLL(path)
    vp, i = C.c_void_p, C.c_int
    lib.mf_last_error.restype = C.c_char_p
    lib.mf_version.restype = i
    lib.mf_ctx_create.argtypes = [i, C.POINTER(vp)]
    lib.mf_ctx_destroy.argtypes = [vp]
    lib.mf_ctx_device.argtypes = [vp, C.POINTER(i), C.POINTER(i)]
    lib.mf_load_sdnet.argtypes = [vp, C.POINTER(SDNetDesc), vp, C.POINTER(vp)]
    lib.mf_load_sdnet_ex.argtypes = [vp, C.POINTER(SDNetDescEx), vp, C.POINTER(vp)]
    lib.mf_free_sdnet.argtypes = [vp]
    lib.mf_create_grid.argtypes = [vp, C.POINTER(GridDesc), vp, C.POINTER(vp)]
    lib.mf_destroy_grid.argtypes = [vp]
    lib.mf_grid_dims.argtypes = [vp, C.POINTER(i), C.POINTER(i)]
    lib.mf_grid_upload.argtypes = [vp, vp, i, vp]
    lib.mf_grid_download.argtypes = [vp, vp, i, vp]
    lib.mf_sweep.argtypes = [vp, vp, C.POINTER(SweepOpts), C.POINTER(SweepResult), vp]
    lib.mf_residual.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    lib.mf_synchronize.argtypes = [vp]
    lib.mf_sweep_noalloc.argtypes = [vp, i, i, vp, i, i, C.POINTER(C.c_double), vp]
    lib.mf_create_batch.argtypes = [vp, i, vp, vp, C.POINTER(vp)]
    lib.mf_destroy_batch.argtypes = [vp]
    lib.mf_batch_info.argtypes = [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(C.c_longlong)]
    lib.mf_batch_upload.argtypes = [vp, i, vp, i, vp]
    lib.mf_batch_download.argtypes = [vp, i, vp, i, vp]
    lib.mf_batch_sweep.argtypes = [vp, vp, C.POINTER(SweepOpts), C.POINTER(SweepResult), vp]
    lib.mf_batch_residual.argtypes = [vp, i, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    lib.mf_check_wait_timeout.argtypes = [C.c_double, C.POINTER(i)]
    lib.mf_create_trainer.argtypes = [vp, C.POINTER(TrainDesc), vp, C.POINTER(vp)]
    lib.mf_destroy_trainer.argtypes = [vp]
    lib.mf_trainer_set_weights.argtypes = [vp, vp, i, vp]
    lib.mf_trainer_get_weights.argtypes = [vp, vp, i, vp]
    lib.mf_trainer_get_grads.argtypes = [vp, vp, i, vp]
    lib.mf_train_grad.argtypes = [vp, i, i, i, vp, vp, vp, vp, C.POINTER(C.c_double), vp]
    lib.mf_train_step.argtypes = [vp, i, i, i, vp, vp, vp, vp, C.c_float, C.POINTER(C.c_double), vp]
    for name in EXPORTS:
        if name not in ("mf_last_error", "mf_version"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def _check(status: int):
    if status != MF_OK:
        raise MFError(status, load().mf_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _buffer(arr):
    """(pointer, on_device, nbytes) of a contiguous float32 NumPy array or torch tensor."""
    if isinstance(arr, np.ndarray):
        if arr.dtype != np.float32 or not arr.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float32 array")
        return arr.ctypes.data, 0, arr.nbytes
    import torch  # torch tensors: device memory or (pinned) host memory
    if arr.dtype != torch.float32 or not arr.is_contiguous():
        raise TypeError("expected a contiguous float32 tensor")
    return arr.data_ptr(), 1 if arr.is_cuda else 0, arr.numel() * 4


class Context:
    """mf_ctx_create / mf_ctx_destroy: the library bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        _check(load().mf_ctx_create(int(device), C.byref(self._h)))
        dev, sms = C.c_int(), C.c_int()
        _check(load().mf_ctx_device(self._h, C.byref(dev), C.byref(sms)))
        self.device, self.sm_count = dev.value, sms.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.mf_ctx_destroy(self._h)
            self._h = None


_CONTEXTS: dict = {}


def default_context(device: int | None = None) -> Context:
    """The context of `device` (default: torch's current CUDA device, else 0), created
    on first use and kept for the process."""
    if device is None:
        device = 0
        try:
            import torch
            if torch.cuda.is_available():
                device = torch.cuda.current_device()
        except ImportError:
            pass
    if device not in _CONTEXTS:
        _CONTEXTS[device] = Context(device)
    return _CONTEXTS[device]


def _ctx(ctx):
    return (ctx if ctx is not None else default_context())._h


class SDNet:
    """mf_load_sdnet / mf_load_sdnet_ex / mf_free_sdnet. activation "tanh" or "gelu";
    embed_channels > 0 adds the conv1d boundary embedding (kernel size embed_kernel)."""

    def __init__(self, weights: np.ndarray, width: int, depth: int, activation: str = "tanh",
                 embed_channels: int = 0, embed_kernel: int = 0, ctx: Context | None = None):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self.width, self.depth = width, depth
        self._h = C.c_void_p()
        if activation == "tanh" and embed_channels == 0:
            _check(load().mf_load_sdnet(_ctx(ctx), C.byref(SDNetDesc(width, depth)), w.ctypes.data,
                                        C.byref(self._h)))
        else:
            d = SDNetDescEx(width, depth, ACTIVATION[activation], embed_channels, embed_kernel)
            _check(load().mf_load_sdnet_ex(_ctx(ctx), C.byref(d), w.ctypes.data, C.byref(self._h)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.mf_free_sdnet(self._h)
            self._h = None


@dataclass
class SweepOutcome:
    sweeps_done: int
    delta: float
    kernel_launches: int = 0
    mlp_launches: int = 0
    ms_gather: float = 0.0
    ms_mlp: float = 0.0
    ms_reduce: float = 0.0
    sweeps_bf16: int = 0
    graph_sweeps: int = 0
    status: int = 0
    launch_mode: str = "per_colour"
    gather_block: int = 16


def _outcome(res) -> SweepOutcome:
    return SweepOutcome(res.sweeps_done, res.delta, res.kernel_launches, res.mlp_launches, res.ms_gather, res.ms_mlp,
                        res.ms_reduce, res.sweeps_bf16, res.graph_sweeps, res.status,
                        LAUNCH_NAMES.get(res.launch_mode, str(res.launch_mode)), res.gather_block)


class Grid:
    """mf_create_grid / mf_grid_* / mf_sweep / mf_residual for one problem."""

    def __init__(self, lx: int, ly: int, bc_ccw: np.ndarray, ctx: Context | None = None):
        bc = np.ascontiguousarray(bc_ccw, dtype=np.float64)
        self.lx, self.ly = lx, ly
        self.nx, self.ny = 32 * lx + 1, 32 * ly + 1
        if bc.size != 2 * (self.nx - 1) + 2 * (self.ny - 1):
            raise ValueError("bc_ccw has the wrong length")
        self._h = C.c_void_p()
        _check(load().mf_create_grid(_ctx(ctx), C.byref(GridDesc(lx, ly)), bc.ctypes.data, C.byref(self._h)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.mf_destroy_grid(self._h)
            self._h = None

    @property
    def shape(self):
        return (self.ny, self.nx)

    def upload(self, src, stream=None):
        ptr, dev, nbytes = _buffer(src)
        if nbytes != self.nx * self.ny * 4:
            raise ValueError("grid size mismatch")
        _check(load().mf_grid_upload(self._h, ptr, dev, _stream_ptr(stream)))

    def download(self, dst=None, stream=None, sync=True):
        if dst is None:
            dst = np.empty(self.shape, dtype=np.float32)
        ptr, dev, nbytes = _buffer(dst)
        if nbytes != self.nx * self.ny * 4:
            raise ValueError("grid size mismatch")
        _check(load().mf_grid_download(self._h, ptr, dev, _stream_ptr(stream)))
        if sync:
            synchronize(stream)
        return dst

    def sweep(self, net: SDNet, n_sweeps: int = 1, schedule: str = "M", precision: str = "fp32",
              colours: int = 0, eps: float = 0.0, check_every: int = 1, stream=None,
              profile: bool = False, eps_coarse: float = 0.0, query: str = "full",
              launch_mode: str = "per_colour") -> SweepOutcome:
        """launch_mode "per_colour" (gather + SDNet launch per colour) or "sweep" (one
        cooperative launch per BF16 sweep)."""
        opts = SweepOpts(n_sweeps, SCHEDULE[schedule], PREC[precision], colours, eps, check_every,
                         1 if profile else 0, eps_coarse, QUERY[query], LAUNCH[launch_mode])
        res = SweepResult()
        _check(load().mf_sweep(self._h, net._h, C.byref(opts), C.byref(res), _stream_ptr(stream)))
        return _outcome(res)

    def assemble(self, net: SDNet, precision: str = "fp32", stream=None) -> SweepOutcome:
        """Algorithm 2's final step after centre-line sweeps: every subdomain predicts all
        its interior points from the current boundaries and each point takes the average
        over the subdomains that hold it (one additive full sweep)."""
        return self.sweep(net, 1, "A", precision, stream=stream)

    def residual(self, stream=None):
        mx, rms = C.c_double(), C.c_double()
        _check(load().mf_residual(self._h, C.byref(mx), C.byref(rms), _stream_ptr(stream)))
        return mx.value, rms.value


class Batch:
    """mf_create_batch / mf_batch_*: many independent problems swept together."""

    def __init__(self, sizes, bcs, ctx: Context | None = None):
        self.n = len(sizes)
        descs = (GridDesc * self.n)(*[GridDesc(int(lx), int(ly)) for lx, ly in sizes])
        bc = np.ascontiguousarray(np.concatenate([np.asarray(b, dtype=np.float64) for b in bcs]))
        self.sizes = [(int(lx), int(ly)) for lx, ly in sizes]
        self._h = C.c_void_p()
        _check(load().mf_create_batch(_ctx(ctx), self.n, descs, bc.ctypes.data, C.byref(self._h)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.mf_destroy_batch(self._h)
            self._h = None

    def shape(self, q):
        lx, ly = self.sizes[q]
        return (32 * ly + 1, 32 * lx + 1)

    def upload(self, q, src, stream=None):
        ptr, dev, nbytes = _buffer(src)
        if nbytes != int(np.prod(self.shape(q))) * 4:
            raise ValueError("grid size mismatch")
        _check(load().mf_batch_upload(self._h, q, ptr, dev, _stream_ptr(stream)))

    def download(self, q, dst=None, stream=None, sync=True):
        if dst is None:
            dst = np.empty(self.shape(q), dtype=np.float32)
        ptr, dev, nbytes = _buffer(dst)
        if nbytes != int(np.prod(self.shape(q))) * 4:
            raise ValueError("grid size mismatch")
        _check(load().mf_batch_download(self._h, q, ptr, dev, _stream_ptr(stream)))
        if sync:
            synchronize(stream)
        return dst

    def sweep(self, net: SDNet, n_sweeps: int = 1, precision: str = "fp32", eps: float = 0.0,
              check_every: int = 1, query: str = "full", graph: bool = False, stream=None,
              launch_mode: str | None = None) -> SweepOutcome:
        """launch_mode: "per_colour", "graph", "sweep" (one cooperative launch per BF16
        sweep) or "auto" (autotuned at the first call); graph=True is "graph"."""
        mode = LAUNCH[launch_mode] if launch_mode is not None else (LAUNCH["graph"] if graph else 0)
        opts = SweepOpts(n_sweeps, 0, PREC[precision], 0, eps, check_every, 0, 0.0, QUERY[query], mode)
        res = SweepResult()
        _check(load().mf_batch_sweep(self._h, net._h, C.byref(opts), C.byref(res), _stream_ptr(stream)))
        return _outcome(res)

    def residual(self, q, stream=None):
        mx, rms = C.c_double(), C.c_double()
        _check(load().mf_batch_residual(self._h, q, C.byref(mx), C.byref(rms), _stream_ptr(stream)))
        return mx.value, rms.value


def sweep_noalloc(u, lx: int, ly: int, net: SDNet, n_sweeps: int = 1, precision: str = "fp32",
                  stream=None) -> float:
    """mf_sweep_noalloc on a caller-owned device grid `u` (a contiguous float32 CUDA
    tensor of shape (32 ly + 1, 32 lx + 1)), updated in place; returns delta."""
    ptr, on_dev, nbytes = _buffer(u)
    if not on_dev:
        raise TypeError("mf_sweep_noalloc needs a device grid")
    if nbytes != (32 * lx + 1) * (32 * ly + 1) * 4:
        raise ValueError("grid size mismatch")
    d = C.c_double()
    _check(load().mf_sweep_noalloc(ptr, lx, ly, net._h, PREC[precision], n_sweeps, C.byref(d), _stream_ptr(stream)))
    return d.value


def check_wait_timeout(limit_ms: float = 20.0):
    """mf_check_wait_timeout: run the bounded device waits against a phase that never
    completes; returns (status, waits_gave_up), (MF_ERR_TIMEOUT, 64) by design."""
    n = C.c_int()
    st = load().mf_check_wait_timeout(limit_ms, C.byref(n))
    return st, n.value


def synchronize(stream=None):
    """mf_synchronize: wait for the work enqueued on `stream` (None = default stream)."""
    _check(load().mf_synchronize(_stream_ptr(stream)))


class Trainer:
    """mf_create_trainer / mf_train_grad / mf_train_step: physics-informed SDNet training
    (Eq. 3, Algorithm 1) with the weights, gradient and optimiser state on the device."""

    def __init__(self, weights: np.ndarray, width: int, depth: int, precision: str = "bf16",
                 optimizer: str = "lamb", max_functions: int = 1024, max_points: int = 1024,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-6, weight_decay: float = 0.0,
                 engine: str = "auto", ctx: Context | None = None):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self.width, self.depth, self.n_params = width, depth, w.size
        d = TrainDesc(width, depth, PREC[precision], OPTIMIZER[optimizer], max_functions, max_points,
                      beta1, beta2, eps, weight_decay, ENGINE[engine])
        self._h = C.c_void_p()
        _check(load().mf_create_trainer(_ctx(ctx), C.byref(d), w.ctypes.data, C.byref(self._h)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.mf_destroy_trainer(self._h)
            self._h = None

    @staticmethod
    def _batch(G, Xc, Xb, Yb):
        F = G.shape[0]
        for name, t, shp in (("G", G, (F, 128)), ("Xc", Xc, (F, Xc.shape[1], 2)),
                             ("Xb", Xb, (F, Xb.shape[1], 2)), ("Yb", Yb, (F, Xb.shape[1]))):
            ptr, on_dev, _ = _buffer(t)
            if not on_dev:
                raise TypeError(f"{name} must be a CUDA tensor")
            if tuple(t.shape) != shp:
                raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {shp}")
        return F, Xc.shape[1], Xb.shape[1], G.data_ptr(), Xc.data_ptr(), Xb.data_ptr(), Yb.data_ptr()

    def grad(self, G, Xc, Xb, Yb, stream=None):
        """Loss (total, data, pde) of the batch; the gradient stays on the device."""
        F, Nc, Nb, g, xc, xb, yb = self._batch(G, Xc, Xb, Yb)
        loss = (C.c_double * 3)()
        _check(load().mf_train_grad(self._h, F, Nc, Nb, g, xc, xb, yb, loss, _stream_ptr(stream)))
        return tuple(loss)

    def step(self, G, Xc, Xb, Yb, lr: float, stream=None):
        """One training iteration: gradient, then the optimiser update; returns the loss."""
        F, Nc, Nb, g, xc, xb, yb = self._batch(G, Xc, Xb, Yb)
        loss = (C.c_double * 3)()
        _check(load().mf_train_step(self._h, F, Nc, Nb, g, xc, xb, yb, lr, loss, _stream_ptr(stream)))
        return tuple(loss)

    def _get(self, fn, dst, stream):
        if dst is None:
            dst = np.empty(self.n_params, dtype=np.float32)
        ptr, dev, nbytes = _buffer(dst)
        if nbytes != self.n_params * 4:
            raise ValueError("parameter vector size mismatch")
        _check(fn(self._h, ptr, dev, _stream_ptr(stream)))
        synchronize(stream)
        return dst

    def weights(self, dst=None, stream=None):
        return self._get(load().mf_trainer_get_weights, dst, stream)

    def grads(self, dst=None, stream=None):
        return self._get(load().mf_trainer_get_grads, dst, stream)

    def set_weights(self, src, stream=None):
        ptr, dev, nbytes = _buffer(src)
        if nbytes != self.n_params * 4:
            raise ValueError("parameter vector size mismatch")
        _check(load().mf_trainer_set_weights(self._h, ptr, dev, _stream_ptr(stream)))


def pinn_loss(weights, trainer: Trainer, G, Xc, Xb, Yb):
    """L = L_data + L_pde (Eq. 3) as a differentiable function of the packed FP32 weight
    tensor (on the GPU): the forward pass and the gradient both come from mf_train_grad."""
    return _pinn_function().apply(weights, trainer, G, Xc, Xb, Yb)


_PINN_FN = None


def _pinn_function():
    global _PINN_FN
    if _PINN_FN is None:
        import torch

        class PinnLoss(torch.autograd.Function):
            @staticmethod
            def forward(ctx, weights, trainer, G, Xc, Xb, Yb):
                stream = torch.cuda.current_stream(weights.device)
                w = weights.detach().contiguous()
                trainer.set_weights(w, stream)
                total, _, _ = trainer.grad(G, Xc, Xb, Yb, stream)
                ctx.save_for_backward(trainer.grads(torch.empty_like(w), stream))
                return weights.new_tensor(total)

            @staticmethod
            def backward(ctx, gout):
                (g,) = ctx.saved_tensors
                return gout * g, None, None, None, None, None

        _PINN_FN = PinnLoss
    return _PINN_FN
