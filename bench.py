#!/usr/bin/env python
"""Benchmark: Mosaic Flow predictor sweeps on one GB300 (or N independent replicas).

Workload (default): global domain [0,64]^2, 127 x 127 = 16,129 unit subdomains at half
overlap, grid 2049 x 2049, SDNet 6 x 128 tanh (Xavier-uniform, seed 2), 8-mode harmonic
Dirichlet data (seed 2): the strong-scaling domain shape of the paper (4096 atomic
subdomains per colour) at 4096x the subdomain area.

One step = one multiplicative sweep: for each of the four colours, the boundary gather
and the SDNet on all 961 interior points of every subdomain of the colour with the
scatter into the grid, then the FP64 delta/residual reduction. `value` is BF16
point-evaluations/s with the grid resident on the device; the FP32 path on the same
workload is reported beside it. L2 is flushed (a 256 MiB write) between timed steps,
outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own replica (no data-path collective);
value = all ranks' point-evaluations / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MF sweep point-evals/s, BF16 vs FP32 at <=1e-3 err; PINN train steps/s"
UNIT = "point-evals/s"
FLOP_PER_EVAL = 5 * 2 * 128 * 128 + 2 * 128  # hidden H x H layers + output, per point
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}

# DRAM traffic of one SDNet (tensor-core) launch from an ncu capture, valid only while
# the kernel source is unchanged (keyed by the source hash).
NCU_TRAFFIC = {
    # ncu --set full, colour 2 of the L = 64 grid: dram__bytes_read 2.640 MB + write 0.316 MB
    "81be73928d336f0a": 2955776,
}
# The unit that bounds the same kernel, from the same capture: the MUFU pipe (tanh),
# sm__pipe_xu_cycles_active of elapsed; the tanh floor is 98,304 tanh per 128-row tile
# at 16 per clock per SM.
NCU_MUFU_BUSY = {
    "81be73928d336f0a": 0.6912,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget")
    ap.add_argument("--L", type=int, default=64, help="domain side in unit subdomains (64 = the benchmark workload; "
                                                      "smaller values only for profiling captures)")
    ap.add_argument("--fp32-steps", type=int, default=-1)
    ap.add_argument("--e2e-steps", type=int, default=-1)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-variant", action="store_true")
    ap.add_argument("--no-converged", action="store_true")
    ap.add_argument("--train-functions", type=int, default=1024,
                    help="functions in the training batch (1024 = the benchmark workload; fewer only for "
                         "profiling captures)")
    ap.add_argument("--train-only", action="store_true",
                    help="run only the training-step measurement and print its JSON object (profiling aid)")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched-workload measurement and print its JSON object (profiling aid)")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda_ok() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_rate(units_per_rank: float, local_seconds: float, world: int) -> float:
    """Whole-job rate of N replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(local_seconds, world)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s >= 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ helpers

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def blas_threads():
    """Threads the oracle's BLAS uses (OpenBLAS query where available)."""
    import ctypes
    import re
    try:
        maps = open("/proc/self/maps").read()
        for lib in sorted(set(re.findall(r"(/\S*openblas\S*\.so\S*)", maps))):
            h = ctypes.CDLL(lib)
            for name in ("scipy_openblas_get_num_threads64_", "scipy_openblas_get_num_threads",
                         "openblas_get_num_threads64_", "openblas_get_num_threads"):
                f = getattr(h, name, None)
                if f is not None:
                    return int(f())
    except Exception:
        pass
    return os.cpu_count()


def source_hash():
    """Hash of the tensor-core SDNet kernel's sources (the kernel and its headers)."""
    h = hashlib.sha256()
    for name in ("mf_mlp_bf16.cu", "mf_tc.cuh", "mf_wait.cuh", "mf_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2308_14258_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------ CPU oracle sample

def oracle_sample(seconds: float, u_state=None, return_values=False, chunk=256):
    """Time the FP64 oracle on whole subdomains of the large workload (colour 0): the
    boundary gather, the batched SDNet on all 961 interior points and the write-back,
    in batches of `chunk` subdomains until about `seconds` have passed."""
    import numpy as np
    from oracle import mosaic_flow as orc
    from paper_2308_14258_gb300 import inputs as I
    w = I.large()
    p = w.problems[0]
    P = orc.unpack_sdnet(w.weights(), 128, 6)
    u = orc.make_grid(p.lx, p.ly, p.bc) if u_state is None else u_state.astype(np.float64)
    subs = orc.subdomains_of_colour(p.lx, p.ly, 0)
    X = orc.interior_coords()
    uu = u.copy()
    done, Vs = 0, []
    t0 = time.perf_counter()
    n = 8
    while done < len(subs):
        batch = subs[done:done + n]
        G = np.stack([orc.gather(u, a, b) for (a, b) in batch])
        V = orc.sdnet_batched(P, G, X)
        for (a, b), v in zip(batch, V):
            orc.write_interior(uu, a, b, v)
        if return_values:
            Vs.append(V)
        done += len(batch)
        n = chunk
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    out = {"evals": done * orc.N_INT, "seconds": dt, "subdomains": done,
           "value": done * orc.N_INT / dt, "threads": blas_threads()}
    if return_values:
        out["V"], out["subs"] = np.concatenate(Vs), subs[:done]
    return out


def run_reference(args, world, rank):
    """The oracle as the reference arm: K timed bounded samples on the host cores."""
    if rank != 0:
        return
    samples = []
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(budget / 4)
    tot_e, tot_t = 0, 0.0
    for _ in range(args.steps):
        s = oracle_sample(budget)
        tot_e += s["evals"]
        tot_t += s["seconds"]
        samples.append(s)
    v = tot_e / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "large_L64: 2049x2049 grid, 16129 subdomains, SDNet 6x128 tanh",
                                         "precision": "fp64 oracle (numpy)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": samples[-1]["threads"], "kind": "oracle",
                         "sample": f"{samples[-1]['subdomains']} whole subdomains of colour 0 per step "
                                   f"(gather + SDNet on 961 points + write), FP64 NumPy"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm

def train_tile_traffic(F, Nc, Nb, NH):
    """Algorithmic HBM bytes of one fused training step: a layer's activations (or
    gradients) are one buffer of 32 KB tiles of 128 GEMM rows (four Taylor channels of
    32 collocation points, or 128 data points). Each two-layer forward launch reads
    A_{l-1} and writes A_l, A_{l+1} (3 passes, for hidden layers 1..NH-1), a single-layer
    one reads and writes one (2); the first of them forms A_0 on chip and writes it
    instead of reading it (3), and only with one hidden layer does a first-layer kernel
    write A_0 (1 pass) for a forward launch to read. The top backward reads A_{NH-1} and
    writes gA (2); each hidden backward layer reads A_{l-1}, gA_l and writes gA_{l-1} (3,
    layers NH-1..2); layer 1 reads A_0 and gA_1 (2)."""
    tiles = 4 * F * Nc // 128 + (F * Nb + 127) // 128
    buf = tiles * 32 * 1024
    fwd = 3 * ((NH - 1) // 2) + (2 if (NH - 1) % 2 else 0) + (0 if NH >= 3 else 1)
    passes = fwd + 2 + 3 * (NH - 2) + 2
    return passes * buf


def measure_converged(m, I, torch, np, net, p, weights, stream, rank, with_oracle):
    """Algorithm 2's loop to convergence on the benchmark grid from the zero interior.

    * fp32: FP32 sweeps alone until delta < 1e-5;
    * mixed: MF_PREC_MIXED, BF16 sweeps until delta < 1e-2 or until a BF16 sweep stops
      reducing delta (its rounding floor, about 1.2e-2 on this grid), then FP32 sweeps
      until delta < 1e-5;
    * bf16: BF16 sweeps alone (40, well past their plateau);
    * f16: F16 sweeps alone (MF_PREC_F16, 40), the other 16-bit type on the same kernel.
    The stop value 1e-5 lies above the FP32 rounding floor of delta on this grid
    (about 1.5e-6). Each field is compared with the FP32 fixed point (FP32 sweeps to
    250, where delta sits at its floor), as max |u - u_ref| / max |u_ref|.
    to_1e-3: the same iterations one sweep at a time, the error against the fixed point
    taken on the device after every sweep; the sweeps each needs until the field is
    within 1e-3 (the target), and that many sweeps at the timed per-sweep cost."""
    res, fields = {}, {}
    # the FP32 fixed point first
    g = m.Grid(p.lx, p.ly, p.bc)
    o = g.sweep(net, 250, "M", "fp32", check_every=25, stream=stream)
    ref_t = torch.empty((g.ny, g.nx), dtype=torch.float32, device="cuda")
    g.download(ref_t, stream=stream)
    ref = ref_t.double().cpu().numpy()
    del g
    scale = float(np.abs(ref).max())
    res["reference"] = {"what": "FP32 sweeps to 250 from the zero interior", "delta": o.delta}
    runs = (("fp32", "fp32", 400, 1e-5, 0.0), ("mixed", "mixed", 400, 1e-5, 1e-2), ("bf16", "bf16", 40, 0.0, 0.0),
            ("f16", "f16", 40, 0.0, 0.0))
    for name, prec, n, eps, eps_c in runs:
        g = m.Grid(p.lx, p.ly, p.bc)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = g.sweep(net, n, "M", prec, eps=eps, eps_coarse=eps_c, stream=stream)
        e1.record(stream)
        e1.synchronize()
        fields[name] = g.download(stream=stream).astype(np.float64)
        n16 = o.sweeps_done if prec == "f16" else 0
        res[name] = {"sweeps": o.sweeps_done, "sweeps_bf16": o.sweeps_bf16, "sweeps_f16": n16,
                     "sweeps_fp32": o.sweeps_done - o.sweeps_bf16 - n16, "delta": o.delta,
                     "ms": e0.elapsed_time(e1),
                     "max_rel_err_vs_fp32_fixed_point": float(np.abs(fields[name] - ref).max() / scale)}
        del g
    res["speedup_mixed_over_fp32"] = res["fp32"]["ms"] / res["mixed"]["ms"]

    # sweeps to a field within 1e-3 of the fixed point
    def sweep_ms(prec):
        g = m.Grid(p.lx, p.ly, p.bc)
        g.sweep(net, 1, "M", prec, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.sweep(net, 4, "M", prec, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 4
    t32, t16, th = sweep_ms("fp32"), sweep_ms("bf16"), sweep_ms("f16")
    cur = torch.empty_like(ref_t)

    def err_now(g):
        g.download(cur, stream=stream)
        with torch.cuda.stream(stream):
            e = float((cur - ref_t).abs().max()) / scale
        return e

    to = {"target": 1e-3, "ms_per_sweep": {"fp32": t32, "bf16": t16, "f16": th}}
    g = m.Grid(p.lx, p.ly, p.bc)
    n32 = None
    for k in range(1, 201):
        g.sweep(net, 1, "M", "fp32", stream=stream)
        if err_now(g) <= 1e-3:
            n32 = k
            break
    to["fp32"] = {"sweeps": n32, "ms": n32 * t32 if n32 else None}
    g = m.Grid(p.lx, p.ly, p.bc)
    nb, prev_d, e_bf16 = 0, float("inf"), None
    for k in range(1, 61):  # BF16 until a sweep no longer reduces delta (the MIXED rule)
        d = g.sweep(net, 1, "M", "bf16", stream=stream).delta
        nb = k
        if d < 1e-2 or d >= prev_d:
            break
        prev_d = d
    e_bf16 = err_now(g)
    nf = 0
    if e_bf16 > 1e-3:
        for k in range(1, 201):
            g.sweep(net, 1, "M", "fp32", stream=stream)
            if err_now(g) <= 1e-3:
                nf = k
                break
    to["mixed"] = {"sweeps_bf16": nb, "err_after_bf16": e_bf16, "sweeps_fp32": nf,
                   "ms": nb * t16 + nf * t32}
    if to["fp32"]["ms"] and to["mixed"]["ms"]:
        to["speedup_mixed_over_fp32"] = to["fp32"]["ms"] / to["mixed"]["ms"]
    # F16 sweeps alone
    g = m.Grid(p.lx, p.ly, p.bc)
    nh = None
    for k in range(1, 61):
        g.sweep(net, 1, "M", "f16", stream=stream)
        if err_now(g) <= 1e-3:
            nh = k
            break
    to["f16"] = {"sweeps": nh, "ms": nh * th if nh else None}
    if to["fp32"]["ms"] and to["f16"]["ms"]:
        to["speedup_f16_over_fp32"] = to["fp32"]["ms"] / to["f16"]["ms"]
    del g
    res["to_1e-3"] = to
    res["workload"] = "large_L64 grid from the zero interior, SDNet 6x128 (seed 2), multiplicative schedule"
    res["stop"] = ("delta < 1e-5 (Algorithm 2); MIXED switches from BF16 to FP32 at delta < 1e-2 or when a BF16 "
                   "sweep no longer reduces delta")
    if with_oracle and rank == 0:
        # fixed-point residual of the MIXED field under the FP64 oracle's map: at a
        # multiplicative fixed point, each last-colour subdomain's prediction from the
        # field's own boundary values reproduces its interior
        from oracle import mosaic_flow as orc
        u = fields["mixed"]
        solver = orc.Solver(orc.unpack_sdnet(weights, 128, 6))
        subs = orc.subdomains_of_colour(p.lx, p.ly, 3)
        pick = [subs[i] for i in np.random.default_rng(1).choice(len(subs), 24, replace=False)]
        V = solver.solve_batch(np.stack([orc.gather(u, a, b) for (a, b) in pick]))
        e = max(float(np.abs(u[16 * b + 1:16 * b + 32, 16 * a + 1:16 * a + 32].ravel() - v).max())
                for (a, b), v in zip(pick, V))
        res["mixed"]["oracle_fixed_point_residual"] = e / scale
        res["mixed"]["oracle_check"] = ("24 sampled colour-3 subdomains: FP64 oracle prediction from the converged "
                                        "field's boundary vs its interior, max abs / max |u|")
    return res


def measure_batched(m, I, torch, stream):
    """The batched workload: 256 problems of sides 2..32 units (seed 4), BF16, one gather
    and one SDNet launch per colour over all problems; plain launches and graph replay."""
    wl = I.batched(256)
    bnet = m.SDNet(wl.weights(), 128, 6)
    bt = m.Batch([(p.lx, p.ly) for p in wl.problems], [p.bc for p in wl.problems])
    b_evals = sum((2 * p.lx - 1) * (2 * p.ly - 1) for p in wl.problems) * 961
    bt.sweep(bnet, 2, "bf16", stream=stream)  # warm-up (uncaptured)
    res = {}
    for mode in ("plain", "graph"):
        kb = 4
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = bt.sweep(bnet, kb, "bf16", graph=(mode == "graph"), check_every=kb, stream=stream)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        res[mode] = {"value": b_evals * kb / t, "ms_per_sweep": 1e3 * t / kb, "graph_sweeps": o.graph_sweeps}
    batched = {"workload": "256 problems, sides uniform in {2,4,8,16,32} units (seed 4), 8-mode BC seed 1000+q, "
                           "SDNet 6x128 BF16; grids 287 MB (> L2)",
               "unit": UNIT, "evals_per_sweep": b_evals, **res}
    del bt
    return batched


def measure_train(args, m, I, torch, np, stream, rank):
    """Training-step measurement (Eq. 3, Algorithm 1): BF16 fused engine (the reported
    value), FP32 and the BF16 GEMM engine for comparison, and the BF16 gradient error
    against the FP64 oracle on sampled functions."""
    # physics-informed training step (Eq. 3, Algorithm 1): 1024 functions x (1024 collocation
    # + 128 boundary points), SDNet 6x128, BF16, LAMB; ~8 GB working set (> L2)
    F, Nc, Nb, H, NH = args.train_functions, 1024, 128, 128, 5
    tb = I.training_batch(F, Nc, 3)
    tdev = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
            for a in (tb.G, tb.Xc, tb.Xb, tb.Yb)]
    tr = m.Trainer(I.xavier_sdnet(I.SDNetShape(H, NH + 1), 4), H, NH + 1, "bf16", "lamb",
                   max_functions=F, max_points=Nc)
    for _ in range(3):
        first_loss = tr.step(*tdev, 1e-3, stream=stream)[0]
    kt = max(3, min(args.steps, 10))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(kt + 1)]
    ev[0].record(stream)
    for i in range(kt):
        last_loss = tr.step(*tdev, 1e-3, stream=stream)[0]
        ev[i + 1].record(stream)
    ev[-1].synchronize()
    t = ev[0].elapsed_time(ev[-1]) / 1e3
    step_ms = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(kt))
    e0, e1 = ev[0], ev[-1]  # reused below for the comparison engines
    # layer-GEMM flops: forward 2 H^2 per channel and layer, backward twice that;
    # 4 Taylor channels per collocation point, 1 channel per data point
    gemm_flop = 3 * 2 * H * H * NH * (4 * F * Nc + F * Nb)
    train = {"value": kt / t, "unit": "train steps/s", "ms_per_step": 1e3 * t / kt,
             "step_ms_median": step_ms[kt // 2], "step_ms_max": step_ms[-1],
             "workload": f"{F} functions (8-mode harmonic, seed 3) x ({Nc} collocation + {Nb} boundary points), "
                         "SDNet 6x128 tanh, BF16, fused tensor-core layer kernels (Taylor-mode forward, "
                         "recomputing backward), LAMB",
             "gemm_tflop_per_step": gemm_flop / 1e12, "gemm_tflops_achieved": gemm_flop * kt / t / 1e12,
             "loss_after_warmup": first_loss, "loss_last": last_loss,
             "l2": f"working set ~{8.0 * F / 1024:.1f} GB (> L2)"}
    peaks, psrc = load_peaks()
    tpeak = peaks.get("bf16_tflops")
    traffic = train_tile_traffic(F, Nc, Nb, NH)
    hpeak = peaks.get("hbm_gbs")
    achieved_gbs = traffic / (t / kt) / 1e9
    # the fused engine moves 19 passes of its 1.1 GB tile buffer per step (activation and
    # gradient tiles between layers): the step is bound by HBM, the layer GEMMs keep the
    # tensor pipe a quarter busy
    train["roofline"] = {"bound": "hbm", "achieved": achieved_gbs, "peak": hpeak, "unit": "GB/s",
                         "frac": achieved_gbs / hpeak, "traffic": None,
                         "peak_source": f"{psrc} hbm_gbs",
                         "note": "whole step: algorithmic tile bytes (tile_bytes_per_step) / step time; ncu DRAM "
                                 "counters on a 256-function batch show each layer kernel moving its algorithmic "
                                 "bytes (profiles/train_bf16_F256_ncu_mem.md)",
                         "tile_bytes_per_step": traffic,
                         "tensor": {"achieved": train["gemm_tflops_achieved"], "peak": tpeak, "unit": "TFLOP/s",
                                    "frac": train["gemm_tflops_achieved"] / tpeak,
                                    "peak_source": f"{psrc} bf16_tflops (burst: the timed region is "
                                                   f"{1e3 * t:.0f} ms)"}}
    del tr
    torch.cuda.empty_cache()
    # FP32 mode on the same batch (the GEMM engine's FP32 layer GEMMs), fewer steps
    tr = m.Trainer(I.xavier_sdnet(I.SDNetShape(H, NH + 1), 4), H, NH + 1, "fp32", "lamb",
                   max_functions=F, max_points=Nc)
    tr.step(*tdev, 1e-3, stream=stream)
    k32t = 3
    e0.record(stream)
    for _ in range(k32t):
        tr.step(*tdev, 1e-3, stream=stream)
    e1.record(stream)
    e1.synchronize()
    t32 = e0.elapsed_time(e1) / 1e3
    train["fp32"] = {"value": k32t / t32, "unit": "train steps/s", "ms_per_step": 1e3 * t32 / k32t,
                     "engine": "GEMM engine: FP32 SIMT layer GEMMs + elementwise kernels"}
    del tr
    torch.cuda.empty_cache()
    tr = m.Trainer(I.xavier_sdnet(I.SDNetShape(H, NH + 1), 4), H, NH + 1, "bf16", "lamb",
                   max_functions=F, max_points=Nc, engine="gemm")
    tr.step(*tdev, 1e-3, stream=stream)
    e0.record(stream)
    for _ in range(k32t):
        tr.step(*tdev, 1e-3, stream=stream)
    e1.record(stream)
    e1.synchronize()
    tg = e0.elapsed_time(e1) / 1e3
    train["bf16_gemm_engine"] = {"value": k32t / tg, "unit": "train steps/s", "ms_per_step": 1e3 * tg / k32t,
                                 "engine": "GEMM engine: BF16 operands, FP32 SIMT layer GEMMs + elementwise kernels"}
    del tr, tdev
    torch.cuda.empty_cache()
    # BF16 gradient against the FP64 oracle on 4 sampled functions (full Nc)
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import pinn
        sl = slice(0, 4)
        small = [np.ascontiguousarray(a[sl], dtype=np.float32) for a in (tb.G, tb.Xc, tb.Xb, tb.Yb)]
        w0 = I.xavier_sdnet(I.SDNetShape(H, NH + 1), 4)
        (lt, ld, lp), gref = pinn.loss_and_grads(w0.astype(np.float64), H, NH + 1,
                                                 *[a.astype(np.float64) for a in small])
        tr = m.Trainer(w0, H, NH + 1, "bf16", "sgd", max_functions=4, max_points=Nc)
        lo = tr.grad(*[torch.from_numpy(a).cuda() for a in small])
        g = tr.grads().astype(np.float64)
        train["err_vs_oracle_bf16"] = {
            "functions": "0..3 of the batch, initial weights",
            "grad_rel_l2": float(np.linalg.norm(g - gref) / np.linalg.norm(gref)),
            "loss_data_rel": abs(lo[1] - ld) / ld, "rms_laplacian_rel": abs(math.sqrt(lo[2]) - math.sqrt(lp)) / math.sqrt(lp)}
        del tr
    return train


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_14258_gb300 import inputs as I
    from paper_2308_14258_gb300 import mosaicflow as m

    w = I.large()
    p = w.problems[0]
    if args.L != 64:
        p = I.Problem(args.L, args.L, I.bc_values(args.L, args.L, I.mode_field(I.mode_coeffs(2), args.L, args.L)))
        args.no_cpu_baseline = True
    weights = w.weights()
    net = m.SDNet(weights, 128, 6)
    grid = m.Grid(p.lx, p.ly, p.bc)
    n_sub = (2 * p.lx - 1) * (2 * p.ly - 1)
    evals_per_sweep = n_sub * 961
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if args.train_only:
        print(json.dumps({"train": measure_train(args, m, I, torch, np, stream, rank)}))
        return
    if args.batched_only:
        print(json.dumps({"batched": measure_batched(m, I, torch, stream)}))
        return

    def timed_steps(prec, k, profile=True):
        ms, mlp_ms, mlp_launch, launches = [], 0.0, 0, 0
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = grid.sweep(net, 1, "M", prec, stream=stream, profile=profile)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            mlp_ms += out.ms_mlp
            mlp_launch += out.mlp_launches
            launches += out.kernel_launches
        return ms, mlp_ms, mlp_launch, launches

    # warm-up (both precisions), then the timed BF16 region with clocks sampled
    for _ in range(args.warmup):
        grid.sweep(net, 1, "M", "bf16", stream=stream)
    grid.sweep(net, 1, "M", "fp32", stream=stream)
    grid.sweep(net, 1, "M", "f16", stream=stream)
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    barrier(world)
    sampler.start()
    ms, mlp_ms, mlp_launch, launches = timed_steps("bf16", args.steps)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    value = aggregate_rate(evals_per_sweep * args.steps, sum(ms) / 1e3, world)
    total_s = world * evals_per_sweep * args.steps / value

    # FP32 paths on the same workload: MF_PREC_FP32 (split-F16 tensor cores) and the
    # SIMT kernel (fewer steps: ~16x slower than BF16)
    k32 = max(3, args.steps // 4) if args.fp32_steps < 0 else args.fp32_steps
    ms32, mlp32, mlp32_launch, _ = timed_steps("fp32", k32)
    fp32_value = evals_per_sweep * k32 / (sum(ms32) / 1e3) if k32 > 0 else None
    ks = 2 if args.fp32_steps < 0 else min(2, args.fp32_steps)
    ms32s, _, _, _ = timed_steps("fp32_simt", ks)
    # the F16 path (the same kernel with the other 16-bit operand type)
    kh = max(3, args.steps // 4)
    msh, mlph, mlph_launch, _ = timed_steps("f16", kh)
    f16_value = evals_per_sweep * kh / (sum(msh) / 1e3)
    fp32_simt_value = evals_per_sweep * ks / (sum(ms32s) / 1e3) if ks > 0 else None

    # centre-line (interface-only) sweeps of the same grid: Algorithm 2's per-iteration work
    k_c = max(3, min(args.steps, 10))
    cl_ms = []
    for _ in range(k_c):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        grid.sweep(net, 1, "M", "bf16", stream=stream, query="centre")
        e1.record(stream)
        e1.synchronize()
        cl_ms.append(e0.elapsed_time(e1))
    n_sub_c = n_sub * 61

    # the batched workload: 256 problems of sides 2..32 units, one SDNet launch per colour
    batched = measure_batched(m, I, torch, stream) if (args.L == 64 and not args.no_batched) else None

    # launch modes of a sweep (per colour, graph replay, one whole-sweep cooperative
    # launch, autotuned) on the large grid and on a batch of 256 small problems (L = 2)
    modes = None
    if args.L == 64 and not args.no_batched:
        def per_sweep(fn, k):
            fn()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / k
        modes = {"unit": "ms per sweep", "large_L64": {}, "small_256xL2": {}}
        for mode in ("per_colour", "sweep"):
            modes["large_L64"][mode] = per_sweep(
                lambda: grid.sweep(net, 1, "M", "bf16", stream=stream, launch_mode=mode), 10)
        sizes = [(2, 2)] * 256
        sb = m.Batch(sizes, [I.bc_values(2, 2, I.mode_field(I.mode_coeffs(1000 + q), 2, 2)) for q in range(256)])
        for mode in ("per_colour", "graph", "sweep", "auto"):
            r = sb.sweep(net, 2, "bf16", launch_mode=mode, stream=stream)
            modes["small_256xL2"][mode] = per_sweep(
                lambda: sb.sweep(net, 20, "bf16", launch_mode=mode, check_every=20, stream=stream), 3) / 20
            if mode == "auto":
                modes["small_256xL2"]["auto_choice"] = {"launch_mode": r.launch_mode, "gather_block": r.gather_block}
        del sb

    # the paper's SDNet variant (Section 3.1): conv1d boundary embedding (8 channels,
    # kernel 5) + GELU, 6 x 128, on the same grid
    variant = None
    if args.L == 64 and not args.no_variant:
        vshape = I.SDNetShape(128, 6, "gelu", 8, 5)
        vnet = m.SDNet(I.xavier_sdnet(vshape, 2), 128, 6, "gelu", 8, 5)
        variant = {"workload": "large_L64 grid, SDNet 6x128 GELU with a circular conv1d boundary embedding "
                               "(8 channels, kernel 5; Xavier seed 2)", "unit": UNIT}
        for prec, kv in (("bf16", max(3, min(args.steps, 10))), ("fp32", 2)):
            vgrid = m.Grid(p.lx, p.ly, p.bc)
            vgrid.sweep(vnet, 2, "M", prec, stream=stream)
            vms = []
            for _ in range(kv):
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vgrid.sweep(vnet, 1, "M", prec, stream=stream)
                e1.record(stream)
                e1.synchronize()
                vms.append(e0.elapsed_time(e1))
            variant[prec] = {"value": evals_per_sweep * kv / (sum(vms) / 1e3), "ms_per_sweep": sum(vms) / kv}
            del vgrid
        del vnet

    train = measure_train(args, m, I, torch, np, stream, rank) if (args.L == 64 and not args.no_train) else None
    converged = None
    if args.L == 64 and not args.no_converged:
        converged = measure_converged(m, I, torch, np, net, p, weights, stream, rank, not args.no_cpu_baseline)

    # end to end through the public API: pinned host grid -> upload -> sweep -> download
    host_in = torch.empty(grid.shape, dtype=torch.float32).pin_memory()
    host_out = torch.empty(grid.shape, dtype=torch.float32).pin_memory()
    grid.download(host_in, stream=stream)
    k_e2e = max(3, min(args.steps, 10)) if args.e2e_steps < 0 else max(1, args.e2e_steps)
    e2e_ms = []
    for _ in range(k_e2e):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        grid.upload(host_in, stream=stream)
        grid.sweep(net, 1, "M", "bf16", stream=stream)
        grid.download(host_out, stream=stream, sync=True)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = aggregate_rate(evals_per_sweep * k_e2e, sum(e2e_ms) / 1e3, world)
    nbytes = grid.nx * grid.ny * 4

    # accuracy of this run's BF16 sweep against the FP64 oracle on sampled subdomains,
    # and of the GPU's delta and residual (FP32 per point, FP64 sums) against the
    # oracle's FP64 values on the same grids
    err = None
    cpu = None
    norms = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import mosaic_flow as orc
        before = grid.download().astype(np.float64)
        o1 = grid.sweep(net, 1, "M", "bf16", stream=stream)
        after1 = grid.download().astype(np.float64)
        r_max, r_rms = grid.residual(stream=stream)
        d_ref = orc.delta(after1, before)
        o_max, o_rms = orc.residual(after1)
        norms = {"delta": o1.delta, "delta_rel_err_vs_fp64": abs(o1.delta - d_ref) / d_ref,
                 "residual_max": r_max, "residual_max_rel_err_vs_fp64": abs(r_max - o_max) / o_max,
                 "residual_rms": r_rms, "residual_rms_rel_err_vs_fp64": abs(r_rms - o_rms) / o_rms,
                 "how": "GPU reduction (FP32 per point with error-free residual sums, FP64 accumulation) against "
                        "the FP64 oracle on the same two grids"}
        state = grid.download()
        grid.sweep(net, 1, "M", "bf16", colours=1, stream=stream)
        after = grid.download()
        cpu = oracle_sample(args.cpu_seconds, u_state=state, return_values=True)
        scale = float(np.abs(state).max())
        e = 0.0
        for (a, b), v in zip(cpu["subs"], cpu["V"]):
            blk = after[16 * b + 1:16 * b + 32, 16 * a + 1:16 * a + 32].astype(np.float64).ravel()
            e = max(e, float(np.abs(blk - v).max()))
        err = e / scale

    peaks, peak_src = load_peaks()
    # the timed region is well under a second: the burst peak applies
    peak = peaks.get("bf16_tflops")
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    per_launch_ms = mlp_ms / max(1, mlp_launch)
    flops_per_launch = evals_per_sweep * FLOP_PER_EVAL / 4.0
    achieved = flops_per_launch / (per_launch_ms / 1e3) / 1e12
    h = source_hash()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": (f"large_L64: [0,64]^2, 127x127=16129 subdomains, grid 2049x2049, "
                                "SDNet 6x128 tanh (Xavier seed 2), 8-mode harmonic BC seed 2") if args.L == 64
                   else f"profiling case L={args.L} (not the benchmark workload)",
                   "schedule": "multiplicative 4-colour", "step": "one sweep + FP64 delta/residual",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "evals_per_step": evals_per_sweep * world,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "sweeps_per_s": world * args.steps / total_s,
        "fp32": {"value": fp32_value, "unit": UNIT, "ms_per_step": sum(ms32) / k32 if k32 else None,
                 "kernel": "mlp_f32tc_kernel: hidden products as three F16 tcgen05 products, FP32 accumulation",
                 "per_launch_ms": mlp32 / max(1, mlp32_launch),
                 "fp32_tflops_algorithmic": (evals_per_sweep * FLOP_PER_EVAL / 4.0) / (mlp32 / max(1, mlp32_launch) / 1e3) / 1e12
                 if mlp32_launch else None,
                 "speedup_bf16_over_fp32": value / world / fp32_value if fp32_value else None},
        "fp32_simt": {"value": fp32_simt_value, "unit": UNIT, "ms_per_step": sum(ms32s) / ks if ks else None,
                      "kernel": "mlp_fp32_kernel: FFMA and tanhf on the CUDA cores"},
        "f16": {"value": f16_value, "unit": UNIT, "ms_per_step": sum(msh) / kh, "per_launch_ms": mlph / max(1, mlph_launch),
                "kernel": "mlp_bf16_kernel with F16 operands (MF_PREC_F16): same MMAs, 11-bit significands"},
        "err_vs_oracle_bf16_sweep": err,
        "convergence_norms": norms,
        "centre_lines": {"sweeps_per_s": 1e3 * k_c / sum(cl_ms), "ms_per_sweep": sum(cl_ms) / k_c,
                         "point_evals_per_sweep": n_sub_c, "unit": "sweeps/s",
                         "note": "interface-only sweeps (61 centre-cross points per subdomain, Algorithm 2)"},
        "batched": batched,
        "train": train,
        "variant_conv1d_gelu": variant,
        "converged": converged,
        "launch_modes": modes,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "roofline": {"kernel": "mlp_bf16_kernel<128,5,tanh>", "bound": "tensor", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": f"{peak_src} bf16_tflops (burst; timed region {sum(ms):.0f} ms)",
                     "traffic": NCU_TRAFFIC.get(h), "per_launch_ms": per_launch_ms,
                     "flops_per_launch": flops_per_launch,
                     "limiter": {"unit": "MUFU (tanh.approx)", "busy_frac_ncu": NCU_MUFU_BUSY.get(h),
                                 "tanh_per_launch": evals_per_sweep / 4.0 * 6 * 128,
                                 "tanh_floor_ms": evals_per_sweep / 4.0 * 6 * 128 / (16 * sms * mhz * 1e6) * 1e3,
                                 "tanh_floor_basis": f"16 tanh/clk/SM x {sms} SMs x {mhz:.0f} MHz (median "
                                                     "sampled SM clock of the timed region)",
                                 "source": "profiles/mlp_bf16_L64_ncu_full.md"}},
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = {"value": cpu["value"], "unit": UNIT, "cores": cpu["threads"], "kind": "oracle",
                                "sample": f"{cpu['subdomains']} whole subdomains of colour 0 of the same grid "
                                          f"(gather + SDNet on 961 points + write), FP64 NumPy, "
                                          f"{cpu['seconds']:.1f} s"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
