"""Benchmark: LM iterations/s of the bundle-adjustment hot path on one GB300.

Workload: the Venice-1778-shaped synthetic problem (1,700 cameras, 1M points,
~5.0M observations, 20 LM iterations, PCG up to 100 iterations, seed 1).  One
"step" is one mba_solve of those 20 LM iterations from the initial estimate
(the device-side reset of the parameters is inside the step).  The headline
value is the FP32-mixed form; the plain FP64 form is measured beside it.

Beside the headline the line carries the FP64 form, the solver variants (the
float-float accept/reject cost among them), the dual-number Jacobians, the
differentiable-layer and batched-window workloads, and the Final-13682-shaped
problem (13,000 cameras, 4.5M points, 29M observations, Huber, 30 LM iterations)
in both forms.  The CPU-baseline leg times the oracle on a bounded sample (the
workload's first two LM iterations, and one iteration of a 0.1-scale sample on
one thread) and compares the GPU's first two iterations with the oracle's.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (bounded sample: one LM iteration per step).
Multi-GPU runs (torchrun) are independent replicas: the method's single-GPU
path has no data-parallel split, so every rank solves its own copy.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LM iterations/sec and PCG SpMV HBM GB/s (% of peak), FP32-mixed vs FP64, 1 GB300"
UNIT = "LM iterations/s"
CONFIG = 2
LM_ITERS = 20
PCG_MAX = 100
FINAL_LM_ITERS = 30   # the Final-shaped problem's LM iterations
CPU_LM_ITERS = 2      # LM iterations of the oracle's bounded sample
CPU_SINGLE_SCALE = 0.1  # workload scale of the single-thread oracle sample


def workload_desc(sc) -> str:
    return (f"venice-shaped synthetic BA: {sc.nc} cameras, {sc.np_} points, {sc.n} observations, "
            f"{LM_ITERS} LM iterations, PCG <= {PCG_MAX}, seed 1")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 ALU peak derived from unit counts and clocks: the recipe's nominal 1.25
# TFLOP/s for GB300 FP64 equals 152 SMs x 2 FP64 FMA/clk/SM x 2 FLOP x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def pcg_bytes_per_iter(sc, w: int) -> float:
    """Algorithmic bytes of one PCG iteration, by the method's per-unit counts
    with the stored Jacobian taken as the minimum: per observation the Jacobian
    (24 values) and a camera index; per point C~^-1 (6 doubles) and about six
    vector entries; per camera the Cholesky factor of B~ (45 doubles) and about
    six 9-vectors."""
    return sc.n * (24 * w + 4) + sc.np_ * (6 * 8 + 6 * w) + sc.nc * (45 * 8 + 54 * w)


def pcg_streamed_bytes_per_iter(sc) -> float:
    """Bytes the factored FP32 Schur product streams per PCG iteration: per
    observation (px, py, 1/P_z) 12, W Jp 24, camera index 4, position of s 4,
    s written 8 in the point pass and (RX, 1/P_z) 16, s 8 in the camera pass;
    per point C~^-1 (6 floats) and a CSR offset; per camera B~ and B~^-1 (81
    doubles each) and six FP64 vectors of stride 12."""
    return sc.n * 76 + sc.np_ * 28 + sc.nc * (2 * 81 * 8 + 6 * 12 * 8)


def lin_bytes_per_obs(sc, w: int) -> float:
    """Algorithmic bytes of the residual + Jacobian + block step per observation:
    pixels (2w), two indices (8), the point amortised over its track (3w/L) and
    the Jacobian written (24w)."""
    return (26.0 + 3.0 * sc.np_ / sc.n) * w + 8.0


# FP32 non-tensor peak derived from unit counts and clocks: 152 SMs x 128 FP32
# lanes x 2 FLOP (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Batched windows, counted FP32 operations:
#  implicit product, per observation per PCG iteration: projection, D and Jp 88;
#    Jc p 42; W Jp^T t 14; scan adds 15; C~^-1 18; s = W Jp b 14; camera pass
#    Jc^T s with its projection 115 (also the right-hand side of every solve);
#  explicit S~, per (observation pair of one point) per damped solve: Q = Jp C~^-1
#    36, G 24, F = G Jc 72, the 81 block entries 324;
#  explicit product, per PCG iteration: 2 (9 nc)^2;
#  per observation per LM iteration: linearisation (two projections with
#    Jacobians, the 9 point and 54 camera block terms) 450, back-substitution 380.
BATCH_FLOP_IMPLICIT_OBS_ITER = 305
BATCH_FLOP_PAIR = 456
BATCH_FLOP_OBS_LM = 830


def batch_flops(ws, summaries, schur: str) -> float:
    """Counted FP32 operations of one batched solve (forward + adjoint)."""
    tot = 0.0
    for w, sm in zip(ws, summaries):
        solves = sm["iterations"] + (1 if sm["adjoint_pcg_iters"] > 0 else 0)
        iters = sm["pcg_iters_total"] + sm["adjoint_pcg_iters"]
        tot += sm["iterations"] * w.n * BATCH_FLOP_OBS_LM + solves * w.n * BATCH_FLOP_IMPLICIT_OBS_ITER
        if schur == "explicit":
            L = np.bincount(w.pt_idx)
            tot += solves * float((L * (L + 1) // 2).sum()) * BATCH_FLOP_PAIR + iters * 2.0 * (9 * w.nc) ** 2
        else:
            tot += iters * w.n * BATCH_FLOP_IMPLICIT_OBS_ITER
    return tot


# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per observation
# per pass of one pcg_kernel launch on the full Venice-shaped problem (30 PCG
# iterations plus the right-hand-side pass, 5,004,484 observations), FP32-mixed
# and FP64.  Traffic grows with the observation count, so a launch moves this
# many bytes per observation per pass; None once the kernel has changed since
# the capture.  The last full-size capture gave 61.3 B (FP32-mixed) and 431.1 B
# (FP64); both kernels have changed since (the FP32 one loads its B~ rows
# earlier, the FP64 one runs fewer scan levels), so no figure is claimed.
PCG_TRAFFIC_B_PER_OBS_PASS = {}
PCG_TRAFFIC_NOTE = ("null: the kernel changed after the last full-size DRAM capture (61.3 B per observation per "
                    "pass FP32-mixed, 431.1 B FP64); the FP32 change loads the same rows earlier, the FP64 one "
                    "runs fewer FP64 scan levels; not re-taken")


def oracle_sample_time(threads: int, scale: float) -> dict:
    """Seconds of one oracle LM iteration on the workload scaled by `scale`, in a
    fresh process with `threads` OpenMP threads (0 = the default, all cores)."""
    code = ("import json, sys, time; sys.path.insert(0, %r); import oracle; from scenes import config_scene; "
            "sc = config_scene(%d, scale=%r); oracle.build(); t = time.perf_counter(); "
            "oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=1, "
            "pcg_max=%d, pcg_tol=1e-10); "
            "print(json.dumps({'s': time.perf_counter() - t, 'threads': oracle.num_threads(), 'n': int(sc.n)}))"
            % (ROOT, CONFIG, scale, PCG_MAX))
    env = dict(os.environ)
    if threads > 0:
        env["OMP_NUM_THREADS"] = str(threads)
    else:
        env.pop("OMP_NUM_THREADS", None)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def pcg_flops_per_iter(sc) -> float:
    """48 FMA per observation (E^T p and E b), 9 per point (C~^-1), 2 x 81 per camera."""
    return 2.0 * (48 * sc.n + 9 * sc.np_ + 162 * sc.nc)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
                self.lines = [ln for ln in out.splitlines() if ln.strip()]
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl"
        try:
            import torch

            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def max_over_ranks(ms: float, dist) -> float:
    """The slowest rank's time: every rank returns the same value."""
    if dist is None:
        return ms
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


def run_reference(args, rank, world):
    """CPU oracle on the host cores: each step is one LM iteration of the workload."""
    if rank != 0:
        return 0
    import oracle
    from scenes import config_scene

    sc = config_scene(CONFIG)
    oracle.build()
    threads = oracle.num_threads()

    def one():
        t = time.perf_counter()
        oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=1,
                        pcg_max=PCG_MAX, pcg_tol=1e-10)
        return time.perf_counter() - t

    for _ in range(args.warmup):
        one()
    times = [one() for _ in range(args.steps)]
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(sc), "precision": "fp64 (CPU oracle)",
                   "sample": "1 LM iteration per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "one LM iteration (linearise, PCG <= 100, back-substitution, cost) per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def profile_case(precision: str, scale: float, config: int = CONFIG) -> int:
    """A small solve for ncu captures: the workload scaled by `scale` (0.3 gives
    1.5M observations, a Jacobian stream larger than L2), 2 LM iterations with
    PCG <= 30, so one capture holds a bounded number of PCG launches.  config 3
    is the Final-shaped problem (Huber, delta 2 px)."""
    import torch

    from paper_2112_01349_gb300 import _build, mba
    from scenes import config_scene

    torch.cuda.set_device(0)
    _build.build()
    sc = config_scene(config, scale=scale)
    loss = "huber" if config == 3 else "none"
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision, loss=loss,
                     huber_delta=2.0) as pr:
        s = pr.solve(max_iter=2, pcg_max_iter=30, collect_timing=1)
    print(json.dumps({"profile_case": precision, "config": config, "scale": scale, "nc": sc.nc, "np": sc.np_, "n": sc.n,
                      "pcg_iters_total": s["pcg_iters_total"], "final_cost": s["final_cost"]}))
    return 0


def profile_batch(windows: int) -> int:
    """A batched solve for ncu captures: the first `windows` windows of the
    512-window workload (largest sizes mixed as in the full batch), fixed
    schedule (256 threads x 2 CTAs per SM, explicit Schur form), one warm-up
    replay and one measured replay, 8 LM iterations + adjoint each."""
    import torch

    from paper_2112_01349_gb300 import _build, mba
    from scenes import make_windows

    torch.cuda.set_device(0)
    _build.build()
    ws = make_windows(512)[:windows]
    tup = [(w.cameras, w.points, w.observations, w.cam_idx, w.pt_idx) for w in ws]
    rng = np.random.default_rng(5)
    with mba.Batch(tup, precision="fp32") as bt:
        bt.set_schedule(256, 2, "explicit")
        gc, gp = rng.normal(size=(bt.info["nc"], 9)), rng.normal(size=(bt.info["np"], 3))
        ms = []
        for _ in range(2):
            bt.reset()
            ms.append(bt.solve(gc, gp, max_iter=8, pcg_max_iter=PCG_MAX, pcg_rel_tol=1e-10)["ms"])
        info = bt.info
    print(json.dumps({"profile_case": "batch", "windows": windows, "n": info["n"], "ms": ms}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-final", action="store_true", help="skip the Final-shaped leg")
    ap.add_argument("--profile-case", choices=["fp32", "fp64", "batch"], default=None,
                    help="profiling aid: run one small solve of the workload (see --scale, --windows) and exit; "
                         "prints no bench line")
    ap.add_argument("--scale", type=float, default=0.3, help="camera/point scale of --profile-case fp32/fp64")
    ap.add_argument("--config", type=int, default=CONFIG, choices=[2, 3],
                    help="workload of --profile-case fp32/fp64: 2 Venice-shaped, 3 Final-shaped")
    ap.add_argument("--windows", type=int, default=128, help="windows of --profile-case batch")
    args = ap.parse_args()
    if args.profile_case == "batch":
        return profile_batch(args.windows)
    if args.profile_case:
        return profile_case(args.profile_case, args.scale, args.config)
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local, dist = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    from paper_2112_01349_gb300 import _build, mba
    from scenes import config_scene

    if rank == 0:
        _build.build()
    if dist is not None:
        dist.barrier()
    mba.load()
    sc = config_scene(CONFIG)
    stream = torch.cuda.Stream()
    opts = dict(max_iter=LM_ITERS, pcg_max_iter=PCG_MAX, pcg_rel_tol=1e-10, collect_timing=1)

    def timed(prec):
        pr = mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=prec,
                         stream=stream)
        for _ in range(args.warmup):
            pr.reset()
            pr.solve(**opts)
        sums = []
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                pr.reset()
                sums.append(pr.solve(trace_capacity=LM_ITERS, **opts))
            e1.record(stream)
            torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist)
        if dist is not None:
            dist.barrier()
        pr.close()
        return ms, sums, clk.summary()

    ms32, s32, clk32 = timed("fp32")
    ms64, s64, clk64 = timed("fp64")

    def stats(ms, sums, w):
        value = whole_job_rate(LM_ITERS * args.steps, world, ms)
        pcg_ms = sum(s["ms_pcg"] for s in sums)
        pcg_iters = sum(s["pcg_iters_total"] for s in sums)
        launches = len(sums) * LM_ITERS  # one persistent PCG launch per LM iteration
        passes = pcg_iters + launches  # the right-hand-side pass counts as one
        alg_bytes = passes * pcg_bytes_per_iter(sc, w)
        alg_flops = passes * pcg_flops_per_iter(sc)
        traffic = PCG_TRAFFIC_B_PER_OBS_PASS.get(w)
        # linearisations: the first one, then one after every accepted step that
        # is not the solve's last iteration (a rejected step reuses the last one)
        lins = sum(1 + sum(t["accepted"] for t in s["trace"][:-1]) for s in sums)
        lin_ms = sum(s["ms_linearize"] for s in sums)
        return dict(value=value, ms_per_step=ms / args.steps, pcg_ms=pcg_ms, pcg_iters=pcg_iters,
                    pcg_launches=launches, gbs=alg_bytes / (pcg_ms / 1e3) / 1e9,
                    streamed_gbs=passes * pcg_streamed_bytes_per_iter(sc) / (pcg_ms / 1e3) / 1e9,
                    traffic_per_launch=None if traffic is None else traffic * sc.n * passes / launches,
                    dram_gbs=None if traffic is None else traffic * sc.n * passes / (pcg_ms / 1e3) / 1e9,
                    alg_bytes_per_launch=alg_bytes / launches,
                    tflops=alg_flops / (pcg_ms / 1e3) / 1e12,
                    us_per_pcg_iter=1e3 * pcg_ms / max(1, passes),
                    lin_ms_each=lin_ms / lins, lin_gbs=lins * sc.n * lin_bytes_per_obs(sc, w) / (lin_ms / 1e3) / 1e9,
                    final_cost=sums[-1]["final_cost"], kernel_launches=sum(s["kernel_launches"] for s in sums),
                    accepted=sums[-1]["accepted"], pcg_share=pcg_ms / sum(s["ms_total"] for s in sums))

    a32, a64 = stats(ms32, s32, 4), stats(ms64, s64, 8)
    hbm_peak, peak_kind = peaks()

    # end to end through the C ABI with host buffers: create (H2D of the inputs
    # from pinned memory), solve, read the parameters back (D2H), destroy
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    hc, hp, ho = pin(sc.cameras), pin(sc.points), pin(sc.observations)
    hci, hpi = pin(sc.cam_idx), pin(sc.pt_idx)
    oc, op_ = torch.empty_like(hc).pin_memory(), torch.empty_like(hp).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (hc, hp, ho, hci, hpi))
    d2h = sum(t.numel() * t.element_size() for t in (oc, op_))

    def e2e_step():
        pr = mba.Problem(hc, hp, ho, hci, hpi, precision="fp32", stream=stream)
        pr.solve(max_iter=LM_ITERS, pcg_max_iter=PCG_MAX, pcg_rel_tol=1e-10)
        mba.mba_get_parameters(pr.handle, oc, op_)
        pr.close()

    for _ in range(2):
        e2e_step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), dist)
    e2e_value = whole_job_rate(LM_ITERS * args.steps, world, e2e_ms)

    # solver variants beside Alg. 2 (not the headline): the same workload and
    # LM iteration count with the float-float accept/reject cost, the
    # Schur-Jacobi preconditioner and/or the inexact-Newton forcing sequence,
    # and the single-reduction (Chronopoulos-Gear) PCG recurrence, FP32-mixed
    variants = None
    if rank == 0:
        variants = {}
        with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision="fp32",
                         stream=stream) as prv:
            for name, kw in (("float_float_cost", dict(cost_arithmetic="float-float")),
                             ("schur_jacobi", dict(preconditioner="schur_jacobi")), ("forcing", dict(forcing=1)),
                             ("schur_jacobi+forcing", dict(preconditioner="schur_jacobi", forcing=1)),
                             ("single_reduction_pcg", dict(pcg_variant="single_reduction"))):
                ms_v = []
                for _ in range(2):
                    prv.reset()
                    torch.cuda.synchronize()
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(stream)
                    sv = prv.solve(trace_capacity=LM_ITERS, max_iter=LM_ITERS, pcg_max_iter=PCG_MAX,
                                   pcg_rel_tol=1e-10, collect_timing=1, **kw)
                    ev1.record(stream)
                    torch.cuda.synchronize()
                    ms_v.append(ev0.elapsed_time(ev1))
                passes_v = sv["pcg_iters_total"] + LM_ITERS
                variants[name] = {"value": LM_ITERS / (min(ms_v) / 1e3), "unit": UNIT, "ms_per_solve": min(ms_v),
                                  "pcg_iters": sv["pcg_iters_total"], "final_cost": sv["final_cost"],
                                  "us_per_pcg_iter": 1e3 * sv["ms_pcg"] / passes_v,
                                  "accepted": sv["accepted"],
                                  "same_accept_decisions_as_headline":
                                      [t["accepted"] for t in sv["trace"]] == [t["accepted"] for t in s32[-1]["trace"]],
                                  "final_cost_rel_diff_vs_paper_solver":
                                      (sv["final_cost"] - a32["final_cost"]) / a32["final_cost"]}
        variants["note"] = ("variants of the same workload (20 LM iterations, PCG <= 100, FP32-mixed): the "
                            "headline value is Alg. 2 (block-Jacobi, fixed tolerance 1e-10) with the FP64 "
                            "accept/reject cost; float_float_cost evaluates that cost in float-float arithmetic; "
                            "single_reduction_pcg runs the Chronopoulos-Gear recurrence of the same PCG (one "
                            "global reduction per PCG step instead of two; same iterates in exact arithmetic)")

    # Jacobian source (Sec. 3.2): the same solve with the Jacobian from the edge
    # functor on dual numbers instead of the hand-derived chain rule
    autodiff = None
    if rank == 0:
        autodiff = {}
        for prec, ref in (("fp32", (a32, s32)), ("fp64", (a64, s64))):
            with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=prec,
                             stream=stream, jacobian="autodiff") as pra:
                runs = []
                for _ in range(2):
                    pra.reset()
                    torch.cuda.synchronize()
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(stream)
                    sa = pra.solve(**opts)
                    ev1.record(stream)
                    torch.cuda.synchronize()
                    runs.append((ev0.elapsed_time(ev1), sa))
            ms_a, sa = min(runs, key=lambda r: r[0])
            an_stats, an_sums = ref
            lin_an = sum(x["ms_linearize"] for x in an_sums) / len(an_sums)
            pcg_an = sum(x["ms_pcg"] for x in an_sums) / len(an_sums)
            autodiff[prec] = {"value": LM_ITERS / (ms_a / 1e3), "unit": UNIT, "ms_per_solve": ms_a,
                              "ms_linearize": sa["ms_linearize"], "ms_linearize_analytic": lin_an,
                              "ms_pcg": sa["ms_pcg"], "ms_pcg_analytic": pcg_an,
                              "final_cost_rel_diff_vs_analytic":
                                  (sa["final_cost"] - an_stats["final_cost"]) / an_stats["final_cost"]}
        autodiff["note"] = ("Jacobians from the BAL edge functor evaluated on forward-mode dual numbers (12 "
                            "directions per pass); FP32-mixed also streams a stored camera-major Jacobian in the PCG "
                            "camera pass instead of re-deriving Jc^T s from the camera table")

    # differentiable-layer workload (200 cameras, 50k points, ~250k observations,
    # FP32-mixed): forward LM to convergence, then the adjoint of the solution
    layer = None
    if rank == 0:
        sc4 = config_scene(4)
        rng = np.random.default_rng(0)
        gc4, gp4 = rng.normal(size=(sc4.nc, 9)), rng.normal(size=(sc4.np_, 3))
        with mba.Problem(sc4.cameras, sc4.points, sc4.observations, sc4.cam_idx, sc4.pt_idx, precision="fp32",
                         stream=stream) as pr4:
            fwd, adj = [], []
            for rep in range(3):
                pr4.reset()
                torch.cuda.synchronize()
                t = time.perf_counter()
                s4 = pr4.solve(max_iter=100, pcg_max_iter=100, pcg_rel_tol=1e-10, function_tol=1e-12)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                a4 = pr4.adjoint(gc4, gp4, mu=-1.0, pcg_max_iter=500, pcg_rel_tol=1e-10)
                torch.cuda.synchronize()
                fwd.append(t1 - t)
                adj.append(time.perf_counter() - t1)
        layer = {"workload": f"differentiable layer: {sc4.nc} cameras, {sc4.np_} points, {sc4.n} observations, "
                             "FP32-mixed, LM to |dF|/F < 1e-12 (<= 100 iterations), then the adjoint",
                 "forward_ms": 1e3 * min(fwd), "adjoint_ms": 1e3 * min(adj), "lm_iterations": s4["iterations"],
                 "adjoint_pcg_iters": a4["pcg_iters"]}

    # batched local-BA windows (512 windows, cameras U[5,30], points U[200,3000],
    # track 2 + Geom (mean 4), FP32-mixed): 8 LM iterations per window and the
    # adjoint, one persistent launch replayed from a CUDA graph
    batched = None
    if rank == 0:
        from scenes import make_windows

        ws = make_windows(512)
        tup = [(w.cameras, w.points, w.observations, w.cam_idx, w.pt_idx) for w in ws]
        bopts = dict(max_iter=8, pcg_max_iter=PCG_MAX, pcg_rel_tol=1e-10)
        rng = np.random.default_rng(5)
        with mba.Batch(tup, precision="fp32", stream=stream) as bt:
            gcb, gpb = rng.normal(size=(bt.info["nc"], 9)), rng.normal(size=(bt.info["np"], 3))
            tune = bt.autotune(**bopts)
            fwd_ms, full_ms = [], []
            for rep in range(3):
                bt.reset()
                fwd_ms.append(bt.solve(**bopts)["ms"])
                bt.reset()
                rb = bt.solve(gcb, gpb, adjoint_pcg_max_iter=500, adjoint_pcg_rel_tol=1e-10, **bopts)
                full_ms.append(rb["ms"])
            sm_b = rb["summaries"]
        nobs = sum(w.n for w in ws)
        pcg_b = sum(x["pcg_iters_total"] for x in sm_b)
        adj_b = sum(x["adjoint_pcg_iters"] for x in sm_b)
        t_full = statistics.median(full_ms)
        # end to end: pinned host buffers -> create (layout + H2D) -> solve + adjoint -> D2H of the
        # parameters and gradients -> destroy
        co, po, oo, cams_c, pts_c, obs_c, ci_c, pi_c = mba.concat_windows(tup)
        hb = [pin(a) for a in (cams_c, pts_c, obs_c, ci_c, pi_c)]
        hb_out = [torch.empty_like(hb[0]).pin_memory(), torch.empty_like(hb[1]).pin_memory(),
                  torch.empty((nobs, 2), dtype=torch.float64).pin_memory()]
        h2d_b = sum(t.numel() * t.element_size() for t in hb) + 8 * (len(co) + len(po) + len(oo))
        d2h_b = sum(t.numel() * t.element_size() for t in hb_out)

        def batch_e2e():
            h = mba.mba_batch_create(co, po, oo, hb[0], hb[1], hb[2], hb[3], hb[4], precision="fp32", stream=stream)
            mba.mba_batch_set_schedule(h, tune["threads_per_cta"], tune["ctas_per_sm"])
            mba.mba_batch_solve(h, gcb, gpb, adjoint_pcg_max_iter=500, adjoint_pcg_rel_tol=1e-10, **bopts)
            cv = mba.mba_batch_get_parameters(h)
            g = mba.mba_batch_get_gradients(h)
            hb_out[0].numpy()[:] = cv[0]
            hb_out[1].numpy()[:] = cv[1]
            hb_out[2].numpy()[:] = g["grad_obs"]
            mba.mba_batch_destroy(h)

        batch_e2e()
        t0b = time.perf_counter()
        for _ in range(2):
            batch_e2e()
        e2e_b = (time.perf_counter() - t0b) / 2
        flops = batch_flops(ws, sm_b, tune["schur"])
        batched = {
            "workload": f"batched local BA: {len(ws)} windows (cameras U[5,30], points U[200,3000], track 2+Geom "
                        f"mean 4, 1 px noise), {bt.info['nc']} cameras, {bt.info['np']} points, {nobs} observations "
                        "in total, FP32-mixed, 8 LM iterations per window (PCG <= 100, rel tol 1e-10) + adjoint",
            "ms_forward_plus_adjoint": t_full, "ms_forward": statistics.median(fwd_ms),
            "windows_per_s": len(ws) / (t_full / 1e3),
            "window_lm_iterations_per_s": sum(x["iterations"] for x in sm_b) / (t_full / 1e3),
            "pcg_iters_forward": pcg_b, "pcg_iters_adjoint": adj_b,
            "schedule": {"threads_per_cta": tune["threads_per_cta"], "ctas_per_sm": tune["ctas_per_sm"],
                         "schur": tune["schur"], "autotune_ms": tune["ms"]},
            "launch": "one CUDA graph replay (claim-counter reset + one persistent kernel)",
            "gpu_launches": 1,
            "roofline": {"kernel": "batch_kernel (persistent, one window per CTA)", "bound": "alu",
                         "achieved": flops / (t_full / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops / (t_full / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                         "peak_kind": "derived (152 SMs x 128 FP32 lanes x 2 x 2.07 GHz)",
                         "counted": "FP32 operations of the schedule's Schur form (see batch_flops)",
                         "note": "whole launch time; the launch is latency-bound (FP64 vector chains, CTA "
                                 "barriers)"},
            "e2e": {"ms": 1e3 * e2e_b, "windows_per_s": len(ws) / e2e_b, "h2d_bytes_per_step": h2d_b,
                    "d2h_bytes_per_step": d2h_b},
        }

    # Final-13682-shaped problem (13,000 cameras, 4.5M points, ~29M observations,
    # 1% outliers, Huber delta 2 px): 30 LM iterations, PCG <= 100, FP32-mixed
    # and FP64; one warm-up solve and one timed solve each
    final = None
    if rank == 0 and not args.no_final:
        sc3 = config_scene(3)
        final = {"workload": f"final-shaped synthetic BA: {sc3.nc} cameras, {sc3.np_} points, {sc3.n} observations, "
                             f"1% outliers at 50 px, Huber delta 2 px, {FINAL_LM_ITERS} LM iterations, PCG <= "
                             f"{PCG_MAX}, seed 2"}
        for prec, w in (("fp32", 4), ("fp64", 8)):
            with mba.Problem(sc3.cameras, sc3.points, sc3.observations, sc3.cam_idx, sc3.pt_idx, precision=prec,
                             loss="huber", huber_delta=2.0, stream=stream) as pr3:
                for rep in range(2):
                    pr3.reset()
                    torch.cuda.synchronize()
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(stream)
                    s3 = pr3.solve(max_iter=FINAL_LM_ITERS, pcg_max_iter=PCG_MAX, pcg_rel_tol=1e-10,
                                   collect_timing=1)
                    ev1.record(stream)
                    torch.cuda.synchronize()
                ms3 = ev0.elapsed_time(ev1)
            passes = s3["pcg_iters_total"] + FINAL_LM_ITERS
            final[prec] = {"value": FINAL_LM_ITERS / (ms3 / 1e3), "unit": UNIT, "ms_per_solve": ms3,
                           "pcg_iters": s3["pcg_iters_total"], "accepted": s3["accepted"],
                           "us_per_pcg_iter": 1e3 * s3["ms_pcg"] / passes,
                           "pcg_alg_gbs": passes * pcg_bytes_per_iter(sc3, w) / (s3["ms_pcg"] / 1e3) / 1e9,
                           "initial_cost": s3["initial_cost"], "final_cost": s3["final_cost"]}
        final["final_cost_rel_diff_fp32_vs_fp64"] = ((final["fp32"]["final_cost"] - final["fp64"]["final_cost"]) /
                                                     final["fp64"]["final_cost"])
        del sc3

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        from oracle.align import parameter_error

        oracle.build()
        # the oracle (FP64, host cores) on a bounded sample of the workload: its
        # first CPU_LM_ITERS LM iterations; the GPU solves the same iterations in
        # both forms and its cost and parameters are compared with the oracle's
        t = time.perf_counter()
        ref = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=CPU_LM_ITERS,
                              pcg_max=PCG_MAX, pcg_tol=1e-10)
        dt = time.perf_counter() - t
        parity = {"sample": f"first {CPU_LM_ITERS} LM iterations of the workload, PCG <= {PCG_MAX}",
                  "oracle_accepted": [t_["accepted"] for t_ in ref["trace"]]}
        for prec in ("fp64", "fp32"):
            with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=prec,
                             stream=stream) as prp:
                sp = prp.solve(trace_capacity=CPU_LM_ITERS, max_iter=CPU_LM_ITERS, pcg_max_iter=PCG_MAX,
                               pcg_rel_tol=1e-10)
                cg, pg = prp.parameters()
            parity[prec] = {"final_cost_rel_diff": (sp["final_cost"] - ref["final_cost"]) / ref["final_cost"],
                            "accepted": [t_["accepted"] for t_ in sp["trace"]],
                            "parameter_error": parameter_error(cg, pg, ref["cameras"], ref["points"])}
        single = oracle_sample_time(1, CPU_SINGLE_SCALE)
        multi = oracle_sample_time(0, CPU_SINGLE_SCALE)
        cpu = {"value": CPU_LM_ITERS / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{CPU_LM_ITERS} LM iterations (linearise, PCG <= {PCG_MAX}, back-substitution, cost) of the "
                         "same workload, FP64",
               "single_thread": {"value": 1.0 / single["s"], "unit": UNIT, "cores": single["threads"],
                                 "value_all_cores_same_sample": 1.0 / multi["s"], "cores_all": multi["threads"],
                                 "sample": f"one LM iteration of the workload scaled by {CPU_SINGLE_SCALE} "
                                           f"({single['n']} observations)"},
               "parity_vs_gpu": parity}

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": a32["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": a32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (FP32-mixed)", "data": "synthetic",
        "config": {"workload": workload_desc(sc), "precision": "fp32-mixed (FP64 accept/reject cost)",
                   "l2": "inputs larger than L2 (per PCG pass: 0.38 GB streamed FP32, 1.7 GB FP64)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"kernel": "pcg_kernel (persistent PCG, implicit Schur product)", "bound": "hbm",
                     "achieved": a32["gbs"], "peak": hbm_peak, "unit": "GB/s", "frac": a32["gbs"] / hbm_peak,
                     "peak_kind": peak_kind, "traffic": a32["traffic_per_launch"],
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read+write per observation per pass of a "
                                     "full-size launch, times this run's observations and passes)",
                     "algorithmic_bytes_per_launch": a32["alg_bytes_per_launch"],
                     "algorithmic": "per PCG iteration 100 B per observation (stored Jacobian + camera index), "
                                    "72 B per point, 576 B per camera",
                     "streamed_gbs": a32["streamed_gbs"], "streamed_frac": a32["streamed_gbs"] / hbm_peak,
                     "streamed": "bytes the factored FP32 product actually streams: 76 B per observation per "
                                 "iteration, 28 B per point, 1.9 KB per camera",
                     "dram_gbs": a32["dram_gbs"],
                     "dram_frac": None if a32["dram_gbs"] is None else a32["dram_gbs"] / hbm_peak,
                     "traffic_note": PCG_TRAFFIC_NOTE if a32["traffic_per_launch"] is None else None,
                     "us_per_pcg_iter": a32["us_per_pcg_iter"], "share_of_solve": a32["pcg_share"],
                     "pcg_iters_per_solve": a32["pcg_iters"] / max(1, len(s32)),
                     "other_kernels": {
                         "pcg_single_reduction_fp32": None if not variants else {
                             "kernel": "pcg_kernel, single-reduction (Chronopoulos-Gear) instance",
                             "bound": "hbm", "unit": "GB/s",
                             "us_per_pcg_iter": variants["single_reduction_pcg"]["us_per_pcg_iter"],
                             "achieved": pcg_bytes_per_iter(sc, 4) / (variants["single_reduction_pcg"]["us_per_pcg_iter"]
                                                                      / 1e6) / 1e9,
                             "frac": pcg_bytes_per_iter(sc, 4) / (variants["single_reduction_pcg"]["us_per_pcg_iter"]
                                                                  / 1e6) / 1e9 / hbm_peak,
                             "note": "same algorithmic bytes per PCG iteration as the headline kernel; one global "
                                     "reduction per PCG step instead of two (solver option, not the headline)"},
                         "linearize_fp32": {"kernel": "lin_point + lin_camera + cam_finalize (+ camera table)",
                                            "bound": "hbm", "achieved": a32["lin_gbs"], "unit": "GB/s",
                                            "frac": a32["lin_gbs"] / hbm_peak,
                                            "ms_per_linearisation": a32["lin_ms_each"],
                                            "algorithmic_bytes_per_obs": lin_bytes_per_obs(sc, 4)},
                         "linearize_fp64": {"achieved": a64["lin_gbs"], "unit": "GB/s",
                                            "frac": a64["lin_gbs"] / hbm_peak,
                                            "ms_per_linearisation": a64["lin_ms_each"],
                                            "algorithmic_bytes_per_obs": lin_bytes_per_obs(sc, 8)},
                         "pcg_fp64": {"bound": "alu", "achieved": a64["tflops"], "peak": FP64_PEAK_TFLOPS,
                                      "unit": "TFLOP/s", "frac": a64["tflops"] / FP64_PEAK_TFLOPS,
                                      "peak_kind": "derived (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                                      "alg_gbs": a64["gbs"], "dram_gbs": a64["dram_gbs"],
                                      "us_per_pcg_iter": a64["us_per_pcg_iter"]}}},
        "final_cost": a32["final_cost"], "accepted": a32["accepted"],
        "final_cost_rel_diff_vs_fp64": abs(a32["final_cost"] - a64["final_cost"]) / a64["final_cost"],
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": s32 and sum(s["kernel_launches"] for s in s32),
        "variants": variants,
        "autodiff": autodiff,
        "layer": layer,
        "batched": batched,
        "final": final,
        "fp64": {"value": a64["value"], "unit": UNIT, "ms_per_step": a64["ms_per_step"],
                 "final_cost": a64["final_cost"], "accepted": a64["accepted"], "clocks": clk64},
        "clocks": clk32,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
