"""Benchmark: LM iterations/s of the bundle-adjustment hot path on one GB300.

Workload: the Venice-1778-shaped synthetic problem (1,700 cameras, 1M points,
~5.0M observations, 20 LM iterations, PCG up to 100 iterations, seed 1).  One
"step" is one mba_solve of those 20 LM iterations from the initial estimate
(the device-side reset of the parameters is inside the step).  The headline
value is the FP32-mixed form; the plain FP64 form is measured beside it.

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
    """Algorithmic bytes of one PCG iteration: the Jacobian stream and camera
    index per observation, C~^-1 and a CSR offset per point, B~, B~^-1 and the
    camera vectors per camera."""
    return sc.n * (24 * w + 4) + sc.np_ * (6 * w + 4) + sc.nc * (2 * 81 * 8 + 6 * 9 * 8)


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


def profile_case(precision: str, scale: float) -> int:
    """A small solve for ncu captures: the workload scaled by `scale` (0.3 gives
    1.5M observations, a Jacobian stream larger than L2), 2 LM iterations with
    PCG <= 30, so one capture holds a bounded number of PCG launches."""
    import torch

    from paper_2112_01349_gb300 import _build, mba
    from scenes import config_scene

    torch.cuda.set_device(0)
    _build.build()
    sc = config_scene(CONFIG, scale=scale)
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision) as pr:
        s = pr.solve(max_iter=2, pcg_max_iter=30, collect_timing=1)
    print(json.dumps({"profile_case": precision, "scale": scale, "nc": sc.nc, "np": sc.np_, "n": sc.n,
                      "pcg_iters_total": s["pcg_iters_total"], "final_cost": s["final_cost"]}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", choices=["fp32", "fp64"], default=None,
                    help="profiling aid: run one small solve of the workload (see --scale) and exit; "
                         "prints no bench line")
    ap.add_argument("--scale", type=float, default=0.3, help="camera/point scale of --profile-case")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case, args.scale)
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
                sums.append(pr.solve(**opts))
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if dist is not None:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            dist.barrier()
        pr.close()
        return ms, sums, clk.summary()

    ms32, s32, clk32 = timed("fp32")
    ms64, s64, clk64 = timed("fp64")

    def stats(ms, sums, w):
        its = LM_ITERS * args.steps * world
        value = its / (ms / 1e3)
        pcg_ms = sum(s["ms_pcg"] for s in sums)
        pcg_iters = sum(s["pcg_iters_total"] for s in sums)
        launches = len(sums) * LM_ITERS  # one persistent PCG launch per LM iteration
        alg_bytes = (pcg_iters + launches) * pcg_bytes_per_iter(sc, w)
        alg_flops = (pcg_iters + launches) * pcg_flops_per_iter(sc)
        return dict(value=value, ms_per_step=ms / args.steps, pcg_ms=pcg_ms, pcg_iters=pcg_iters,
                    pcg_launches=launches, gbs=alg_bytes / (pcg_ms / 1e3) / 1e9,
                    tflops=alg_flops / (pcg_ms / 1e3) / 1e12,
                    us_per_pcg_iter=1e3 * pcg_ms / max(1, pcg_iters + launches),
                    final_cost=sums[-1]["final_cost"], kernel_launches=sum(s["kernel_launches"] for s in sums),
                    pcg_share=pcg_ms / sum(s["ms_total"] for s in sums))

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
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = LM_ITERS * args.steps * world / e2e_s

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

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        t = time.perf_counter()
        oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=1, pcg_max=PCG_MAX)
        dt = time.perf_counter() - t
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "one LM iteration (linearise, PCG <= 100, back-substitution, cost) of the same workload, FP64"}

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": a32["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": a32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 (FP32-mixed)", "data": "synthetic",
        "config": {"workload": workload_desc(sc), "precision": "fp32-mixed",
                   "l2": "inputs larger than L2 (Jacobian stream 0.48 GB FP32 / 0.96 GB FP64 per pass)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"kernel": "pcg_kernel (persistent PCG, implicit Schur product)", "bound": "hbm",
                     "achieved": a32["gbs"], "peak": hbm_peak, "unit": "GB/s", "frac": a32["gbs"] / hbm_peak,
                     "peak_kind": peak_kind, "traffic": None,
                     "us_per_pcg_iter": a32["us_per_pcg_iter"], "share_of_solve": a32["pcg_share"]},
        "fp64": {"value": a64["value"], "unit": UNIT, "ms_per_step": a64["ms_per_step"],
                 "final_cost": a64["final_cost"],
                 "roofline": {"kernel": "pcg_kernel<double>", "bound": "alu", "achieved": a64["tflops"],
                              "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": a64["tflops"] / FP64_PEAK_TFLOPS,
                              "peak_kind": "derived (152 SMs x 2 DFMA/clk x 2.07 GHz)", "hbm_gbs": a64["gbs"],
                              "us_per_pcg_iter": a64["us_per_pcg_iter"]},
                 "clocks": clk64},
        "final_cost": a32["final_cost"],
        "final_cost_rel_diff_vs_fp64": abs(a32["final_cost"] - a64["final_cost"]) / a64["final_cost"],
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": s32 and sum(s["kernel_launches"] for s in s32),
        "layer": layer,
        "clocks": clk32,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
