"""Benchmark of the 2D NsDLCT (CM-CC-CM-CC chain) on GB300.

Workload (one step): a 4096 x 4096 complex64 field (8 complex Gaussian blobs +
CN(0, 0.05^2) white noise, seed 2) transformed by 16 random symplectic ABCD
matrices (seeds 200..215), i.e. 16 forward HA-NsDLCTs of 4096^2 samples, each
into its own output buffer (working set 2.1 GB, far above the 126 MB L2, so no
L2 flush is needed between steps).

Prints ONE JSON line (rank 0). Metric: forward-transform Msamples/s. Also:
* roofline of the dominant kernel (per-pass CUDA events in the same run),
* e2e: the same metric with the input copied from pinned host memory and all
  16 outputs copied back inside the timed region,
* cpu_baseline: the FP64 oracle timed on this host on one 4096^2 transform,
* rel_l2 of that transform against the oracle,
* clocks sampled with nvidia-smi during the timed region.

``--impl reference`` times the oracle (the only reference this method has: the
paper publishes formulas, not code) on the same workload, one 4096^2
transform per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX = NY = 4096
N_ABCD = 16
FIELD_SEED = 2
NOISE_SEED = 102
ABCD_SEED0 = 200
BYTES_PER_SAMPLE_PASS = 16        # read + write one complex64 per sample per pass
PASSES = 5
METRIC = "2D NsLCT Msamples/s and % HBM roofline, mixed vs FP32 at stated rel-L2 error"
WORKLOAD = ("4096x4096 complex64 field (8 Gaussian blobs + 5% complex white noise), 16 random "
            "symplectic ABCD, forward HA-NsDLCT per ABCD")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local) if args.impl != "reference" else None
        dist.init_process_group("nccl" if args.impl != "reference" else "gloo")
    elif args.impl != "reference":
        torch.cuda.set_device(0)
    return world, rank, local


def _make_inputs():
    from paper_1707_03688_gb300 import inputs as I
    g = I.add_white_noise(I.blob_field(NX, NY, seed=FIELD_SEED), sigma=0.05, seed=NOISE_SEED)
    mats = [I.random_symplectic_abcd(ABCD_SEED0 + k) for k in range(N_ABCD)]
    return g, mats


def run_reference(args, world, rank):
    """Oracle arm: one FP64 direct-sum 4096^2 transform per step, rank 0 only."""
    if rank != 0:
        return
    from oracle import nslct_oracle as O
    g, mats = _make_inputs()
    d = math.sqrt(2 * math.pi / NX)
    plans = [O.plan(m) for m in mats[: max(1, min(N_ABCD, args.warmup + args.steps))]]
    for k in range(args.warmup):
        O.forward(g, plans[k % len(plans)], d, d)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        O.forward(g, plans[(args.warmup + k) % len(plans)], d, d)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * NX * NY / total / 1e6
    cores = _blas_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "n_abcd": N_ABCD,
                                        "reference_step": "one 4096^2 transform (of the 16) per step"},
        "cpu_baseline": {"value": value, "unit": "Msamples/s", "cores": cores, "kind": "oracle",
                         "sample": "one 4096x4096 forward transform per step, FP64 dense DFT-matrix sums"},
        "e2e": {"value": value, "unit": "Msamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import torch
    from paper_1707_03688_gb300 import nslct as N
    from paper_1707_03688_gb300 import build as B
    if not os.path.exists(N.LIB_PATH):
        B.build()
    N.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    g, mats = _make_inputs()
    plans = [N.Plan(m, NX, NY) for m in mats]
    x = torch.from_numpy(g).to(torch.complex64).to(dev)
    outs = [torch.empty_like(x) for _ in range(N_ABCD)]
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step():
        for p, o in zip(plans, outs):
            N.nslct_forward(p.handle, x, o, stream)

    # ---- warm-up
    for _ in range(args.warmup):
        step()
    barrier()

    # ---- timed region (device events on the launching stream)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        barrier()
    ms_total = ev0.elapsed_time(ev1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    samples_step = N_ABCD * NX * NY
    value = world * samples_step / (ms_step * 1e-3) / 1e6

    # ---- per-pass durations (same work, events between the five passes)
    npass_iters = max(1, args.steps)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(PASSES + 1)] for _ in range(npass_iters * N_ABCD)]
    barrier()
    k = 0
    for _ in range(npass_iters):
        for p, o in zip(plans, outs):
            e = evs[k]
            e[0].record(stream)
            for j in range(PASSES):
                N.nslct_forward_pass(p.handle, j, x, o, stream)
                e[j + 1].record(stream)
            k += 1
    barrier()
    pass_ms = np.zeros(PASSES)
    for e in evs:
        for j in range(PASSES):
            pass_ms[j] += e[j].elapsed_time(e[j + 1])
    pass_ms /= len(evs)
    peak, peak_kind = _peaks()
    bytes_launch = BYTES_PER_SAMPLE_PASS * NX * NY
    # the dominant kernel: the column pass (kernels 1 and 3 are the same kernel)
    col_ms = 0.5 * (pass_ms[1] + pass_ms[3])
    row_ms = (pass_ms[0] + pass_ms[2] + pass_ms[4]) / 3
    dom_ms, dom_name = (col_ms, "pass_kernel<float,4096,col>") if col_ms >= row_ms else \
        (row_ms, "pass_kernel<float,4096,row>")
    achieved = bytes_launch / (dom_ms * 1e-3) / 1e9
    chain_gbs = PASSES * bytes_launch / (pass_ms.sum() * 1e-3) / 1e9

    # ---- end to end: pinned host input -> device -> 16 transforms -> pinned host outputs
    host_in = torch.from_numpy(g).to(torch.complex64).pin_memory()
    host_outs = [torch.empty((NX, NY), dtype=torch.complex64).pin_memory() for _ in range(N_ABCD)]
    x_e2e = torch.empty_like(x)

    def e2e_step():
        x_e2e.copy_(host_in, non_blocking=True)
        for p, o, h in zip(plans, outs, host_outs):
            N.nslct_forward(p.handle, x_e2e, o, stream)
            h.copy_(o, non_blocking=True)

    e2e_steps = max(1, min(args.steps, 5))
    e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_value = world * samples_step / (e2e_ms * 1e-3) / 1e6

    result = {
        "metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "n_abcd": N_ABCD, "precision": "fp32",
                   "h_choice": "HA (Eq. HA24)", "parallelism": f"replicas x{world}",
                   "l2": "no flush: 16 distinct 128 MiB outputs per step, working set 2.1 GB > 126 MB L2"},
        "gpu_launches": args.steps * N_ABCD * PASSES,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": dom_name,
                     "peak_source": f"hbm_gbs ({peak_kind})",
                     "bytes_per_launch": bytes_launch, "avg_launch_ms": dom_ms},
        "chain": {"pass_ms": [round(v, 5) for v in pass_ms], "modelled_bytes_per_sample": PASSES * BYTES_PER_SAMPLE_PASS,
                  "achieved_gbs": chain_gbs, "frac_of_hbm": chain_gbs / peak,
                  "compulsory_frac": 16 * NX * NY / (pass_ms.sum() * 1e-3) / 1e9 / peak},
        "e2e": {"value": e2e_value, "unit": "Msamples/s", "h2d_bytes_per_step": NX * NY * 8,
                "d2h_bytes_per_step": N_ABCD * NX * NY * 8},
        "clocks": clk.summary(),
    }

    # ---- CPU baseline and rel-L2: the oracle on one 4096^2 transform (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import nslct_oracle as O
        p0 = plans[0]
        params = O.decompose(p0.info()["abcd"], p0.params()["H"])
        t0 = time.perf_counter()
        ref = O.forward(g, params, p0.dx, p0.dy)
        t_cpu = time.perf_counter() - t0
        gpu_out = outs[0].cpu().numpy().astype(np.complex128)
        result["rel_l2"] = {"fp32_vs_oracle": O.rel_l2(gpu_out, ref), "field": "ABCD seed 200, 4096^2",
                            "tolerance": 2e-5}
        result["cpu_baseline"] = {"value": NX * NY / t_cpu / 1e6, "unit": "Msamples/s", "cores": _blas_threads(),
                                  "kind": "oracle",
                                  "sample": "one 4096x4096 forward transform (ABCD seed 200), FP64 dense DFT-matrix sums",
                                  "seconds": t_cpu}
    if rank == 0:
        print(json.dumps(result), flush=True)
    for p in plans:
        p.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-abcd", type=int, default=16,
                    help="ABCD matrices per step (16 is the benchmark workload; fewer only for profiling captures)")
    args = ap.parse_args()
    global N_ABCD
    N_ABCD = max(1, min(16, args.n_abcd))
    world, rank, local = _dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
