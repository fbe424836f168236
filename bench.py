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
import tempfile
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
# ncu dram__bytes_read.sum + dram__bytes_write.sum per 4096^2 launch of the
# current FP32 pass kernels (one full capture of one forward transform; the
# column kernel: the mean of passes 2 and 4). Reset whenever a kernel changes.
NCU_TRAFFIC = {"pass_kernel_pair<4096, 0, 1>": 213.2e6, "pass_kernel_pair<4096, 1, 4>": 214.8e6,
               "pass_kernel_pair<4096, 0, 2>": 207.9e6, "pass_kernel_pair<4096, 0, 3>": 208.0e6,
               "pass_kernel_pair<4096, 0, 5>": 212.5e6}
# the kernel (as ncu names it) that runs each pass of the forward transform:
# the line-pair kernel's template arguments are (length, column pass, mode),
# the mode naming the first and last transform directions of the pass
PASS_KERNELS = {
    ("fp32", 5): ["pass_kernel_pair<4096, 0, 1>", "pass_kernel_pair<4096, 1, 4>", "pass_kernel_pair<4096, 0, 2>",
                  "pass_kernel_pair<4096, 1, 4>", "pass_kernel_pair<4096, 0, 3>"],
    ("fp32", 3): ["pass_kernel_pair<4096, 0, 5>", "pass_kernel_pair<4096, 1, 4>", "pass_kernel_pair<4096, 0, 3>"],
    ("mixed", 5): ["pass_kernel_tc<0>", "pass_kernel_tc<1>", "pass_kernel_tc<0>", "pass_kernel_tc<1>",
                   "pass_kernel_tc<0>"],
    ("mixed", 3): ["pass_kernel_tc<0>", "pass_kernel_tc<1>", "pass_kernel_tc<0>"],
}
# tensor-core work of the split-precision kernel per sample and per stage: a
# data row of R = 64 complex samples (K = 128 real inputs, three FP16 products:
# K = 384) times the 128-output real-block DFT_R matrix, 2 * 384 * 128 / 64
# flops; a pass runs two stages per 1D transform
TC_FLOPS_PER_SAMPLE_STAGE = 2 * 384 * 128 // 64
# the split-precision tcgen05 kernel (one capture of passes 1-3 of a forward,
# profiles/pass_kernel_tc_4096x4096_ncu.md; rows: mean of passes 1 and 3)
NCU_TRAFFIC_MIXED = {"pass_kernel_tc<1>": 215.0e6, "pass_kernel_tc<0>": 213.3e6}
# ncu sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_elapsed / 100, same capture
TC_PIPE_ACTIVE = {"pass_kernel_tc<1>": 0.226, "pass_kernel_tc<0>": 0.249}
# the same for the batched kernel (256 fields {128..2048}^2, all batched; row
# kernel: mean of passes 1, 3, 5; profiles/batch_and_adjoint_kernels_dram.md)
# and the adjoint kernel (64 x 1024^2)
NCU_TRAFFIC_BATCH = {"batch_pass_kernel<0, 128>": 2.149e9}
NCU_TRAFFIC_GRAD = {"dual_pass_kernel<float, 1024, 0>": 2.088e9, "dual_pass_kernel<float, 1024, 1>": 2.089e9}
H_CHOICE = {"ha": "HA (Eq. HA24), five passes", "lc_y": "LC (Eq. LC10, H = (0,0;0,h)), three passes"}
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
    PERIOD_S = 0.05

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"nslct_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # start timing only once samples are flowing; the samples taken
            # before that are left out of the summary
            deadline = time.time() + 5.0
            while time.time() < deadline and self._lines() == 0:
                time.sleep(0.02)
            self.skip = self._lines()
        except Exception:
            self.proc = None
        return self

    def _lines(self) -> int:
        try:
            with open(self.path) as f:
                return sum(1 for ln in f if ln.count(",") >= 8)
        except OSError:
            return 0

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(self.PERIOD_S * 1.5)  # the sample that closes the region
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
            lines = [ln for ln in open(self.path) if ln.count(",") >= 8][getattr(self, "skip", 0):]
            for line in lines:
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


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: every rank contributes its own, all receive the max."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(samples_per_rank_step: int, ms_step: float, world: int) -> float:
    """Msamples/s over all ranks (replicas: every rank does the same step's work)."""
    return world * samples_per_rank_step / (ms_step * 1e-3) / 1e6


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


def _measure_step(N, torch, plans, x, outs, stream, steps, warmup, barrier, clocks=None):
    """Time `steps` steps of the 16 independent transforms (one nslct_forward_group
    call each), then each pass of every transform with events between passes.
    Returns (ms per step, mean ms of each pass)."""
    handles = [p.handle for p in plans]
    xs = [x] * len(plans)

    def step():
        N.nslct_forward_group(handles, xs, outs, stream)

    for _ in range(warmup):
        step()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if clocks is not None:
        clocks.__enter__()
    try:
        barrier()
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        barrier()
    finally:
        if clocks is not None:
            clocks.__exit__(None, None, None)
    ms_step = ev0.elapsed_time(ev1) / steps
    npass = plans[0].passes()
    iters = max(1, steps)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(npass + 1)] for _ in range(iters * len(plans))]
    barrier()
    k = 0
    for _ in range(iters):
        for p, o in zip(plans, outs):
            e = evs[k]
            e[0].record(stream)
            for j in range(npass):
                N.nslct_forward_pass(p.handle, j, x, o, stream)
                e[j + 1].record(stream)
            k += 1
    barrier()
    pass_ms = np.zeros(npass)
    for e in evs:
        for j in range(npass):
            pass_ms[j] += e[j].elapsed_time(e[j + 1])
    pass_ms /= len(evs)
    return ms_step, pass_ms


def _roofline_of(precision, npass, pass_ms, traffic):
    """The dominant kernel's roofline (see _dominant_roofline) and the chain's
    fraction of the 16 B per sample per pass model."""
    peak, _ = _peaks()
    bytes_launch = BYTES_PER_SAMPLE_PASS * NX * NY
    roof = _dominant_roofline(pass_ms, PASS_KERNELS[(precision, npass)], bytes_launch, traffic)
    chain_gbs = npass * bytes_launch / (pass_ms.sum() * 1e-3) / 1e9
    chain = {"pass_ms": [round(float(v), 5) for v in pass_ms], "modelled_bytes_per_sample": npass * BYTES_PER_SAMPLE_PASS,
             "achieved_gbs": chain_gbs, "frac_of_hbm": chain_gbs / peak,
             "compulsory_frac": 16 * NX * NY / (pass_ms.sum() * 1e-3) / 1e9 / peak}
    return roof, chain


def run_gpu(args, world, rank, local):
    import torch
    from paper_1707_03688_gb300 import nslct as N
    from paper_1707_03688_gb300 import build as B
    if not os.path.exists(N.LIB_PATH):
        B.build()
    N.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    g, mats = _make_inputs()
    plans = [N.Plan(m, NX, NY, precision=args.precision, method=args.method, decomposition=args.decomposition)
             for m in mats]
    npass = plans[0].passes()
    if any(p.passes() != npass for p in plans):
        raise RuntimeError("plans of one bench run must share their pass count")
    x = torch.from_numpy(g).to(torch.complex64).to(dev)
    outs = [torch.empty_like(x) for _ in range(N_ABCD)]
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # the transforms of a step are independent: one library call enqueues them
    # alternately on two streams, so one transform's passes fill the last
    # partial wave of the other's. Timed region: device events on the
    # launching stream, clocks sampled meanwhile.
    clk = ClockSampler(dev.index)
    ms_step, pass_ms = _measure_step(N, torch, plans, x, outs, stream, args.steps, args.warmup, barrier, clk)
    ms_step = max_over_ranks(ms_step, world, dev)
    samples_step = N_ABCD * NX * NY
    value = whole_job_value(samples_step, ms_step, world)
    roof, chain = _roofline_of(args.precision, npass, pass_ms, NCU_TRAFFIC)

    # ---- end to end: pinned host input -> device -> 16 transforms -> pinned host outputs.
    # Each output's device->host copy runs on a copy stream while the next
    # transform computes; the step ends when the last copy has landed.
    host_in = torch.from_numpy(g).to(torch.complex64).pin_memory()
    host_outs = [torch.empty((NX, NY), dtype=torch.complex64).pin_memory() for _ in range(N_ABCD)]
    x_e2e = torch.empty_like(x)
    # one copy stream (four concurrent device-to-host streams measured slower:
    # 7.4 vs 21.7 Gsamples/s end to end)
    copy_streams = [torch.cuda.Stream(dev)]
    done = [torch.cuda.Event() for _ in range(N_ABCD)]

    def e2e_step():
        x_e2e.copy_(host_in, non_blocking=True)
        for k, (p, o, h, ev) in enumerate(zip(plans, outs, host_outs, done)):
            N.nslct_forward(p.handle, x_e2e, o, stream)
            ev.record(stream)
            cs = copy_streams[k % len(copy_streams)]
            cs.wait_event(ev)
            with torch.cuda.stream(cs):
                h.copy_(o, non_blocking=True)
        for cs in copy_streams:
            stream.wait_stream(cs)

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
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev) / e2e_steps
    e2e_value = whole_job_value(samples_step, e2e_ms, world)

    result = {
        "metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f16-split+f32", "data": "synthetic",
        "config": {"workload": (WORKLOAD if args.method == "ha" else WORKLOAD.replace("HA-NsDLCT", "LC-NsDLCT"))
                   + ("" if args.decomposition == "type1" else f", decomposition {args.decomposition}"),
                   "nx": NX, "ny": NY, "n_abcd": N_ABCD, "precision": args.precision,
                   "h_choice": H_CHOICE[args.method], "passes": npass, "parallelism": f"replicas x{world}",
                   "streams": "nslct_forward_group: the 16 independent transforms alternate over two CUDA streams",
                   "l2": "no flush: 16 distinct 128 MiB outputs per step, working set 2.1 GB > 126 MB L2"},
        "gpu_launches": args.steps * N_ABCD * npass,
        "roofline": roof,
        "chain": chain,
        "e2e": {"value": e2e_value, "unit": "Msamples/s", "h2d_bytes_per_step": NX * NY * 8,
                "d2h_bytes_per_step": N_ABCD * NX * NY * 8},
        "clocks": clk.summary(),
    }

    # ---- the split-precision tensor-core form on the same GPU in the same run
    mixed_outs = None
    if args.precision == "fp32" and not args.no_mixed:
        mplans = [N.Plan(m, NX, NY, precision="mixed", method=args.method, decomposition=args.decomposition)
                  for m in mats]
        mixed_outs = [torch.empty_like(x) for _ in range(N_ABCD)]
        mclk = ClockSampler(dev.index)
        m_ms, m_pass = _measure_step(N, torch, mplans, x, mixed_outs, stream, args.steps, args.warmup, barrier, mclk)
        m_ms = max_over_ranks(m_ms, world, dev)
        m_roof, m_chain = _roofline_of("mixed", npass, m_pass, NCU_TRAFFIC_MIXED)
        # tensor-core work of the dominant kernel per launch: two stages per
        # 1D transform of its passes (five-pass chain: 1, 2, 2, 2, 1 transforms;
        # three-pass chain: 3, 2, 1), averaged over the passes it runs
        ntrs = [1, 2, 2, 2, 1] if npass == 5 else [3, 2, 1]
        names = PASS_KERNELS[("mixed", npass)]
        dom = [t for t, nm in zip(ntrs, names) if nm == m_roof["kernel"]]
        m_flops = TC_FLOPS_PER_SAMPLE_STAGE * 2 * (sum(dom) / len(dom)) * NX * NY
        result["mixed"] = {
            "value": whole_job_value(samples_step, m_ms, world), "unit": "Msamples/s", "ms_per_step": m_ms,
            "dtype": "f16-split+f32",
            "vs_fp32": (whole_job_value(samples_step, m_ms, world) / value) if value else None,
            "roofline": m_roof, "chain": m_chain,
            "tensor": {"flops_per_launch": m_flops, "achieved_tflops": m_flops / (m_roof["avg_launch_ms"] * 1e-3) / 1e12,
                       "pipe_tensor_active": TC_PIPE_ACTIVE.get(m_roof["kernel"])},
            "clocks": mclk.summary(),
        }
        for p in mplans:
            p.close()

    # ---- CPU baseline and rel-L2: the oracle on one 4096^2 transform (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import nslct_oracle as O
        p0 = plans[0]
        if p0.info()["flags"] & N.NSLCT_TYPE2:
            # a type-2 plan reports the type-1 factors of M^-1 with H = -H1
            params = O.decompose_type2(p0.info()["abcd"], -p0.params()["H"])
            t0 = time.perf_counter()
            ref = O.forward_type2(g, params, p0.dx, p0.dy)
        else:
            params = O.decompose(p0.info()["abcd"], p0.params()["H"])
            t0 = time.perf_counter()
            ref = O.forward(g, params, p0.dx, p0.dy)
        t_cpu = time.perf_counter() - t0
        gpu_out = outs[0].cpu().numpy().astype(np.complex128)
        result["rel_l2"] = {f"{args.precision}_vs_oracle": O.rel_l2(gpu_out, ref), "field": "ABCD seed 200, 4096^2",
                            "tolerance": 2e-5 if args.precision == "fp32" else 1e-4}
        if mixed_outs is not None:
            # both precisions plan ABCD seed 200 with the same H (the same search)
            err = O.rel_l2(mixed_outs[0].cpu().numpy().astype(np.complex128), ref)
            result["rel_l2"]["mixed_vs_oracle"] = err
            result["mixed"]["rel_l2_vs_oracle"] = err
            result["mixed"]["tolerance"] = 1e-4
        result["cpu_baseline"] = {"value": NX * NY / t_cpu / 1e6, "unit": "Msamples/s", "cores": _blas_threads(),
                                  "kind": "oracle",
                                  "sample": "one 4096x4096 forward transform (ABCD seed 200), FP64 dense DFT-matrix sums",
                                  "seconds": t_cpu}
    if rank == 0:
        print(json.dumps(result), flush=True)
    for p in plans:
        p.close()


def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _pass_times(run_pass, npass, iters, stream):
    """Mean duration (ms) of each of npass passes, run in order `iters` times
    with CUDA events between them on `stream`."""
    import torch
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(npass + 1)] for _ in range(iters)]
    for e in evs:
        e[0].record(stream)
        for k in range(npass):
            run_pass(k)
            e[k + 1].record(stream)
    torch.cuda.synchronize()
    return np.mean([[e[k].elapsed_time(e[k + 1]) for k in range(npass)] for e in evs], axis=0)


def _dominant_roofline(pass_ms, names, bytes_launch, traffic=None):
    """Roofline of the kernel (as ncu names it) with the largest share of the
    passes' time: algorithmic bytes per launch over its mean launch time."""
    per = {}
    for j, name in enumerate(names):
        tot, n = per.get(name, (0.0, 0))
        per[name] = (tot + float(pass_ms[j]), n + 1)
    dom = max(per, key=lambda k: per[k][0])
    ms = per[dom][0] / per[dom][1]
    peak, kind = _peaks()
    achieved = bytes_launch / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": (traffic or {}).get(dom), "kernel": dom, "share": per[dom][0] / float(np.sum(pass_ms)),
            "peak_source": f"hbm_gbs ({kind})", "bytes_per_launch": bytes_launch, "avg_launch_ms": ms}


def run_batch_workload(args, world, rank):
    """256 fields with Nx, Ny drawn from {128, ..., 2048}, each with its own ABCD:
    the batched persistent launches (captured in one CUDA graph) against the
    same transforms launched field by field."""
    import torch
    from paper_1707_03688_gb300 import inputs as I
    from paper_1707_03688_gb300 import nslct as N
    N.load()
    sizes = [128, 192, 256, 384, 512, 768, 1024, 1536, 2048]
    rng = np.random.default_rng(3)
    shapes = [(int(rng.choice(sizes)), int(rng.choice(sizes))) for _ in range(256)]
    abcds = [I.random_symplectic_abcd(30000 + k) for k in range(len(shapes))]
    b = N.Batch(abcds, shapes)
    ins = [torch.from_numpy(I.blob_field(nx, ny, seed=31000 + k)).to(torch.complex64).cuda()
           for k, (nx, ny) in enumerate(shapes)]
    outs = [torch.empty_like(x) for x in ins]
    b.bind(ins, outs)
    stream = torch.cuda.Stream()
    samples = sum(nx * ny for nx, ny in shapes)
    with torch.cuda.stream(stream):
        ms_each = _timed(lambda: b.forward_each(stream), args.steps, args.warmup, stream)
        b.set_split(1 << 30)
        if args.batch_threads:
            # pinned CTA size (for profiling captures of one variant): the first
            # batched launches of the run use it
            b.set_threads(args.batch_threads)
        ms_all_batched = _timed(lambda: b.forward(stream), args.steps, args.warmup, stream)
        split, _ = b.tune(stream, iters=2)
        # the tuned CTA size with every field batched: each pass is one
        # persistent launch over all samples
        th_all = b.threads
        b.set_split(1 << 30)
        pass_ms = _pass_times(lambda k: b.forward_pass(k, stream), 5, max(1, args.steps // 5), stream)
        b.set_split(split)
        ms_launch = _timed(lambda: b.forward(stream), args.steps, args.warmup, stream)
        b.capture(stream)
        with ClockSampler(torch.cuda.current_device()) as clk:
            ms_graph = _timed(lambda: b.forward(stream), args.steps, args.warmup, stream)
    value = samples / (ms_graph * 1e-3) / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "256 fields, Nx and Ny each from {128,...,2048}, own ABCD per field, forward, "
                               "batched persistent launches (autotuned split) captured in one CUDA graph",
                   "samples_per_step": samples, "l2": "working set 2 x samples x 8 B > L2",
                   "tuned_split": split, "tuned_cta_threads": b.threads},
        "per_field_launches": {"ms_per_step": ms_each, "value": samples / (ms_each * 1e-3) / 1e6},
        "all_batched_no_graph": {"ms_per_step": ms_all_batched, "value": samples / (ms_all_batched * 1e-3) / 1e6},
        "tuned_no_graph": {"ms_per_step": ms_launch, "value": samples / (ms_launch * 1e-3) / 1e6},
        # five batched launches, plus one per column pass for the packed 3*2^a
        # lines at 128-thread CTAs, plus five per field run alone
        "gpu_launches": 5 + (2 if b.threads == 128 and any(
            nx & (nx - 1) and min(nx, ny) < split for nx, ny in shapes) else 0)
        + 5 * sum(1 for nx, ny in shapes if min(nx, ny) >= split),
        "clocks": clk.summary(),
        # the batched kernel with every field batched, passes timed one by one
        "roofline": _dominant_roofline(pass_ms, [f"batch_pass_kernel<{int(chain_col)}, {th_all}>"
                                                 for chain_col in (0, 1, 0, 1, 0)],
                                       BYTES_PER_SAMPLE_PASS * samples, NCU_TRAFFIC_BATCH),
        "pass_ms_all_batched": [round(float(v), 5) for v in pass_ms],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()


def _fft_chain_tables(params, nx, ny, dx, dy, device, cdtype):
    """Chirp tables of the chain for a library FFT (context only, not the
    product): chi_H and chi_B' over FFT bins (centred frequency k(b) = b for
    b < N/2, b - N above; spacing 2 pi / (N d); sign -), CM^{C2} and CM^{C1}
    over centred samples (sign +). Phases in FP64, tables in `cdtype`."""
    import torch

    def quad(c, a, b, da, db, sign):
        c = np.asarray(c, dtype=np.float64)
        c12 = 0.5 * (c[0, 1] + c[1, 0])
        ph = 0.5 * (c[0, 0] * (a * da) ** 2 + 2.0 * c12 * (a * da) * (b * db) + c[1, 1] * (b * db) ** 2)
        return torch.polar(torch.ones_like(ph), sign * ph).to(cdtype)

    f64 = dict(dtype=torch.float64, device=device)
    bx, by = torch.arange(nx, **f64), torch.arange(ny, **f64)
    kx = torch.where(bx < nx // 2, bx, bx - nx)[:, None]
    ky = torch.where(by < ny // 2, by, by - ny)[None, :]
    mx, my = (bx - nx // 2)[:, None], (by - ny // 2)[None, :]
    dwx, dwy = 2 * math.pi / (nx * dx), 2 * math.pi / (ny * dy)
    return (quad(params["H"], kx, ky, dwx, dwy, -1.0), quad(params["C2"], mx, my, dx, dy, 1.0),
            quad(params["Bp"], kx, ky, dwx, dwy, -1.0), quad(params["C1"], mx, my, dx, dy, 1.0))


def _fft_chain(x, tabs):
    """CM^{C1} CC^{B'} CM^{C2} CC^{H} x with CC^B = -(1/(Nx Ny)) IFFT_u(chi_B FFT(.))
    = -ifft2(chi_B fft2(.)); the two CCs' signs cancel."""
    import torch
    chi_h, cm2, chi_b, cm1 = tabs
    y = torch.fft.fft2(x)
    y.mul_(chi_h)
    y = torch.fft.ifft2(y)
    y.mul_(cm2)
    y = torch.fft.fft2(y)
    y.mul_(chi_b)
    y = torch.fft.ifft2(y)
    y.mul_(cm1)
    return y


def run_libfft_workload(args, world, rank):
    """Context only, not the product: the same 16 transforms of the 4096^2
    field as a library chain (torch.fft, i.e. cuFFT: two fft2, two ifft2 and
    four table multiplies per transform, chirp tables precomputed from each
    plan's own H, B', C1, C2), beside the library's fused passes on the same
    GPU, and the two outputs' agreement."""
    import torch
    from paper_1707_03688_gb300 import nslct as N
    N.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    g, mats = _make_inputs()
    plans = [N.Plan(m, NX, NY) for m in mats]
    x = torch.from_numpy(g).to(torch.complex64).to(dev)
    tabs = [_fft_chain_tables(p.params(), NX, NY, p.dx, p.dy, dev, torch.complex64) for p in plans]
    outs = [torch.empty_like(x) for _ in plans]
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        ours = plans[0].forward(x)
        lib = _fft_chain(x, tabs[0])
        stream.synchronize()
        agree = float((torch.linalg.vector_norm(lib - ours) / torch.linalg.vector_norm(ours)).item())

        def lib_step():
            for t in tabs:
                _fft_chain(x, t)

        def our_step():
            for p, o in zip(plans, outs):
                p.forward(x, out=o)

        with ClockSampler(dev.index) as clk:
            ms_lib = _timed(lib_step, args.steps, args.warmup, stream)
            ms_ours = _timed(our_step, args.steps, args.warmup, stream)
    samples = N_ABCD * NX * NY
    line = {
        "metric": "context: library-FFT chain vs the fused passes, forward NsDLCT Msamples/s",
        "value": samples / (ms_lib * 1e-3) / 1e6, "unit": "Msamples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_lib, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + "; torch.fft (cuFFT) chain with precomputed chirp tables, one stream",
                   "nx": NX, "ny": NY, "n_abcd": N_ABCD},
        "fused_same_run": {"value": samples / (ms_ours * 1e-3) / 1e6, "ms_per_step": ms_ours,
                           "note": "nslct_forward per transform on one stream"},
        "ratio_fused_over_library": ms_lib / ms_ours,
        "rel_l2_library_vs_fused": agree,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    for p in plans:
        p.close()


def run_filter_workload(args, world, rank):
    """Filtering in two NsLCT domains (Sec. 5.B) on the 4096^2 field: Eq. Add04
    (two masked forwards, two inverses) and Eq. Add08 (two masked forwards,
    one inverse of the composed matrix), each captured in one CUDA graph."""
    import torch
    from paper_1707_03688_gb300 import inputs as I
    from paper_1707_03688_gb300 import nslct as N
    N.load()
    # a smooth 2048^2 field zero-padded to the 4096^2 grid (the paper's remedy
    # for aliasing, Sec. 5.A): the first forward pads on load, the last inverse
    # crops back to 2048^2
    n0 = NX // 2
    g = I.blob_field(n0, n0, seed=FIELD_SEED, width_range=(40.0, 160.0))
    m1, m3 = I.random_symplectic_abcd(300), I.random_symplectic_abcd(301)
    d = math.sqrt(2 * math.pi / NX)
    q1 = N.Plan(m1, n0, n0, dx=d, dy=d, pad=(NX, NY))
    q3 = N.Plan(m3, NX, NY, dx=d, dy=d)
    q31 = N.Plan(m3 @ m1, n0, n0, dx=d, dy=d, pad=(NX, NY))
    x = torch.from_numpy(g).to(torch.complex64).cuda()
    big = torch.empty((NX, NY), dtype=torch.complex64, device="cuda")
    h1 = torch.from_numpy(I.gaussian_mask(NX, NY, 0.3, tilt=2.0)).to(torch.complex64).cuda()
    h3 = torch.from_numpy(I.gaussian_mask(NX, NY, 0.4)).to(torch.complex64).cuda()
    y1, y2, y3 = (torch.empty_like(big) for _ in range(3))
    out04, out08 = torch.empty_like(x), torch.empty_like(x)

    def add04():
        q1.forward(x, out=y1, mask=h1)
        q3.forward(y1, out=y2, mask=h3)
        q3.inverse(y2, out=y3)
        q1.inverse(y3, out=out04)

    def add08():
        q1.forward(x, out=y1, mask=h1)
        q3.forward(y1, out=y2, mask=h3)
        q31.inverse(y2, out=out08)

    stream = torch.cuda.Stream()
    graphs = {}
    with torch.cuda.stream(stream):
        for _ in range(2):
            add04()
            add08()
    torch.cuda.synchronize()
    for name, fn in (("add04", add04), ("add08", add08)):
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=stream):
            fn()
        graphs[name] = gr
    res = {}
    with torch.cuda.stream(stream), ClockSampler(torch.cuda.current_device()) as clk:
        for name, gr in graphs.items():
            res[name] = _timed(gr.replay, args.steps, args.warmup, stream)
    torch.cuda.synchronize()
    diff = float((torch.linalg.vector_norm(out08 - out04) / torch.linalg.vector_norm(out04)).item())
    n = NX * NY   # samples of the grid each transform runs on
    line = {
        "metric": "NsLCT-domain filtering Msamples/s (Eq. Add08 pipeline)", "value": n / (res["add08"] * 1e-3) / 1e6,
        "unit": "Msamples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["add08"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "2048x2048 complex64 field zero-padded to a 4096x4096 grid, Gaussian masks in the "
                               "M1 and M3 domains (ABCD seeds 300, 301), output cropped to 2048x2048, "
                               "each pipeline one CUDA graph",
                   "transforms": {"add04": 4, "add08": 3}},
        "add04": {"ms_per_step": res["add04"], "value": n / (res["add04"] * 1e-3) / 1e6},
        "rel_l2_add08_vs_add04": diff,
        "gpu_launches": 3 * 5, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    for q in (q1, q3, q31):
        q.close()


def run_grad_workload(args, world, rank):
    """Batch of 64 fields of 1024 x 1024 sharing one ABCD: forward, loss
    ||L(x) - y||^2 and the backward pass with gradients for x and the 10 ABCD
    parameters (summed over the batch), each pass one launch over the batch."""
    import torch
    from paper_1707_03688_gb300 import inputs as I
    from paper_1707_03688_gb300 import nslct as N
    N.load()
    n, nb = 1024, 64
    m = I.random_symplectic_abcd(4)
    plan = N.Plan(m, n, n)
    # targets: seeded target fields under the perturbed parameters theta + N(0, 0.05^2)
    theta = plan.theta()
    delta = np.random.default_rng(4).normal(0.0, 0.05, size=10)
    target_plan = N.Plan.from_theta(theta + delta, n, n, h0=plan.params()["H"])
    x = torch.from_numpy(np.stack([I.blob_field(n, n, seed=4000 + k) for k in range(nb)])).to(torch.complex64).cuda()
    xt = torch.from_numpy(np.stack([I.blob_field(n, n, seed=5000 + k) for k in range(nb)])).to(torch.complex64).cuda()
    yt = target_plan.forward(xt)
    torch.cuda.synchronize()
    del xt
    target_plan.close()
    y = torch.empty_like(x)
    gy = torch.empty_like(x)
    gx = torch.empty_like(x)
    ws = torch.empty_like(x)
    gth = torch.zeros(10, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        N.nslct_forward_many(plan.handle, x, y, stream)
        torch.sub(y, yt, out=gy)
        gy.mul_(2)
        N.nslct_backward_many(plan.handle, gy, y, gx, gth, None, ws, stream)

    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = _timed(step, args.steps, args.warmup, stream)
    value = nb * n * n / (ms * 1e-3) / 1e6
    # the forward alone, and the five dual passes of the backward one by one
    ms_fwd = _timed(lambda: N.nslct_forward_many(plan.handle, x, y, stream), args.steps, args.warmup, stream)
    pass_ms = _pass_times(lambda k: N.nslct_backward_pass(plan.handle, k, gy, y, gx, ws, stream), 5,
                          max(1, args.steps // 5), stream)
    # moving the parameters between optimisation steps: a fresh theta plan
    # (FP64 host derivation, device tables and workspace allocated and uploaded)
    # against nslct_plan_theta_set on one plan (the same host derivation only)
    h0 = plan.params()["H"]
    reps = 20
    t0 = time.perf_counter()
    for k in range(reps):
        pk = N.Plan.from_theta(theta + 1e-4 * k, n, n, h0=h0)
        pk.close()
    torch.cuda.synchronize()
    replan_ms = (time.perf_counter() - t0) * 1e3 / reps
    moved = N.Plan.from_theta(theta, n, n, h0=h0)
    t0 = time.perf_counter()
    for k in range(reps * 50):
        moved.set_theta(theta + 1e-6 * (k % 7))
    set_us = (time.perf_counter() - t0) * 1e6 / (reps * 50)
    moved.close()
    # each dual pass reads and writes two complex64 fields (gradient and value paths)
    roof = _dominant_roofline(pass_ms, [f"dual_pass_kernel<float, {n}, {c}>" for c in (0, 1, 0, 1, 0)],
                              2 * BYTES_PER_SAMPLE_PASS * nb * n * n, NCU_TRAFFIC_GRAD)
    roof["share"] = roof["share"] * float(np.sum(pass_ms)) / ms
    line = {
        "metric": "forward + backward (x and ABCD-parameter gradients) Msamples/s", "value": value,
        "unit": "Msamples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "64 x 1024^2 complex64 sharing one ABCD, loss ||L(x) - y||^2 with y = "
                               "L_{theta+delta}(x_target), delta ~ N(0, 0.05^2) on the 10 ABCD parameters, "
                               "nslct_forward_many + nslct_backward_many",
                   "note": "the residual 2(y - y_t) is formed with torch ops between the two library calls"},
        "gpu_launches": 5 + 5 + 1, "clocks": clk.summary(),
        # share: of the whole step (forward, residual, backward, finalisation)
        "roofline": roof,
        "forward_ms": ms_fwd, "backward_pass_ms": [round(float(v), 5) for v in pass_ms],
        "theta_update": {"fresh_plan_ms": replan_ms, "plan_theta_set_us": set_us,
                         "note": "host time per parameter update; the step itself does neither"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 150, about 0.8 s of FP32 and 1.8 s of split-precision transforms, "
                         "so that the clock sampler sees the timed region; 10 for --impl reference, whose step "
                         "takes ~14 s)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="leave out the split-precision form that the default line reports beside FP32")
    ap.add_argument("--workload", default="fp32", choices=["fp32", "batch", "grad", "filter", "libfft"],
                    help="fp32: 4096^2 x 16 ABCD (the benchmark line); batch: 256 uneven fields; "
                         "grad: 64 x 1024^2 forward + backward; filter: two-domain filtering, Eqs. Add04/Add08; "
                         "libfft: context only, the same transforms as a torch.fft (cuFFT) chain")
    ap.add_argument("--method", default="ha", choices=["ha", "lc_y"],
                    help="H of Eq. HA24 (five passes) or of Eq. LC10 (three passes)")
    ap.add_argument("--decomposition", default="type1", choices=["type1", "type2", "trace"],
                    help="CM-CC-CM-CC (Eq. HA28), CC-CM-CC-CM (Eq. CCCMCCCM16) or the tr(B) rule (Eq. Reversible08)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed"],
                    help="fp32: FP32 FFT arithmetic; mixed: 4096-point lines as four-step DFT-64 stages on the "
                         "tensor cores (split FP16, FP32 accumulation)")
    ap.add_argument("--batch-threads", type=int, default=0, choices=[0, 128, 256, 512],
                    help="--workload batch: CTA size of the first all-batched launches (0: the library default)")
    ap.add_argument("--n-abcd", type=int, default=16,
                    help="ABCD matrices per step (16 is the benchmark workload; fewer only for profiling captures)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else 150
    global N_ABCD
    N_ABCD = max(1, min(16, args.n_abcd))
    world, rank, local = _dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batch":
        run_batch_workload(args, world, rank)
    elif args.workload == "grad":
        run_grad_workload(args, world, rank)
    elif args.workload == "filter":
        run_filter_workload(args, world, rank)
    elif args.workload == "libfft":
        run_libfft_workload(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
