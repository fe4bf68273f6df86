"""Benchmark of one stochastic DINR training step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--prec bf16|fp32] [--no-cpu-baseline]

Workload: parallel beam, 512 views over 4 rotations, 128 x 128 detector,
128 samples per ray, 10-octave encoding (84 inputs), MLP 5 x 256 ReLU,
65,536 rays per step (8,388,608 samples); 16 moving, growing ellipsoids
give the measurements. A step is the whole hot path: minibatch draw, ray
generation, encoding, MLP forward, forward model and loss, backward, Adam.
Metric: training ray-samples per second (whole job over all ranks). A
serving leg replays a seeded Poisson stream of mixed queries (time slices,
sub-volumes, re-projections) against the query server of a cone-beam 6 x 256
network and adds p50/p99 latency and outputs/s under "serving". An
equal-error leg trains the FP32 path for 1,000 steps and the BF16 path from
the same weights on the same minibatches until it reaches the FP32 path's
final reconstruction error against the phantom, and reports the wall time
each path takes to that error ("equal_error").

Our arm runs the library (default BF16 tensor-core path; the plain FP32 path
is timed beside it). The timed steps are replayed from the library's CUDA
graph of one step (dinr_train_graph); per-kernel times (roofline, shares)
come from the same number of steps run again as ordinary, event-timed
launches. The reference arm (--impl reference) times the FP64 CPU
oracle on a bounded ray sample of the same workload on the host cores.
One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
from dataclasses import replace
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "train ray-samples/s"
WORKLOAD = 2
FP32_SIMT_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x FMA x max clock


# DRAM bytes per sample of the fused kernels, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over the launch / samples of
# the launch; 1,048,576-sample cases of the parallel-beam workloads 2 (ReLU,
# octave encoding) and 6 (GRFF + Swish), summarised in profiles/). Valid only
# for the kernel source the counters were taken on: a different source hash
# reports traffic as null.
# Either bytes per sample of every launch, or (for kernels whose bytes per
# launch vary by layer) the measured DRAM bytes over the algorithmic bytes of
# the captured launch, applied to each launch's algorithmic bytes.
_CSRC = "paper_2404_19075_b300/csrc/"
_CHAIN = {"source": [_CSRC + f for f in ("tc_chain.cu", "tc_chain.cuh", "tc_ptx.cuh")],
          "sha256_16": "0b95c887b4baf3b9"}
TRAFFIC = {"tc_fwd_chain": [dict(_CHAIN, bf16_workload=2,
                                 bytes_per_sample=(10.45888e6 + 2.507943e9) / 1048576)],
           "tc_bwd_chain": [dict(_CHAIN, bf16_workload=2,
                                 bytes_per_sample=(176.600064e6 + 2.624401e9) / 1048576)],
           "tc_dw": [{"ratio_to_algorithmic": (1.074876e9 + 4.859648e6) / (2 * 1048576 * 256 * 2),
                      "bf16_workload": 2,
                      "source": [_CSRC + f for f in ("tc_gemm.cu", "tc_gemm.cuh", "tc_ptx.cuh",
                                                     "tc_pair.cuh")],
                      "sha256_16": "ef0ab8935cae0d04"}]}

# Kernels without tensor-core work of the method: their roofline is GB/s of
# algorithmic bytes. Every other BF16 / FP8 kernel is measured against the
# tensor pipe on the method's own FLOPs (the MLP GEMMs of the step); its HBM
# figure (algorithmic bytes, stored activations included) is kept beside it.
HBM_BOUND = {"dw_out", "encode"}


def source_hash(paths):
    """First 16 hex digits of the SHA-256 of the files' bytes, concatenated."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_of(kernel, workload, samples, alg_bytes):
    """DRAM bytes of one launch from the recorded counters, or None when
    there are none for this kernel and workload or its source has changed."""
    t = next((e for e in TRAFFIC.get(kernel, []) if e["bf16_workload"] == workload), None)
    if t is None:
        return None
    if source_hash(t["source"]) != t["sha256_16"]:
        return None
    if "bytes_per_sample" in t:
        return t["bytes_per_sample"] * samples
    return t["ratio_to_algorithmic"] * alg_bytes


def roofline_of(name, k, pk, src, prec, workload, samples_per_launch):
    """Roofline entry of one profiled kernel (k: launches, ms, flops, bytes
    summed over its launches). Tensor-core kernels: achieved = the method's
    FLOPs per launch / mean launch time, against the sustained BF16 peak
    (the kernels run inside a long step) and, as frac_burst, the burst
    peak; their algorithmic HBM bytes per launch over the same time under
    "hbm"."""
    t = k["ms"] / k["launches"] / 1e3                       # seconds per launch
    hbm = {"achieved": k["bytes"] / k["launches"] / t / 1e9, "peak": pk["hbm_gbs"],
           "unit": "GB/s", "peak_source": f"hbm_gbs ({src})"}
    hbm["frac"] = hbm["achieved"] / hbm["peak"]
    if name in HBM_BOUND or (prec in ("bf16", "fp8") and k["flops"] <= 0):
        r = dict(hbm, bound="hbm")
    elif prec == "bf16" or prec == "fp8":
        ach = k["flops"] / k["launches"] / t / 1e12
        scale = 2 if prec == "fp8" else 1
        peak = pk["bf16_tflops_sustained"] * scale
        r = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
             "peak_source": ("2 x " if prec == "fp8" else "") + f"bf16_tflops_sustained ({src})",
             "frac_burst": ach / (pk["bf16_tflops"] * scale),
             "peak_burst": pk["bf16_tflops"] * scale, "hbm": hbm}
    else:
        ach = k["flops"] / k["launches"] / t / 1e12
        r = {"bound": "alu", "achieved": ach, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
             "peak_source": "148 SMs x 128 FP32 lanes x 2 x 2032 MHz"}
    r["frac"] = r["achieved"] / r["peak"]
    r["kernel"] = name
    r["launches"] = k["launches"]
    r["ms_per_launch"] = 1e3 * t
    r["traffic"] = (traffic_of(name, workload, samples_per_launch, k["bytes"] / k["launches"])
                    if prec != "fp32" else None)
    r["traffic_unit"] = "bytes per launch (DRAM read + write)"
    return r


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def config(w, extra=None):
    g, net = w.geom, w.net
    c = {"workload": ("parallel-beam 512 views x 128x128 detector, S=128, 10-octave encoding, "
                      "MLP 5x256 ReLU, 65536 rays/step") if w.index == WORKLOAD else w.name,
         "rays_per_step": w.train.batch_rays, "samples_per_ray": g.samples_per_ray,
         "samples_per_step": w.train.batch_rays * g.samples_per_ray,
         "mlp": f"{net.hidden_layers}x{net.width}", "d_in": net.d_in,
         "l2": "inputs larger than L2 (activations of a step are tens of GB)"}
    if extra:
        c.update(extra)
    return c


def algorithmic_flops_per_sample(net):
    """2 * sum(fan_in * fan_out) forward, twice that backward minus the
    first layer's input gradient (not computed)."""
    pw = sum(o * i for o, i in net.layer_shapes())
    return 2 * pw + 4 * pw - 2 * net.d_in * net.width


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        for ln in out.splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 8:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        load = [r for r in self.rows if (num(r[3]) or 0) > 50] or self.rows
        sm = [num(r[0]) for r in load if num(r[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in load for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(load[0][1]), "samples": len(load), "reasons": reasons}


def oracle_rate(w, n_rays, seed=11):
    """The FP64 oracle's samples/s on n_rays rays of the workload (one full
    forward + backward + Adam step on that sample)."""
    from oracle import phantom as oph, step as ostep
    from synthetic import workloads as wl
    g, net = w.geom, w.net
    idx = wl.ray_subset(g.n_proj, n_rays, seed)
    proj = np.zeros(g.n_proj)
    proj[idx] = oph.projections(wl.phantom(w), g, idx)
    th = wl.he_init(net, w.seeds["weights"])
    t0 = time.perf_counter()
    out = ostep.train_step(th, np.zeros_like(th), np.zeros_like(th), 1, g, net, w.train, idx, proj)
    dt = time.perf_counter() - t0
    samples = int(out["n_pix"].sum()) if "n_pix" in out else n_rays * g.samples_per_ray
    return samples / dt, dt


def cpu_baseline(w, n_rays=2048):
    rate, dt = oracle_rate(w, n_rays)
    return {"value": rate, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n_rays} rays x {w.geom.samples_per_ray} samples of the workload, one "
                      f"FP64 step (numpy, BLAS threads = host cores), {dt:.1f} s"}


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    from synthetic import workloads as wl
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = wl.workload(args.workload)
    n_rays = 256
    for _ in range(args.warmup):
        oracle_rate(w, n_rays, seed=7)
    samples, total = 0.0, 0.0
    for k in range(args.steps):
        r, dt = oracle_rate(w, n_rays, seed=100 + k)
        samples += r * dt
        total += dt
    value = samples / total
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config(w, {"reference_sample_rays_per_step": n_rays}),
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{n_rays} rays x {w.geom.samples_per_ray} samples "
                                       "per step"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_steps(model, steps, n, graph=False):
    """Seconds for `steps` training steps of n sampled rays, CUDA events on
    the context stream: replayed from the library's graph of one step, or
    as ordinary launches (every launch event-timed when profiling)."""
    import torch
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    if graph:
        model.train_graph(n, steps, sync=False)
    else:
        for _ in range(steps):
            model.train_step(None, n=n, sync=False)
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2404_19075_b300 import Dinr, DinrError, phantom_project
    from synthetic import workloads as wl

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    w = wl.workload(args.workload)
    if args.rays:
        w = replace(w, train=replace(w.train, batch_rays=args.rays))
    g, net = w.geom, w.net
    B, S = w.train.batch_rays, g.samples_per_ray
    proj = phantom_project(g, wl.phantom(w))            # measurements, resident in HBM
    theta = wl.he_init(net, w.seeds["weights"]).astype(np.float32)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    results = {}
    precs = [args.prec] + ([p for p in ("fp32",) if p != args.prec] if args.compare else [])
    for prec in precs:
        try:
            m = Dinr(g, net, w.train, proj, prec=prec, init_params=theta,
                     sampler_seed=w.seeds["sampler"] + 1000 * rank, recompute=args.recompute)
        except DinrError as e:
            results[prec] = {"error": str(e)}
            continue
        steps = args.steps if prec == args.prec else max(2, args.steps // 4)
        # warm-up steps replayed from the step graph (the first captures it)
        m.train_graph(B, args.warmup, sync=False)
        barrier()
        m.profile(True)
        m.profile(False)          # clears the launch counter; graph replays need profiling off
        with Clocks(local) as ck:
            barrier()
            dt = time_steps(m, steps, B, graph=True)
            barrier()
        launches = m.profile_report()["total_launches"]["launches"]
        dt = max_over_ranks(dt)
        # per-kernel times: the same number of steps again as ordinary
        # launches with every launch event-timed
        m.profile(True)
        dt_ordinary = time_steps(m, steps, B)
        m.profile(False)
        prof = m.profile_report()
        loss = m.loss()
        # end to end through the public API: each step's host indices (pinned,
        # drawn before the timed region like a loader's prefetched batches)
        # copied in by the library, the loss read back
        rng = np.random.default_rng(rank)
        e2e_steps = max(2, steps // 2)
        idx_host = torch.from_numpy(rng.integers(0, g.n_proj, (e2e_steps, B))).pin_memory()
        barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            m.train_step_host(idx_host[k], sync=True)
        barrier()
        e2e_dt = max_over_ranks(time.perf_counter() - t0)
        results[prec] = dict(dt=dt, steps=steps, prof=prof, clocks=ck.summary(), loss=loss,
                             e2e=ws * e2e_steps * B * S / e2e_dt, launches=launches,
                             dt_ordinary=dt_ordinary)
        m.close()
    if args.equal_error_steps > 0:
        try:
            results["equal_error"] = run_equal_error(args, w, proj, theta, rank)
        except Exception as e:                       # reported, not hidden
            results["equal_error"] = {"error": repr(e)}
    if args.serve_queries > 0:
        try:
            results["serving"] = run_serving(args, rank)
        except Exception as e:                       # reported, not hidden
            results["serving"] = {"error": repr(e)}
    if rank == 0:
        emit(args, w, results, ws)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def settled_at(curve, target):
    """The first scored point of `curve` from which the error stays at or
    below `target` to the end (None if the last point is above it). The
    error is not monotone early in training: a nearly empty volume scores
    about 0.94 before the phantom takes shape, so the first point below the
    target alone could be that early one."""
    k = len(curve)
    while k > 0 and curve[k - 1]["rel_l2"] <= target:
        k -= 1
    return curve[k] if k < len(curve) else None


def run_equal_error(args, w, proj, theta, rank):
    """Time to equal reconstruction error on the BF16 and FP32 paths (same
    initial weights, same minibatch stream). The FP32 path trains
    `equal_error_steps` steps; its final error is the target. The BF16 path
    trains the same steps, scored at the same points, and then goes on,
    scored every fifth of the interval, for up to as many steps again until
    its error reaches the target; a path's time to the target is the wall
    time at the first scored step from which its error stays at or below
    it. Error: relative L2 (and PSNR) of mu0 M
    against the phantom's attenuation on a 64^3 grid inside the field of
    view, at 8 view times. Wall times exclude the scoring."""
    import torch

    from paper_2404_19075_b300 import Dinr
    from synthetic import truth, workloads as wl

    g, net = w.geom, w.net
    B, steps = w.train.batch_rays, args.equal_error_steps
    every = max(1, min(args.equal_error_every, steps))
    fine = max(1, every // 5)
    ph = wl.phantom(w)
    times = [(k + 0.5) / 8 for k in range(8)]
    mask = truth.fov_mask(64)
    gt = [truth.attenuation_grid(ph, t, 64) for t in times]
    out = {"steps": steps, "grid": "64^3 cell centres inside the FOV cylinder",
           "times": times, "batch_rays": B, "lr": w.train.lr}
    target = None
    for prec in ("fp32", "bf16"):
        m = Dinr(g, net, w.train, proj, prec=prec, init_params=theta,
                 sampler_seed=w.seeds["sampler"] + 1000 * rank)
        curve, wall, done = [], 0.0, 0

        def advance(n):
            nonlocal wall, done
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(n):
                m.train_step(None, n=B, sync=False)
            torch.cuda.synchronize()
            wall += time.perf_counter() - t0
            done += n
            sc = [truth.scores(m.query_grid(t, (-1, -1, -1), (1, 1, 1), (64, 64, 64))
                               .cpu().numpy(), gt_t, mask) for t, gt_t in zip(times, gt)]
            curve.append({"step": done, "wall_s": wall, "loss": m.loss(),
                          "rel_l2": float(np.mean([x["rel_l2"] for x in sc])),
                          "psnr_db": float(np.mean([x["psnr_db"] for x in sc]))})

        while done < steps:
            advance(min(every, steps - done))
        at_steps = dict(curve[-1])
        if prec == "fp32":
            target = at_steps["rel_l2"]
        else:
            while curve[-1]["rel_l2"] > target and done < 2 * steps:
                advance(min(fine, 2 * steps - done))
        hit = settled_at(curve, target)
        out[prec] = {"rel_l2": at_steps["rel_l2"], "psnr_db": at_steps["psnr_db"],
                     "loss": at_steps["loss"], "wall_s": at_steps["wall_s"],
                     "samples_per_s": steps * B * g.samples_per_ray / at_steps["wall_s"],
                     "steps_to_fp32_final_error": hit["step"] if hit else None,
                     "wall_s_to_fp32_final_error": hit["wall_s"] if hit else None,
                     "curve": curve}
        m.close()
    out["target_rel_l2"] = target
    out["bf16_over_fp32_rel_l2"] = out["bf16"]["rel_l2"] / target
    # equal error: the BF16 path reaches the FP32 path's final error
    out["equal_error"] = out["bf16"]["wall_s_to_fp32_final_error"] is not None
    if out["equal_error"]:
        tb = out["bf16"]["wall_s_to_fp32_final_error"]
        out["time_to_equal_error_speedup"] = out["fp32"]["wall_s_to_fp32_final_error"] / tb
        # the FP32 path's samples (what that error took it) over the BF16
        # path's wall time to the same error
        out["bf16_samples_per_s_at_equal_error"] = (
            out["fp32"]["steps_to_fp32_final_error"] * B * g.samples_per_ray / tb)
    return out


def run_serving(args, rank):
    """Query serving on the cone-beam 6x256 network: a seeded Poisson stream
    of mixed time slices, sub-volumes and re-projections (256^2 detector,
    256 samples per ray) replayed against the continuous-batching server.
    Weights are the seeded initialisation of that architecture."""
    import torch

    from paper_2404_19075_b300 import Dinr, serving
    from synthetic import workloads as wl

    w = wl.workload(5)
    g, net = w.geom, w.net
    proj = torch.zeros(g.n_proj, device="cuda")
    theta = wl.he_init(net, w.seeds["weights"]).astype(np.float32)
    m = Dinr(g, net, replace(w.train, batch_rays=8192), proj, prec="bf16", init_params=theta)
    m.serve_config(max_batch_samples=args.serve_batch)
    warm = wl.query_stream(6, rate=1e6, seed=4999)
    serving.run(m, warm)
    qs = wl.query_stream(args.serve_queries, rate=args.serve_rate, seed=5000 + rank)
    m.profile(True)
    with Clocks(torch.cuda.current_device()) as ck:
        res = serving.run(m, qs, time_limit=120.0)
    m.profile(False)
    prof = m.profile_report()
    # the same stream under the least-work-first schedule
    m.serve_policy("least_work")
    lw = serving.run(m, qs, time_limit=120.0)
    m.serve_policy("arrival")
    # a rate the server can carry: 70 % of the samples per second of device
    # time it served above, in requests of the stream's mean size; the same
    # queries (kinds, sizes) arrive at that rate, under both policies, and
    # the utilisation is the device time of the replay over its wall time
    busy_s = sum(v["ms"] for k, v in prof.items() if not k.startswith("total_")) / 1e3
    served = sum(serving.request_args(q)[3] for q in qs)
    mean_smp = served / len(qs)
    rate_sus = 0.7 * (served / busy_s) / mean_smp if busy_s > 0 else None
    sus = None
    if rate_sus:
        qs2 = wl.query_stream(args.serve_queries, rate=rate_sus, seed=5000 + rank)
        m.profile(True)
        r2 = serving.run(m, qs2, time_limit=120.0)
        m.profile(False)
        p2 = m.profile_report()
        busy2 = sum(v["ms"] for k, v in p2.items() if not k.startswith("total_")) / 1e3
        m.serve_policy("least_work")
        lw2 = serving.run(m, qs2, time_limit=120.0)
        m.serve_policy("arrival")
        sus = {"arrival_rate_per_s": rate_sus,
               "offered_samples_per_s": rate_sus * mean_smp,
               "capacity_samples_per_s": served / busy_s,
               "utilisation": busy2 / r2["wall"],
               "p50_ms": r2.get("p50_ms"), "p99_ms": r2.get("p99_ms"),
               "completed": r2["completed"], "outputs_per_s": r2["outputs_per_s"],
               "least_work_policy": {"p50_ms": lw2.get("p50_ms"), "p99_ms": lw2.get("p99_ms"),
                                     "completed": lw2["completed"]}}
    # 4D export: 8 volumes of 256^3 streamed to pinned host memory
    ex_dims, ex_times = (256, 256, 256), [(k + 0.5) / 8 for k in range(8)]
    sums = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.export(ex_times, (-1, -1, -1), (1, 1, 1), ex_dims,
             lambda k, t, vol: sums.append(float(vol[0, 0, 0])))
    ex_wall = time.perf_counter() - t0
    n_vox = len(ex_times) * ex_dims[0] * ex_dims[1] * ex_dims[2]
    export = {"volumes": len(ex_times), "dims": list(ex_dims), "wall_s": ex_wall,
              "voxels_per_s": n_vox / ex_wall, "host_gb_per_s": 4 * n_vox / ex_wall / 1e9}
    m.close()
    chain = prof.get("tc_serve_chain", {"ms": float("nan"), "flops": 0, "launches": 0})
    pk, src = peaks()
    tf = chain["flops"] / (chain["ms"] / 1e3) / 1e12 if chain["ms"] else None
    kinds = {k: sum(1 for q in qs if q.kind == k) for k in ("slice", "subvolume", "reprojection")}
    return {"metric": "query voxels/s (outputs: voxels and detector pixels)",
            "value": res["outputs_per_s"], "unit": "outputs/s",
            "samples_per_s": res["samples_per_s"],
            "p50_ms": res.get("p50_ms"), "p99_ms": res.get("p99_ms"),
            "policy": "arrival order",
            "least_work_policy": {"p50_ms": lw.get("p50_ms"), "p99_ms": lw.get("p99_ms"),
                                  "outputs_per_s": lw["outputs_per_s"],
                                  "completed": lw["completed"]},
            "queries": len(qs), "completed": res["completed"], "wall_s": res["wall"],
            "arrival_rate_per_s": args.serve_rate, "mix": kinds,
            "arrivals_span_s": qs[-1].arrival,
            "max_batch_samples": args.serve_batch,
            "chain": {"launches": chain["launches"], "ms": chain["ms"], "tflops": tf,
                      "frac_of_bf16_sustained": tf / pk["bf16_tflops_sustained"] if tf else None,
                      "peak_source": f"bf16_tflops_sustained ({src})"},
            "gpu_launches": prof.get("total_launches", {}).get("launches"),
            "utilisation": busy_s / res["wall"],
            "sustainable_rate": sus,
            "export_4d": export,
            "clocks": ck.summary(),
            "config": "cone beam SOD 4 / SDD 8, MLP 6x256 ReLU, 10-octave encoding; "
                      "slices 128^2..1024^2, sub-volumes 32^3..256^3, re-projections "
                      "256^2 x 256 samples; seeded Poisson arrivals"}


def emit(args, w, results, ws):
    g, net = w.geom, w.net
    B, S = w.train.batch_rays, g.samples_per_ray
    main = results[args.prec]
    if "error" in main:
        print(json.dumps({"metric": METRIC, "error": main["error"]}), flush=True)
        return
    pk, src = peaks()
    prof = main["prof"]
    prof.pop("total_launches", None)
    launches = main["launches"]
    counted = prof.pop("total_samples", {}).get("launches")
    # samples per step: B S with one ray per pixel; counted by the library
    # with the App. A model (a variable number per pixel)
    S_step = counted / main["steps"] if g.subpixels and counted else B * S
    value = ws * main["steps"] * S_step / main["dt"]
    kern = {k: v for k, v in prof.items()}
    top = max(kern, key=lambda k: kern[k]["ms"])
    tk = kern[top]
    per_launch = S_step * main["steps"] / max(1, tk["launches"])   # samples per launch
    roof = roofline_of(top, tk, pk, src, args.prec, w.index, per_launch)
    major = {name: roofline_of(name, k, pk, src, args.prec, w.index,
                               S_step * main["steps"] / max(1, k["launches"]))
             for name, k in kern.items() if k["ms"] >= 0.1 * tk["ms"] and k["launches"] > 0}
    total_ms = sum(v["ms"] for v in kern.values())
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws,
            "steps": main["steps"], "warmup": args.warmup,
            "ms_per_step": 1e3 * main["dt"] / main["steps"], "higher_is_better": True,
            "ms_per_step_ordinary_launches": 1e3 * main["dt_ordinary"] / main["steps"],
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": config(w, {"parallelism": f"replicas{ws}" if ws > 1 else "single GPU",
                                 "step_launch": "replayed CUDA graph of one step",
                                 "prec": args.prec, "samples_per_step": S_step,
                                 **({"forward_model": f"App. A, {g.subpixels}x{g.subpixels} "
                                                      "sub-pixel rays, samples per pixel vary"}
                                    if g.subpixels else {})}),
            "tflops_algorithmic": value * algorithmic_flops_per_sample(net) / 1e12,
            **({"tflops_frac_sustained": value * algorithmic_flops_per_sample(net) / 1e12
                / pk["bf16_tflops_sustained"],
                "tflops_frac_burst": value * algorithmic_flops_per_sample(net) / 1e12
                / pk["bf16_tflops"]} if args.prec == "bf16" else {}),
            "roofline": roof,
            "rooflines": major,
            "kernel_shares": {k: round(v["ms"] / total_ms, 4) for k, v in kern.items()},
            "clocks": main["clocks"], "gpu_launches": launches,
            "e2e": {"value": main["e2e"] * S_step / (B * S), "unit": "samples/s",
                    "h2d_bytes_per_step": 8 * B, "d2h_bytes_per_step": 4},
            "loss_last": main["loss"]}
    for key in ("equal_error", "serving"):
        extra = results.pop(key, None)
        if extra is not None:
            line[key] = extra
    for p, r in results.items():
        if p != args.prec:
            line[f"{p}_path"] = ({"error": r["error"]} if "error" in r else
                                 {"value": ws * r["steps"] * S_step / r["dt"], "unit": "samples/s",
                                  "ms_per_step": 1e3 * r["dt"] / r["steps"]})
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp32", "fp8"])
    ap.add_argument("--no-compare", dest="compare", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rays", type=int, default=0,
                    help="rays per step (default: the workload's 65,536); smaller batches "
                         "are for profiler captures, not bench lines")
    ap.add_argument("--workload", type=int, default=WORKLOAD, choices=[2, 3, 4, 6, 8],
                    help="training workload (default: the benchmark workload 2; 3 and 4 are "
                         "the cone-beam 6x256 and 8x512 networks, 6 the paper's GRFF + Swish "
                         "network on the geometry of 2, 8 the same with the App. A forward "
                         "model)")
    ap.add_argument("--recompute", type=int, default=0,
                    help="activation recomputation of the unfused BF16 path (0, 1, -1 auto)")
    ap.add_argument("--equal-error-steps", type=int, default=1000,
                    help="Adam steps of the FP32 path in the time-to-equal-error comparison "
                         "(its final error is the target; BF16 runs up to twice as many; "
                         "0 skips it)")
    ap.add_argument("--equal-error-every", type=int, default=250,
                    help="steps between scorings of the reconstruction in that comparison")
    ap.add_argument("--serve-queries", type=int, default=200,
                    help="queries of the serving leg (0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--serve-batch", type=int, default=1 << 21,
                    help="samples per serving launch at most")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
