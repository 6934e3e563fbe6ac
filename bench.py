"""Benchmark: solver iterations per second and time to the simplified field
on the 256^3 warm-start evaluation field.

Workload (`warm_start_256`): the mean of a 64-bump Gaussian mixture and a
64-loop filament field plus U[0, 0.05) noise, normalised to [0, 1], signal
threshold 0.05 of the range (seed 5; about 3.3 M diagram points at f_0).

One step = one solver iteration (Algorithm 1): gradient step, persistence
diagram of the new field (vertex order, lower-star gradient, critical cells,
D0/D2/D1 pairs), still pairs and exact reduced assignment, loss.  Inputs are
resident in HBM; L2 is flushed (a 256 MiB write) before every timed step and
the step is timed with CUDA events on the solver's stream.  The headline
steps run without stage profiling; the same steps are then repeated on a
fresh field with per-stage CUDA events (no extra synchronisation) for the
stage table and the roofline of the dominant stage.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs N independent replicas (one per GPU, launched by torchrun): the
path has no exchange step, so there is no collective on the data path.
--impl reference times the CPU oracle (plain boundary-matrix reduction and the
same solver loop) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "warm_start_256"
SHAPE = (256, 256, 256)
SEED = 5
TAU = 0.05
METRIC = "solver iterations/s and time to the simplified field (256^3 fp32 field)"
UNIT = "iters/s"
CPU_BLOCK = 128  # the oracle's sample: the 128^3 octant of the field

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples (SM clock, throttle reasons) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def replica_throughput(total_ms, steps, world, device=None):
    """Whole-job iterations/s for `world` independent replicas: every rank ran
    `steps` iterations; the job took as long as the slowest rank (max-reduce,
    the only collective; the path itself exchanges nothing)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1e3), total_ms


def make_field():
    """The 256^3 field (about half a minute of numpy); cached per host in the
    temporary directory so a second run on the same machine reuses it."""
    from paper_2407_12399_gb300 import synthetic
    import tempfile
    path = os.path.join(tempfile.gettempdir(), f"tsf_bench_{WORKLOAD}_{SHAPE[0]}_seed{SEED}.npy")
    if os.path.exists(path):
        try:
            f = np.load(path)
            if f.shape == SHAPE and f.dtype == np.float32:
                return f
        except Exception:
            pass
    f = synthetic.warm_start_field(SHAPE, seed=SEED)
    try:
        tmp = path + f".{os.getpid()}.tmp.npy"
        np.save(tmp, f)
        os.replace(tmp, path)
    except Exception:
        pass
    return f


def host_info():
    """Cores and model of the host CPU (the oracle's hardware)."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    mem = None
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemTotal:"):
                    mem = round(int(line.split()[1]) / 1e6, 1)
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model, "arch": platform.machine(), "mem_gb": mem}


def differentiable_loss(evals=10):
    """Differentiable topological loss (96^3 Gaussian mixture, 32 bumps, 5 %
    noise; signal >= 0.1 of the range; the field is moved by U(-0.005, 0.005)
    so signal pairs have a non-zero gradient): device time of one
    tsf_loss_and_gradient call on the whole field, and of a call after one
    vertex value changed (the diagram follows the change incrementally)."""
    import torch

    import paper_2407_12399_gb300 as tsf
    from paper_2407_12399_gb300 import synthetic as S
    f0 = S.mixture_96()
    rng = np.random.default_rng(7)
    f = (f0 + rng.uniform(-0.005, 0.005, f0.shape)).astype(np.float32)
    fld = tsf.Field(torch.from_numpy(f0).cuda())
    fld.set_threshold(0.1)
    ft = torch.from_numpy(f).cuda()
    gt = torch.empty(f.shape, dtype=torch.float64, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    loss, _ = fld.loss_and_grad(ft, gt)
    ev1.record()
    torch.cuda.synchronize()
    first = ev0.elapsed_time(ev1)
    flat = ft.view(-1)
    times = []
    for k in range(evals):
        flat[1000 + 37 * k] += 1e-3
        ev0.record()
        fld.loss_and_grad(ft, gt)
        ev1.record()
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
    st = fld.step(stop_s=0.0)
    return {"workload": "mixture_96", "grid": [96, 96, 96], "signal_threshold": 0.1, "loss": loss,
            "points": int(st["n_points"]), "ms_full_evaluation": first,
            "ms_after_one_change": float(np.median(times)), "evaluations_per_s": 1e3 / float(np.median(times))}


def batched_solve(prec=0.01, converge_tau=0.025):
    """Batched solve of 48 independent uneven fields (per-axis dims from
    {48, 64, 96, 128, 160}, 16-bump mixtures + 5 % noise, thresholds
    U[0.02, 0.2]), every field on its own stream, the assignment by the
    auction at relative precision 0.01 (Section 5's setting).  Measured,
    batch against the same fields one at a time: (a) targets plus the first
    solver iteration of all 48 fields; (b) time to the simplified field of
    the fields with threshold >= converge_tau (the others, with 10^4
    targets inside the noise, need seconds per later iteration in the
    assignment)."""
    import torch

    import paper_2407_12399_gb300 as tsf
    from paper_2407_12399_gb300 import synthetic as S
    fields, taus = S.uneven_batch()
    dev = [torch.from_numpy(f).cuda() for f in fields]
    torch.cuda.synchronize()
    vox = int(sum(f.size for f in fields))
    kw = dict(stop_s=0.01, assignment_precision=prec)

    def first_iteration_batch():
        free0 = torch.cuda.mem_get_info()[0]
        b = tsf.Batch(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.set_thresholds(taus)
        st = b.step(**kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        gb = (free0 - torch.cuda.mem_get_info()[0]) / 1e9
        b.close()
        return dt, st, gb

    def first_iteration_lone():
        t = 0.0
        for f, tau in zip(dev, taus):
            x = tsf.Field(f)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x.set_threshold(float(tau))
            x.step(**kw)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            x.close()
        return t

    # the batch autotuner picks the D1 phase-A schedule on these fields' own
    # diagrams (process-wide choice; results never depend on it)
    bt = tsf.Batch(dev)
    choice, tune_ms = bt.autotune()
    bt.close()
    tb, st, gb = first_iteration_batch()
    tl = first_iteration_lone()
    targets = [int(s["n_points"]) for s in st]
    sub = [i for i, tau in enumerate(taus) if tau >= converge_tau]

    b = tsf.Batch([dev[i] for i in sub])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.set_thresholds(taus[sub])
    sts = b.simplify(**kw)
    torch.cuda.synchronize()
    tcb = time.perf_counter() - t0
    iters_b = int(sum(x["iters"] for x in sts))
    done = int(sum(x["done"] for x in sts))
    b.close()
    tcl = 0.0
    for i in sub:
        x = tsf.Field(dev[i])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x.set_threshold(float(taus[i]))
        tsf.tsf_simplify(x._h, tsf.params(**kw))
        torch.cuda.synchronize()
        tcl += time.perf_counter() - t0
        x.close()
    crowded = [{"field": i, "grid": list(fields[i].shape), "signal_threshold": float(taus[i])}
               for i in range(len(fields)) if i not in sub]
    tsf.tsf_debug_set(7, 0)
    return {"workload": "uneven_batch_48", "fields": len(fields), "voxels": vox, "assignment_precision": prec,
            "autotune": {"candidates": ["half warp 64+128", "half warp 32+64", "quarter warp 16+32", "warp 64+128"],
                         "diagram_ms": tune_ms, "chosen": choice},
            "first_iteration": {"batch_s": tb, "one_at_a_time_s": tl, "speedup": tl / tb,
                                "field_iterations_per_s": len(fields) / tb, "device_gb": gb},
            "to_simplified_field": {"fields": len(sub), "threshold_min": converge_tau, "batch_s": tcb,
                                    "one_at_a_time_s": tcl, "speedup": tcl / tcb, "iterations": iters_b,
                                    "converged": done, "iterations_per_s": iters_b / tcb},
            "not_run_to_convergence": crowded,
            "diagram_points_after_first_step": {"min": min(targets), "max": max(targets)}}


def oracle_octant_iteration(f0, warmup=0):
    """One oracle iteration (gradient step, plain reduction of the full
    lexicographic filtration, still pairs, exact reduced assignment) on the
    128^3 octant of the field, single-threaded; the octant's own diagram
    (iteration 0) is computed first and not timed."""
    import oracle
    oracle.build()
    b = CPU_BLOCK
    crop = np.ascontiguousarray(f0[:b, :b, :b])
    s = oracle.Solver(crop, tau=TAU)
    for _ in range(warmup):
        s.iterate(stop_s=0.0)
    return s


def cpu_sample_text(dt, steps):
    scale = float(CPU_BLOCK ** 3) / float(np.prod(SHAPE))
    return (f"{steps} oracle iteration(s) on the {CPU_BLOCK}^3 octant of the {SHAPE[0]}^3 field, "
            f"{dt / steps:.1f} s each on one core; value = octant iterations/s x {scale:.4f} (vertex ratio; the "
            f"reduction grows faster than the vertex count, so this overstates the oracle's 256^3 rate)"), scale


def cpu_baseline(f0, steps=1):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    workload (its 128^3 octant)."""
    s = oracle_octant_iteration(f0)
    t = time.perf_counter()
    for _ in range(steps):
        s.iterate(stop_s=0.0)
    dt = time.perf_counter() - t
    text, scale = cpu_sample_text(dt, steps)
    return {"value": steps / dt * scale, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": text,
            "octant_iteration_s": dt / steps, "host": host_info()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    f0 = make_field()
    s = oracle_octant_iteration(f0, warmup=args.warmup)
    t = time.perf_counter()
    for _ in range(args.steps):
        s.iterate(stop_s=0.0)
    dt = time.perf_counter() - t
    text, scale = cpu_sample_text(dt, args.steps)
    value = args.steps / dt * scale
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(SHAPE), "signal_threshold": TAU, "seed": SEED},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": text,
                             "host": host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# Algorithmic bytes per launch of each stage that streams memory (units of
# work per launch x the bytes one unit must move); the pairing stages
# (union-find rounds, the D1 reduction, the assignment) have no byte model:
# their work is O(#critical x path length) and they are latency-bound.
def stage_bytes(stage, st, nv, incremental_order):
    if stage == "vertex_order":
        # incremental merge: read order, skey; write order2, skey2, rank; or
        # the full radix sort: histogram, 4 passes of key+id, rank scatter
        return nv * (20.0 if incremental_order else 84.0), nv, "vertices"
    if stage == "gradient":
        # per recomputed lower star: 15 ranks + 14 values read; 32 B record,
        # 1 B descending-line pointer and the 144 B D1 table row written
        n = st["n_gradient_vertices"]
        return n * 293.0, n, "lower stars"
    if stage == "critical_cells":
        # per vertex in rank order: its 32 B record and 4 B order entry
        return nv * 36.0, nv, "vertices"
    if stage == "pairs_d1_morse":
        # per lower-star visit: its 144 B table row (the pending masks stay in
        # shared memory)
        n = st["d1_blocks_total"]
        return n * 144.0, n, "lower-star visits"
    return None, None, None


def run_steps(tsf, torch, f_dev, stream, flush, steps, profile):
    """A fresh field from f_dev with the target set, then `steps` solver
    iterations (stop rule off), each bracketed by CUDA events on the solver
    stream after an L2 flush.  Returns (per-step ms, stats, profile, launches)."""
    p = tsf.params(stop_s=0.0)
    fld = tsf.Field(f_dev, stream=stream)
    fld.set_threshold(TAU)
    if profile:
        tsf.tsf_profile_enable(fld._h, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stats = []
    torch.cuda.synchronize()
    launches0 = tsf.tsf_kernel_launches()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
            ev[k][0].record(stream)
        st = tsf.tsf_solver_step(fld._h, p)
        ev[k][1].record(stream)
        stats.append(st.as_dict())
    torch.cuda.synchronize()
    launches = tsf.tsf_kernel_launches() - launches0
    prof = tsf.tsf_profile_read(fld._h) if profile else None
    fld.close()
    return [a.elapsed_time(b) for a, b in ev], stats, prof, launches


def e2e_solve(tsf, host, stream, params):
    """Create from host values, set the signal threshold, simplify to the
    paper's stop rule and read the field back, all through the C ABI with
    host buffers; wall time and the solve's figures."""
    lz, ly, lx = host.shape
    t = time.perf_counter()
    h = tsf.tsf_create_field(lx, ly, lz, host.ctypes.data, 0, stream.cuda_stream)
    tsf.tsf_set_signal_threshold(h, TAU)
    out = np.empty_like(host)
    st = tsf.tsf_simplify(h, params, out.ctypes.data, 0)
    dt = time.perf_counter() - t
    tsf.tsf_destroy_field(h)
    diff = out.astype(np.float64) - host.astype(np.float64)
    return dt, st, out, {"l2_change": float(np.sqrt((diff ** 2).sum())), "linf_change": float(np.abs(diff).max())}


def secondary_filament_128(tsf, torch, stream, flush, steps):
    """The 128^3 filament field of the plain-solver parity configuration
    (threshold 0.05): iterations/s (device) and the end-to-end solve."""
    from paper_2407_12399_gb300 import synthetic
    f = synthetic.filament_field((128, 128, 128), seed=1)
    dev = torch.from_numpy(f).cuda()
    ms, stats, _, _ = run_steps(tsf, torch, dev, stream, flush, steps, False)
    dt, st, _, q = e2e_solve(tsf, np.ascontiguousarray(f), stream, tsf.params(stop_s=0.01))
    return {"workload": "filament_128", "grid": [128, 128, 128], "signal_threshold": 0.05,
            "iters_per_s": steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
            "e2e": {"iterations": int(st.iters), "time_to_simplified_field_s": dt, "loss0": float(st.loss0),
                    "final_loss": float(st.loss), "non_signal_remaining": int(st.n_uncancelled), **q}}


def ablation_128(tsf, stream):
    """Section 4.2 / 4.3 accelerations on and off (the paper's Table 2), at
    the filament field's threshold and at Appendix A's aggressive 45 %; then
    the cut and fill modes of Section 5.3 (alpha_d = 0, alpha_b = 0)."""
    import torch
    from paper_2407_12399_gb300 import synthetic
    host = np.ascontiguousarray(synthetic.filament_field((128, 128, 128), seed=1))

    def solve(tau, **kw):
        h = tsf.tsf_create_field(128, 128, 128, host.ctypes.data, 0, stream.cuda_stream)
        tsf.tsf_set_signal_threshold(h, tau)
        torch.cuda.synchronize()
        t = time.perf_counter()
        st = tsf.tsf_simplify(h, tsf.params(stop_s=0.01, **kw), None, 0)
        dt = time.perf_counter() - t
        tsf.tsf_destroy_field(h)
        return {"iterations": int(st.iters), "solve_s": dt, "iters_per_s": int(st.iters) / dt,
                "final_loss": float(st.loss), "non_signal_remaining": int(st.n_uncancelled)}

    out = {"workload": "filament_128"}
    for tau in (0.05, 0.45):
        runs = {}
        for fg in (1, 0):
            for fa in (1, 0):
                runs[f"gradient_update_{'fast' if fg else 'full'}/assignment_{'reuse' if fa else 'full'}"] = \
                    solve(tau, fast_gradient_update=fg, fast_assignment_update=fa)
        out[f"threshold_{tau:g}"] = runs
    out["modes"] = {"cut (alpha_d = 0)": solve(0.05, alpha_d=0.0), "fill (alpha_b = 0)": solve(0.05, alpha_b=0.0)}
    return out


def warm_start_block(tsf, torch, f0, stream):
    """Learned warm start (not in the paper) on the headline field: the
    network's g0 = net(f), then the solver from g0 against f's own targets,
    against the plain solve from f, both timed from host memory to the host
    result.  Reported: wall times, iterations, final losses, ||g - f||_2 and
    the non-signal pairs of D(f) each solve cancelled (the same set?)."""
    from paper_2407_12399_gb300 import warm_start as W
    if not os.path.exists(W.WEIGHTS):
        return {"unavailable": f"no trained weights at {os.path.relpath(W.WEIGHTS, ROOT)}"}
    net = W.load(W.WEIGHTS, stream=stream)
    fd = torch.from_numpy(np.ascontiguousarray(f0)).cuda()
    net.forward(fd, TAU)  # buffers for this grid
    torch.cuda.synchronize()
    g_plain, st_p, t_plain = W.solve(f0, TAU, stream=stream)
    g_warm, st_w, t_warm, t_inf = W.warm_solve(net, f0, TAU, stream=stream)
    theta = np.float32(np.float32(TAU) * np.float32(f0.max() - f0.min()))

    def keys(values, nonsignal_only):
        fld = tsf.Field(torch.from_numpy(np.ascontiguousarray(values)).cuda(), stream=stream)
        d = fld.diagram()
        fld.close()
        pers = d["death"] - d["birth"]
        sel = (d["essential"] == 0) & ((pers < theta) if nonsignal_only else (pers > 0))
        return set(zip(d["dim"][sel].tolist(), d["v_birth"][sel].tolist(), d["v_death"][sel].tolist()))

    nonsig = keys(f0, True)
    left_p, left_w = keys(g_plain, False) & nonsig, keys(g_warm, False) & nonsig
    canc_p, canc_w = nonsig - left_p, nonsig - left_w
    l2 = lambda g: float(np.sqrt(((g.astype(np.float64) - f0.astype(np.float64)) ** 2).sum()))
    return {"plain": {"wall_s": t_plain, "iterations": int(st_p.iters), "final_loss": float(st_p.loss),
                      "l2_to_f": l2(g_plain), "non_signal_cancelled": len(canc_p)},
            "warm": {"wall_s": t_warm, "inference_s": t_inf, "iterations": int(st_w.iters),
                     "final_loss": float(st_w.loss), "l2_to_f": l2(g_warm), "non_signal_cancelled": len(canc_w)},
            "non_signal_pairs_of_f": len(nonsig),
            "cancelled_sets_equal": canc_p == canc_w,
            "cancelled_symmetric_difference": len(canc_p ^ canc_w),
            "l2_ratio_warm_over_plain": l2(g_warm) / max(l2(g_plain), 1e-300),
            "speedup_plain_over_warm": t_plain / t_warm,
            "loss0": float(st_p.loss0)}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2407_12399_gb300 as tsf
    from paper_2407_12399_gb300 import build as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    tsf.lib()

    t_gen = time.perf_counter()
    f0 = make_field()
    t_gen = time.perf_counter() - t_gen
    nv = f0.size
    stream = torch.cuda.Stream()
    dev_f0 = torch.from_numpy(f0).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # warm-up on a separate field from the same input
    warm = tsf.Field(dev_f0, stream=stream)
    warm.set_threshold(TAU)
    for _ in range(args.warmup):
        tsf.tsf_solver_step(warm._h, tsf.params(stop_s=0.0))
    warm.close()

    # the headline: K iterations from f_0, no stage profiling
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        step_ms, stats, _, launches = run_steps(tsf, torch, dev_f0, stream, flush, args.steps, False)
    total_ms = float(sum(step_ms))
    value, total_ms = replica_throughput(total_ms, args.steps, world, device="cuda")
    if world > 1:
        dist.barrier()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # the same iterations with per-stage CUDA events: stage table, roofline
    prof_ms, prof_stats, prof, _ = run_steps(tsf, torch, dev_f0, stream, flush, args.steps, True)

    # end to end through the public API with host buffers: create from host
    # values, set the signal, simplify to the paper's stop rule, read back
    e2e = None
    if not args.no_e2e:
        host = np.ascontiguousarray(f0)
        e2e_solve(tsf, host[:64, :64, :64].copy(), stream, tsf.params(stop_s=0.01))  # allocator warm-up
        dt, st, _, q = e2e_solve(tsf, host, stream, tsf.params(stop_s=0.01))
        iters = max(int(st.iters), 1)
        e2e = {"value": iters / dt, "unit": UNIT, "h2d_bytes_per_step": int(4 * nv / iters),
               "d2h_bytes_per_step": int(4 * nv / iters), "iterations": int(st.iters),
               "time_to_simplified_field_s": dt,
               "timed": "tsf_create_field (host values) + tsf_set_signal_threshold + tsf_simplify (host output)",
               "stop_rule": "loss <= 0.01 loss_0 (Algorithm 1)", "loss0": float(st.loss0),
               "final_loss": float(st.loss), "points_final": int(st.n_points),
               "non_signal_remaining": int(st.n_uncancelled),
               "still_fraction_last": float(st.n_still) / max(int(st.n_points), 1), **q}

    hbm, peak_kind = peaks()
    n_upd = float(np.mean([s["n_updated_vertices"] for s in prof_stats]))
    incremental_order = n_upd <= tsf.INCREMENTAL_ORDER_MAX
    mean_st = {k: float(np.mean([s[k] for s in prof_stats])) for k in
               ("n_gradient_vertices", "d1_blocks_total", "n_points")}
    prof_total = float(sum(prof_ms))
    stage_rows = {}
    for name, (ms, calls) in prof.items():
        row = {"ms_per_step": round(ms / args.steps, 4), "share": round(ms / max(prof_total, 1e-9), 4),
               "launch_groups": calls}
        nbytes, units, what = stage_bytes(name, mean_st, nv, incremental_order)
        if nbytes is not None and calls > 0:
            avg = ms / calls
            row.update({"avg_ms": avg, "algorithmic_bytes": nbytes, "units": units, "unit_of_work": what,
                        "achieved_gbs": nbytes / (avg * 1e-3) / 1e9,
                        "frac": nbytes / (avg * 1e-3) / 1e9 / hbm})
        stage_rows[name] = row
    top = max(prof, key=lambda k: prof[k][0])
    modelled = [k for k in stage_rows if "achieved_gbs" in stage_rows[k]]
    dom = max(modelled, key=lambda k: prof[k][0])
    r = stage_rows[dom]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(SHAPE), "seed": SEED, "signal_threshold": TAU, "alpha": 0.5,
                   "fast_gradient_update": 1, "assignment": "exact",
                   "steps": "iterations 1..K from f_0 with the stop rule off",
                   "l2": "flushed (256 MiB write) before every timed step; working set several GB",
                   "parallelism": f"replicas x{world}", "input_generation_s": t_gen},
        "roofline": {"kernel": dom, "selection": "largest stage with a byte model", "bound": "hbm", "achieved": r["achieved_gbs"],
                     "peak": hbm, "unit": "GB/s", "frac": r["frac"], "traffic": None, "peak_kind": peak_kind,
                     "avg_launch_ms": r["avg_ms"], "algorithmic_bytes_per_launch": r["algorithmic_bytes"],
                     "units_per_launch": r["units"], "unit_of_work": r["unit_of_work"],
                     "bytes_per_unit": r["algorithmic_bytes"] / max(r["units"], 1.0),
                     "largest_stage": top, "largest_stage_share": stage_rows[top]["share"]},
        "stages": stage_rows,
        "profiled_ms_per_step": prof_total / args.steps,
        "solver": {"points_per_step": mean_st["n_points"],
                   "critical_per_step": np.mean([s["n_critical"] for s in stats], axis=0).tolist(),
                   "still_fraction": float(np.mean([s["n_still"] / max(s["n_points"], 1) for s in stats])),
                   "gradient_vertices_per_step": mean_st["n_gradient_vertices"],
                   "updated_vertices_per_step": n_upd,
                   "d1_columns": float(np.mean([s["d1_columns"] for s in stats])),
                   "d1_rounds_max_column": float(np.mean([s["d1_rounds_max"] for s in stats])),
                   "d1_reduce_rounds": float(np.mean([s["d1_reduce_rounds"] for s in stats])),
                   "d1_reduce_big_rounds": float(np.mean([s["d1_reduce_big_rounds"] for s in stats])),
                   "d1_reduce_big_cycle_share": float(np.sum([s["d1_reduce_big_cycles"] for s in stats]) /
                                                      max(np.sum([s["d1_reduce_cycles"] for s in stats]), 1)),
                   "step_ms": [round(x, 3) for x in step_ms]},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if not args.no_warm_start:
        line["warm_start"] = warm_start_block(tsf, torch, f0, stream)
    if not args.no_secondary:
        line["filament_128"] = secondary_filament_128(tsf, torch, stream, flush, 20)
    if not args.no_ablation:
        line["ablation"] = ablation_128(tsf, stream)
    if not args.no_loss:
        line["differentiable_loss"] = differentiable_loss()
    if not args.no_batch:
        line["batched_solve"] = batched_solve()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(f0)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end solve (short profiling runs)")
    ap.add_argument("--no-loss", action="store_true", help="skip the differentiable-loss measurement")
    ap.add_argument("--no-ablation", action="store_true", help="skip the Section 4.2/4.3 on/off solves")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched solve of 48 uneven fields")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 128^3 filament figures")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the learned warm-start comparison")
    ap.add_argument("--grid", type=int, default=256,
                    help="side of the evaluation field (256 = the headline; smaller grids for profiling)")
    args = ap.parse_args()
    if args.grid != 256:
        global SHAPE, WORKLOAD, METRIC
        SHAPE = (args.grid,) * 3
        WORKLOAD = f"warm_start_{args.grid}"
        METRIC = METRIC.replace("256^3", f"{args.grid}^3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
