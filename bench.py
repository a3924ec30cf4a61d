#!/usr/bin/env python
"""Benchmark: Cartesian FMM particles/s on one GB300 (and N replicas).

Default workload: 1,000,000 point dipoles uniform in the unit cube, field only,
p = 6, theta = 0.5, at most 128 particles per leaf, FP64.  One step is the
whole path: Morton keys, radix sort, cells, dual-tree lists, derivative
tables, P2M, M2M, M2L, L2L, L2P, P2P and the un-permute.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU FP64
oracle on the host cores instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_12351_gb300 import synth  # noqa: E402

METRIC = "FMM particles/sec at p=6 & rel err vs FP64 direct sum; served p50/p99 latency"
UNIT = "particles/s"
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2

# DRAM bytes (read + write) per particle of the dominant kernels, from full ncu captures of
# the 125k-dipole case (same leaf occupancy; the kernels' traffic grows with the particles):
# k_p2p_sym 7.546 MB + 0.183 MB, k_p2p32 11.210 MB + 0 MB per launch
# (profiles/fp64_pass_kernels_dipole_125k_p6.md, profiles/k_p2p32_k_m2l32_tile2_fp32_dipole_125k_p6.md)
TRAFFIC_PER_PARTICLE = {("fp64", 1): 7.7291e6 / 125_000, ("fp32", 1): 11.2097e6 / 125_000,
                        ("3xtf32", 1): 11.2097e6 / 125_000}


def flops_per_pair(s: int, want_phi: bool, want_field: bool) -> int:
    """Algorithmic FP64 flops of one P2P pair (rsqrt counted as one op)."""
    base = 3 + 5 + 1 + 2               # R, r^2, rsqrt, 1/r^2 and 1/r^3
    if s == 0:
        return base + (2 if want_phi else 0) + (7 if want_field else 0)
    if s == 1:
        return base + 5 + (2 if want_phi else 0) + (15 if want_field else 0)
    return base + 1 + 15 + 5 + (4 if want_phi else 0) + (19 if want_field else 0)


def m2p_flops(s: int, p: int, want_phi: bool, want_field: bool) -> int:
    """Algorithmic FP64 flops of one Barnes-Hut M2P (multipoles s <= |m| <= p): D_n(R)
    up to order p + 1 (p without the field) by the recurrence
    r^2 D_n = -(2 n_i - 1) R_i D_{n-e_i} - (n_i - 1)^2 D_{n-2e_i}
              - sum_{j != i} [2 n_j R_j D_{n-e_j} + n_j (n_j - 1) D_{n-2e_j}]
    (3 flops per term with R_j, 2 without, 1 for the 1/r^2 factor; r^2, 1/r^2 and
    1/r: 7), then 2 flops per multipole term for the potential and 6 for the field."""
    P = p + (1 if want_field else 0)
    fl = 7
    for k in range(1, P + 1):
        for nx in range(k, -1, -1):
            for ny in range(k - nx, -1, -1):
                n = (nx, ny, k - nx - ny)
                i = 0 if n[0] else (1 if n[1] else 2)
                fl += 3 + (2 if n[i] >= 2 else 0) + 1
                for j in range(3):
                    if j != i and n[j]:
                        fl += 3 + (2 if n[j] >= 2 else 0)
    nM = sum((k + 1) * (k + 2) // 2 for k in range(s, p + 1))
    return fl + nM * ((2 if want_phi else 0) + (6 if want_field else 0))


def m2l_macs_per_pair(s: int, p: int, want_phi: bool) -> int:
    """Terms of L_n += D_{n+m} M_m kept by |n| + |m| <= p + s (n from 0 or 1)."""
    tri = lambda k: (k + 1) * (k + 2) // 2
    lo = 0 if want_phi else 1
    return sum(tri(a) * sum(tri(b) for b in range(s, p + s - a + 1)) for a in range(lo, p + 1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(w: dict, n_sample, seed_shift: int = 0):
    """Time the oracle FMM on a bounded sample: the full tree and lists of the
    workload, then the FMM result for n_sample particles (upward pass on all
    cells, downward pass on their ancestor chains, L2P and P2P for them);
    n_sample None evaluates every particle.  For a batch workload the sample is
    whole systems (every 64th), each evaluated completely."""
    import oracle
    if "batch" in w:
        pos, S, off = synth.make_batch(w["batch"], w["nlo"], w["nhi"], w["s"], w["seed"] + seed_shift,
                                       w["dist"])
        t0 = time.perf_counter()
        k_tot = 0
        for k in range(0, w["batch"], 64):
            a, b = int(off[k]), int(off[k + 1])
            tree = oracle.Tree(pos[a:b], w["ncrit"])
            tree.lists(w["theta"])
            tree.fmm(S[a:b], w["s"], w["p"])
            k_tot += b - a
        return time.perf_counter() - t0, k_tot, oracle.num_threads()
    pos, S = synth.make_system(w["n"], w["s"], w["dist"], w["seed"] + seed_shift)
    tg = None if n_sample is None else synth.sample_indices(w["n"], n_sample, 17)
    k = w["n"] if tg is None else len(tg)
    t0 = time.perf_counter()
    tree = oracle.Tree(pos, w["ncrit"])
    tree.lists(w["theta"])
    t1 = time.perf_counter()
    tree.fmm(S, w["s"], w["p"], targets=tg)
    t2 = time.perf_counter()
    # tree and lists serve all N particles: charge the sample its share; the
    # upward pass and the ancestors' M2L are charged in full whatever the sample
    dt = (t2 - t1) + (t1 - t0) * k / w["n"]
    return dt, k, oracle.num_threads()


def fit_full_rate(counts, times, n: int):
    """Oracle particles/s on the whole n-particle workload from steps of sampled
    sizes: t(k) = fixed + per_particle * k by least squares (the fixed part is the
    upward pass and the sample's ancestor M2L, paid whatever k is), evaluated at
    k = n.  With one sample size only, the sampled rate."""
    counts, times = np.asarray(counts, float), np.asarray(times, float)
    if len(set(counts.tolist())) < 2:
        return float(counts.sum() / times.sum()), None, None
    per, fixed = np.polyfit(counts, times, 1)
    per, fixed = max(float(per), 1e-12), max(float(fixed), 0.0)
    return n / (fixed + per * n), fixed, per


def run_reference(args, w):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    # steps alternate between two sample sizes so that the fixed part of a step
    # (upward pass, ancestors' M2L) can be told from the per-particle part
    n_all = w.get("n") or 0
    sizes = [max(1, args.oracle_sample // 2), args.oracle_sample * 2]
    if "batch" not in w:
        sizes = [None if k >= n_all else k for k in sizes]      # None: every particle
    for i in range(args.warmup):
        oracle_sample(w, sizes[i % 2])
    times, counts = [], []
    cores, k = 1, 0
    for i in range(args.steps):
        dt, k, cores = oracle_sample(w, sizes[i % 2])
        times.append(dt)
        counts.append(k)
    ms = 1e3 * float(np.mean(times))
    if "batch" in w:
        value = float(np.sum(counts) / np.sum(times))
        sample = ("oracle FMM (C, FP64, OpenMP) on every 64th system of the batch, each evaluated "
                  "completely (%d particles per step); value = those particles / step time" % k)
    else:
        value, fixed, per = fit_full_rate(counts, times, w["n"])
        if fixed is None:
            sample = ("oracle FMM (C, FP64, OpenMP): tree, lists and the FMM result of all %d "
                      "particles per step; value = %d / step time" % (w["n"], w["n"]))
        else:
            sample = ("oracle FMM (C, FP64, OpenMP) on the full %d-particle tree and lists; FMM result "
                      "for %d or %d sampled particles per step, alternately (full upward pass, "
                      "downward pass on their ancestor chains, L2P + P2P); value = %d / (fixed + "
                      "per-particle x %d) fitted to the step times (fixed %.3f s, per particle %.3g s)"
                      % (w["n"], counts[0], counts[1], w["n"], w["n"], fixed, per))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args),
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": cores,
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(w, args):
    extra = {}
    if "batch" in w:
        extra = {"systems": w["batch"], "n_per_system": "log-uniform [%d, %d]" % (w["nlo"], w["nhi"]),
                 "form": "forest: one octree per system, every phase one launch for all systems"}
    return {**extra, "workload": args.workload, "n": w.get("n"), "source_order": w["s"], "p": w["p"],
            "theta": w["theta"], "max_leaf": w["ncrit"], "distribution": w["dist"],
            "outputs": "field" if not w.get("phi", False) else "potential+field",
            "precision": args.precision, "l2": "flushed (256 MB write) between timed steps",
            "replicas": args.gpus}


FP32_PEAK_TFLOPS = 80.5     # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz


def tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 GEMM rate of this machine's GPUs
    times the nominal TF32/bf16 ratio (1.1 / 2.25 PFLOP/s); TFLOP/s, source."""
    ratio = 1.1 / 2.25
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
        return bf16 * ratio, "measured bf16 %.1f TFLOP/s x nominal TF32/bf16 ratio 1.1/2.25" % bf16
    except (OSError, KeyError, ValueError):
        return 1900.0 * ratio, "fallback bf16 1900 TFLOP/s x nominal TF32/bf16 ratio 1.1/2.25"


def measure_form(args, w, precision, dev, world, rank, pos_h, S_h, pos_d, S_d, flush):
    """Time K whole steps of one precision form; returns a dict of results."""
    import torch
    from paper_2005_12351_gb300 import fmm
    s, p, theta, n = w["s"], w["p"], w["theta"], w["n"]
    want_phi, want_field = bool(w.get("phi", False)), True
    E_d = torch.empty((n, 3), dtype=torch.float64, device=dev)
    phi_d = torch.empty(n, dtype=torch.float64, device=dev) if want_phi else None
    E_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream(dev)
    tree = fmm.create_tree(device=dev.index, stream=stream, max_leaf=w["ncrit"],
                           precision=precision)
    tree.set_profiling(True)

    def step():
        if "batch" in w:
            tree.set_sources_batch(pos_d, S_d, w["offsets"], s)
        else:
            tree.set_sources(pos_d, S_d, s)
        tree.evaluate(p, theta, want_phi, want_field, potential=phi_d, field=E_d)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)

    # ---- device-timed steps (inputs resident in HBM)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phases = []
    clk = ClockSampler(dev.index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clk.start()
    time.sleep(0.3)
    launches0 = tree.launch_count()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        phases.append(tree.phase_times())
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    launches = tree.launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(float(np.mean(step_ms)), world, dev)
    value = n * world / (ms / 1e3)

    # ---- end to end through the public API with host buffers
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pos_d.copy_(pos_h, non_blocking=True)
        S_d.copy_(S_h, non_blocking=True)
        step()
        E_h.copy_(E_d, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e = max_over_ranks(float(np.mean(e2e_ms)), world, dev)
    h2d = pos_h.numel() * 8 + S_h.numel() * 8
    d2h = E_h.numel() * 8

    # ---- accuracy against the FP64 direct sum (GPU), sampled targets
    if "batch" in w:
        # a sample of whole systems, each summed directly against itself
        off = w["offsets"]
        ks = synth.sample_indices(len(off) - 1, 64, 23)
        refs, outs = [], []
        for k in ks:
            a, bb = int(off[k]), int(off[k + 1])
            _, Er = fmm.direct_sum(pos_d[a:bb].contiguous(), S_d[a:bb].contiguous(), s,
                                   want_potential=False)
            refs.append(Er)
            outs.append(E_d[a:bb])
        E_ref, Ef = torch.cat(refs), torch.cat(outs)
        tg = np.arange(E_ref.shape[0])
    else:
        tg = synth.sample_indices(n, args.err_samples, 23)
        tg_d = torch.from_numpy(tg.astype(np.int32)).to(dev)
        _, E_ref = fmm.direct_sum(pos_d, S_d, s, targets=tg_d, want_potential=False)
        Ef = E_d[tg_d.long()]
    num = ((Ef - E_ref) ** 2).sum().item()
    den = (E_ref ** 2).sum().item()
    per = (torch.linalg.norm(Ef - E_ref, dim=1) / torch.linalg.norm(E_ref, dim=1)).cpu().numpy()
    rel_err = {"field_rel_rms": math.sqrt(num / den), "field_rel_median": float(np.median(per)),
               "field_rel_p99": float(np.quantile(per, 0.99)), "field_rel_max": float(per.max()),
               "targets": int(len(tg)), "reference": "GPU FP64 direct sum (parity-tested vs oracle)"}

    # ---- roofline of the dominant kernel (per-phase CUDA events on this stream)
    info = tree.info()
    ph = {k: float(np.mean([q[k] for q in phases])) for k in phases[0]}
    pair_flops = flops_per_pair(s, want_phi, want_field) * info["n_p2p_interactions"]
    m2l_flops = 2 * m2l_macs_per_pair(s, p, want_phi) * info["n_m2l"]
    if precision == "fp64":
        peak, src = args.fp64_peak_tflops, args.fp64_peak_source
    else:
        peak, src = FP32_PEAK_TFLOPS, "152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz"
    cand = {"p2p": pair_flops, "m2l": m2l_flops}
    dom = max(cand, key=lambda k: ph[k])
    achieved = cand[dom] / (ph[dom] / 1e3) / 1e12
    tpp = TRAFFIC_PER_PARTICLE.get((precision, s)) if dom == "p2p" and "batch" not in w else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": tpp * n if tpp is not None else None,
                "traffic_source": ("ncu dram bytes of the 125k-dipole capture, scaled by particles"
                                   if tpp is not None else None),
                "algorithmic_flops": cand[dom], "peak_source": src}
    if precision == "3xtf32" and info["tc_rows"] > 0:
        # the M2L on the tensor cores: 3 TF32 products per FP32 multiply-add of the method
        tpk, tsrc = tf32_peak()
        t_ach = 3 * m2l_flops / (ph["m2l"] / 1e3) / 1e12
        roofline_m2l = {"bound": "tensor", "kernel": "m2l (k_m2l_tc + plan, 3xTF32)", "achieved": t_ach,
                        "peak": tpk, "unit": "TFLOP/s", "frac": t_ach / tpk, "traffic": None,
                        "algorithmic_flops": 3 * m2l_flops, "peak_source": tsrc,
                        "tile_fill": info["n_m2l"] / (128.0 * info["tc_rows"]),
                        "tc_rows": info["tc_rows"], "tc_chunks": info["tc_chunks"]}
    else:
        roofline_m2l = None
    res = {"value": value, "ms_per_step": ms, "rel_err": rel_err, "roofline_m2l": roofline_m2l,
           "e2e": {"value": n * world / (e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": e2e},
           "roofline": roofline, "phase_ms": ph, "clocks": clocks, "gpu_launches": launches,
           "wall_s_timed": t_wall,
           "tree": {k: info[k] for k in ("ncells", "nleaves", "nlevels", "n_m2l", "n_p2p",
                                         "n_p2p_interactions", "n_doffsets")}}
    tree.destroy()
    return res


def measure_graph(args, w, precision, dev, world, pos_d, S_h, S_d, flush):
    """Repeated evaluation of one geometry: autotune once (untimed), then K steps of
    (moment update + the evaluate replayed as one CUDA graph launch)."""
    import torch
    from paper_2005_12351_gb300 import fmm
    s, p, theta, n = w["s"], w["p"], w["theta"], w["n"]
    want_phi = bool(w.get("phi", False))
    stream = torch.cuda.current_stream(dev)
    tree = fmm.create_tree(device=dev.index, stream=stream, max_leaf=w["ncrit"], precision=precision)
    if "batch" in w:
        tree.set_sources_batch(pos_d, S_d, w["offsets"], s)
    else:
        tree.set_sources(pos_d, S_d, s)
    tuning = tree.autotune(p, theta, want_phi, True, reps=2)
    E_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    step = lambda: (tree.update_moments(S_d), tree.evaluate_graph(p, theta, want_phi, True))
    for _ in range(max(args.warmup, 1)):
        _, E_d = step()[1]
    torch.cuda.synchronize(dev)
    launches0 = tree.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    launches = tree.launch_count() - launches0
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world, dev)
    e2e = []
    for k in range(args.steps):
        flush.fill_(k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S_d.copy_(S_h, non_blocking=True)
        _, E_d = step()[1]
        E_h.copy_(E_d, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e.append(a.elapsed_time(b))
    e2e_ms = max_over_ranks(float(np.mean(e2e)), world, dev)
    tree.destroy()
    return {"precision": precision, "value": n * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "step": "fmm_update_moments + fmm_evaluate_graph (tree and lists fixed; one graph launch)",
            "gpu_launches": launches,
            "e2e": {"value": n * world / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": S_h.numel() * 8, "d2h_bytes_per_step": E_h.numel() * 8},
            "tuning": tuning}


def measure_bh(args, w, dev, world, pos_d, S_d, flush):
    """Multipolar Barnes-Hut on the same workload: a step = tree build + fmm_evaluate_bh
    at order p, opening angle theta_BH (the paper: theta_FMM ~ 2 theta_BH for a similar
    error).  The walk kernel is timed alone for its roofline."""
    import torch
    from paper_2005_12351_gb300 import fmm
    s, p, n = w["s"], w["p"], w["n"]
    theta = args.bh_theta if args.bh_theta is not None else w["theta"] / 2
    stream = torch.cuda.current_stream(dev)
    tree = fmm.create_tree(device=dev.index, stream=stream, max_leaf=w["ncrit"])
    E_d = torch.empty((n, 3), dtype=torch.float64, device=dev)
    walk = []

    def step():
        tree.set_sources(pos_d, S_d, s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tree.evaluate_bh(p, theta, False, True, field=E_d)
        b.record(stream)
        walk.append((a, b))

    step()
    torch.cuda.synchronize(dev)
    walk.clear()
    steps = max(1, min(args.steps, 2))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world, dev)
    walk_ms = float(np.mean([a.elapsed_time(b) for a, b in walk]))
    info = tree.info()
    tg = synth.sample_indices(n, args.err_samples, 23)
    tg_d = torch.from_numpy(tg.astype(np.int32)).to(dev)
    _, E_ref = fmm.direct_sum(pos_d, S_d, s, targets=tg_d, want_potential=False)
    Ef = E_d[tg_d.long()]
    err = math.sqrt(((Ef - E_ref) ** 2).sum().item() / (E_ref ** 2).sum().item())
    flops = (info["bh_m2p"] * m2p_flops(s, p, False, True)
             + info["bh_p2p"] * flops_per_pair(s, False, True))
    achieved = flops / (walk_ms / 1e3) / 1e12
    tree.destroy()
    return {"theta_bh": theta, "p": p, "value": n * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "step": "tree build + fmm_evaluate_bh (field)", "walk_ms": walk_ms,
            "field_rel_rms": err, "targets": int(len(tg)),
            "m2p": info["bh_m2p"], "p2p_pairs": info["bh_p2p"],
            "roofline": {"bound": "alu", "kernel": "k_bh", "achieved": achieved,
                         "peak": args.fp64_peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / args.fp64_peak_tflops, "traffic": None,
                         "algorithmic_flops": flops,
                         "per_m2p_flops": m2p_flops(s, p, False, True),
                         "peak_source": args.fp64_peak_source}}


def measure_mixed_orders(args, w, dev, world, flush):
    """Mixed source orders on the headline geometry: every particle carries a charge and
    a dipole (orders 0..1; the expansion starts at order 0, so multipoles run to p).  A
    step = tree build + evaluate, as the main line; FP64, the handle's default P2P (the
    symmetric kernel, each shell's reverse term with its own parity)."""
    import torch
    from paper_2005_12351_gb300 import fmm
    n, p, theta = w["n"], w["p"], w["theta"]
    lo, hi = 0, 1
    pos_np, S_np = synth.make_system_mixed(n, lo, hi, w["dist"], w["seed"] + 7)
    pos_d = torch.from_numpy(pos_np).to(dev)
    S_d = torch.from_numpy(S_np).to(dev)
    stream = torch.cuda.current_stream(dev)
    tree = fmm.create_tree(device=dev.index, stream=stream, max_leaf=w["ncrit"])
    tree.set_profiling(True)
    E_d = torch.empty((n, 3), dtype=torch.float64, device=dev)

    def step():
        tree.set_sources_mixed(pos_d, S_d, lo, hi)
        tree.evaluate(p, theta, False, True, field=E_d)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 5))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    phases = []
    for k in range(steps):
        flush.fill_(k)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        phases.append(tree.phase_times())
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world, dev)
    ph = {k: float(np.mean([q[k] for q in phases])) for k in phases[0]}
    info = tree.info()
    tg = synth.sample_indices(n, args.err_samples, 23)
    tg_d = torch.from_numpy(tg.astype(np.int32)).to(dev)
    _, E_ref = fmm.direct_sum(pos_d, S_d, lo, targets=tg_d, want_potential=False, source_order_hi=hi)
    Ef = E_d[tg_d.long()]
    err = math.sqrt(((Ef - E_ref) ** 2).sum().item() / (E_ref ** 2).sum().item())
    pair = flops_per_pair(0, False, True) + flops_per_pair(1, False, True)
    flops = pair * info["n_p2p_interactions"]
    achieved = flops / (ph["p2p"] / 1e3) / 1e12
    tree.destroy()
    return {"sources": "charge + dipole per particle (orders 0..1)", "p": p, "theta": theta,
            "value": n * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "field_rel_rms": err,
            "targets": int(len(tg)), "phase_ms": ph, "p2p_kernel": "symmetric",
            "roofline": {"bound": "alu", "kernel": "p2p", "achieved": achieved,
                         "peak": args.fp64_peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / args.fp64_peak_tflops, "traffic": None,
                         "algorithmic_flops": flops, "peak_source": args.fp64_peak_source}}


def measure_config(args, wname: str, precisions, dev, flush):
    """One of the other benchmark configurations as a sub-object of the line:
    per precision form, particles/s of the whole step (tree, lists, evaluate;
    inputs resident, one untimed warm-up step, min(steps, 3) timed) and the error
    of its result against the FP64 direct sum -- 4,096 sampled particles of a
    single system, or 64 sampled whole systems of a batch -- with the ratio to the
    FP64 form's error on the same targets."""
    import torch
    from paper_2005_12351_gb300 import fmm
    w = dict(synth.WORKLOADS[wname])
    s, p, theta = w["s"], w["p"], w["theta"]
    want_phi = True
    if "batch" in w:
        pos_np, S_np, off = synth.make_batch(w["batch"], w["nlo"], w["nhi"], s, w["seed"], w["dist"])
        offsets = [int(x) for x in off]
    else:
        pos_np, S_np = synth.make_system(w["n"], s, w["dist"], w["seed"])
        offsets = None
    n = len(pos_np)
    pos_d = torch.from_numpy(pos_np).to(dev)
    S_d = torch.from_numpy(S_np).to(dev)
    stream = torch.cuda.current_stream(dev)
    # reference: the GPU FP64 direct sum at the sampled targets
    if offsets is not None:
        ks = synth.sample_indices(len(offsets) - 1, 64, 23)
        idx, refs = [], []
        for k in ks:
            a, b = offsets[k], offsets[k + 1]
            ph, Er = fmm.direct_sum(pos_d[a:b].contiguous(), S_d[a:b].contiguous(), s)
            refs.append((ph, Er))
            idx.append(torch.arange(a, b, device=dev))
        tg_d = torch.cat(idx)
        phi_ref = torch.cat([r[0] for r in refs])
        E_ref = torch.cat([r[1] for r in refs])
        sample = "64 sampled whole systems (%d particles)" % tg_d.numel()
    else:
        tg = synth.sample_indices(n, args.err_samples, 23)
        tg_d = torch.from_numpy(tg.astype(np.int64)).to(dev)
        phi_ref, E_ref = fmm.direct_sum(pos_d, S_d, s, targets=tg_d.int())
        sample = "%d sampled particles" % tg_d.numel()
    out = {"workload": wname, "n": n, "source_order": s, "p": p, "theta": theta,
           "max_leaf": w["ncrit"], "distribution": w["dist"], "outputs": "potential+field",
           "error_targets": sample, "reference": "GPU FP64 direct sum (parity-tested vs oracle)"}
    if offsets is not None:
        out["systems"] = len(offsets) - 1
    steps = max(1, min(args.steps, 3))
    err64 = None
    for prec in precisions:
        tree = fmm.create_tree(device=dev.index, stream=stream, max_leaf=w["ncrit"], precision=prec)
        phi_d = torch.empty(n, dtype=torch.float64, device=dev)
        E_d = torch.empty((n, 3), dtype=torch.float64, device=dev)

        def step():
            if offsets is not None:
                tree.set_sources_batch(pos_d, S_d, offsets, s)
            else:
                tree.set_sources(pos_d, S_d, s)
            tree.evaluate(p, theta, want_phi, True, potential=phi_d, field=E_d)

        step()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        launches0 = tree.launch_count()
        for k in range(steps):
            flush.fill_(k)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        E_s, phi_s = E_d[tg_d], phi_d[tg_d]
        per = (torch.linalg.norm(E_s - E_ref, dim=1) / torch.linalg.norm(E_ref, dim=1)).cpu().numpy()
        err = {"field_rel_rms": math.sqrt(((E_s - E_ref) ** 2).sum().item() / (E_ref ** 2).sum().item()),
               "potential_rel_rms": math.sqrt(((phi_s - phi_ref) ** 2).sum().item()
                                              / (phi_ref ** 2).sum().item()),
               "field_rel_median": float(np.median(per)), "field_rel_p99": float(np.quantile(per, 0.99)),
               "field_rel_max": float(per.max())}
        if prec == "fp64":
            err64 = err
        res = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
               "gpu_launches_per_step": (tree.launch_count() - launches0) / steps, "rel_err": err}
        if err64 is not None and prec != "fp64":
            res["error_ratio_vs_fp64"] = {"field": err["field_rel_rms"] / err64["field_rel_rms"],
                                          "potential": err["potential_rel_rms"] / err64["potential_rel_rms"]}
            res["within_1p1_of_fp64"] = bool(max(res["error_ratio_vs_fp64"].values()) <= 1.1)
        if prec == "3xtf32":
            info = tree.info()
            res["tc_rows"] = info["tc_rows"]
        out[prec] = res
        tree.destroy()
    return out


class RequestPools:
    """Particle pools the serving requests are cut from: per distribution
    (uniform cube, Plummer) 2,000,000 positions, and per source order that many
    moments.  A request of size N takes N consecutive particles at a random
    offset -- an i.i.d. sample of its distribution -- so thousands of requests
    need no more host memory than the pools."""
    NMAX = 2_000_000

    def __init__(self, seed: int):
        self.pos = {d: synth.make_system(self.NMAX, 0, d, seed + k)[0]
                    for k, d in enumerate(("uniform", "plummer"))}
        self.mom = {s: synth.sources(self.NMAX, seed + 10 + s, s) for s in (0, 1, 2)}

    def cut(self, n: int, s: int, dist: str, u: float):
        a = int(u * (self.NMAX - n + 1))
        return self.pos[dist][a:a + n], self.mom[s][a:a + n]


def serving_stream(count: int, seed: int, pools: RequestPools):
    """Requests drawn like the serving workload: N log-uniform in [1e3, 2e6],
    source order uniform over {0, 1, 2}, p uniform over {4..10}, uniform or
    Plummer positions 50/50, theta 0.5, n_crit 128."""
    sizes = synth.log_uniform_int(count, 1000, 2_000_000, seed)
    u = synth.uniform01(seed, 17, 4 * count).reshape(count, 4)
    reqs = []
    for k in range(count):
        s = int(u[k, 0] * 3)
        p = 4 + int(u[k, 1] * 7)
        dist = "plummer" if u[k, 2] < 0.5 else "uniform"
        pos, mom = pools.cut(int(sizes[k]), s, dist, float(u[k, 3]))
        reqs.append(dict(positions=pos, moments=mom, source_order=s, p=p, theta=0.5,
                         max_leaf=128, want_potential=False, want_field=True))
    return reqs


def _serve(sv, reqs, arrivals, keep):
    """Submit reqs at the given arrival offsets (seconds; None = all at once),
    reaping finished tickets as it goes so that only the requests in flight hold
    outputs.  Returns (latencies ms, first submit, last end, particles done,
    failures, kept results {index: field})."""
    from paper_2005_12351_gb300 import fmm
    lat, out, failures = [], {}, []
    live = {}
    t_first, t_last, done_particles = None, None, 0
    start = time.perf_counter()

    def reap(block):
        nonlocal t_first, t_last, done_particles
        for k in list(live):
            if not block and not sv.done(live[k]):
                continue
            r = reqs[k]
            try:
                _, E, info = sv.wait(live.pop(k))
            except fmm.FMMError as e:
                failures.append({"n": len(r["positions"]), "s": r["source_order"], "p": r["p"],
                                 "error": str(e)[:200]})
                continue
            lat.append(1e3 * (info["end_s"] - info["submit_s"]))
            t_first = info["submit_s"] if t_first is None else min(t_first, info["submit_s"])
            t_last = info["end_s"] if t_last is None else max(t_last, info["end_s"])
            done_particles += len(r["positions"])
            if k in keep:
                out[k] = E

    for k, r in enumerate(reqs):
        if arrivals is not None:
            while True:
                delay = start + arrivals[k] - time.perf_counter()
                if delay <= 0:
                    break
                reap(False)
                time.sleep(min(delay, 0.002))
        live[k] = sv.submit(**r)
        reap(False)
    reap(True)
    return lat, t_first, t_last, done_particles, failures, out


def run_serving(args, dev):
    """Continuous batching on the device: calibrate the server's capacity closed
    loop, then replay Poisson arrivals at 0.5, 0.8 and 0.95 of it and report
    latency percentiles per load; a sample of served results is checked against
    the FP64 direct sum (and the FP64 form's error on the same requests)."""
    import torch
    from paper_2005_12351_gb300 import fmm
    pools = RequestPools(20260014)
    reqs = serving_stream(args.serving_requests, 20260004, pools)
    total = sum(len(r["positions"]) for r in reqs)
    budget = 120 << 30
    sv = fmm.Server(device=dev.index, slots=args.serving_slots, precision=args.serving_precision,
                    mem_budget_bytes=budget)
    for t in [sv.submit(**r) for r in reqs[:args.serving_slots]]:      # warm the slots
        sv.wait(t)
    t0 = time.perf_counter()
    _, _, _, done0, fail0, _ = _serve(sv, reqs, None, set())
    capacity = done0 / (time.perf_counter() - t0)
    keep = set(range(0, len(reqs), max(1, len(reqs) // 16)))
    loads = []
    kept = {}
    for li, load in enumerate((0.5, 0.8, 0.95)):
        rate = load * capacity / (total / len(reqs))                      # requests per second
        gaps = -np.log(1.0 - synth.uniform01(20260005 + li, 1, len(reqs))) / rate
        lat, t_first, t_last, done, failures, out = _serve(sv, reqs, np.cumsum(gaps),
                                                            keep if li == 1 else set())
        kept.update(out)
        loads.append({"offered_load": load, "offered_particles_per_s": load * capacity,
                      "particles_per_s": done / (t_last - t_first) if done else 0.0,
                      "p50_latency_ms": float(np.percentile(lat, 50)) if lat else None,
                      "p99_latency_ms": float(np.percentile(lat, 99)) if lat else None,
                      "max_latency_ms": float(np.max(lat)) if lat else None,
                      "completed": len(lat), "failed": len(failures), "failures": failures[:5]})
    st = sv.stats()
    sv.close()
    # accuracy of served results: field error at 256 sampled targets of each kept
    # request against the GPU FP64 direct sum, beside the FP64 form's error
    acc = []
    for k in sorted(kept):
        r = reqs[k]
        n = len(r["positions"])
        P = torch.from_numpy(np.ascontiguousarray(r["positions"])).to(dev)
        Sd = torch.from_numpy(np.ascontiguousarray(r["moments"])).to(dev)
        tg = synth.sample_indices(n, min(n, 256), 41 + k)
        tg_d = torch.from_numpy(tg.astype(np.int32)).to(dev)
        _, E_ref = fmm.direct_sum(P, Sd, r["source_order"], targets=tg_d, want_potential=False)
        E_ref = E_ref.cpu().numpy()
        t64 = fmm.create_tree(device=dev.index, max_leaf=r["max_leaf"])
        t64.set_sources(P, Sd, r["source_order"])
        _, E64 = t64.evaluate(r["p"], r["theta"], False, True)
        E64 = E64.cpu().numpy()[tg]
        t64.destroy()
        e = float(np.sqrt(((kept[k][tg] - E_ref) ** 2).sum() / (E_ref ** 2).sum()))
        e64 = float(np.sqrt(((E64 - E_ref) ** 2).sum() / (E_ref ** 2).sum()))
        acc.append({"n": n, "s": r["source_order"], "p": r["p"], "field_rel_rms": e,
                    "fp64_field_rel_rms": e64, "ratio": e / e64 if e64 > 0 else None})
    ratios = [a["ratio"] for a in acc if a["ratio"] is not None]
    return {"requests": len(reqs), "particles": total, "slots": args.serving_slots,
            "precision": args.serving_precision, "mem_budget_gb": 120,
            "capacity_particles_per_s": capacity, "capacity_failed": len(fail0),
            "loads": loads, "peak_device_gb": st["peak_device_bytes"] / 2 ** 30,
            "accuracy": {"requests_checked": len(acc), "targets_per_request": 256,
                         "reference": "GPU FP64 direct sum (parity-tested vs oracle)",
                         "max_ratio_vs_fp64": max(ratios) if ratios else None,
                         "median_ratio_vs_fp64": float(np.median(ratios)) if ratios else None,
                         "per_request": acc},
            "mix": "N log-uniform [1e3, 2e6], s in {0,1,2}, p in {4..10}, uniform/Plummer 50/50, "
                   "each request N consecutive particles of a 2M-particle pool at a random offset"}


def run_ours(args, w):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if "batch" in w:
        pos_np, S_np, off = synth.make_batch(w["batch"], w["nlo"], w["nhi"], w["s"],
                                             w["seed"] + 1000 * rank, w["dist"])
        w["offsets"] = [int(x) for x in off]
        w["n"] = n = int(off[-1])
    else:
        n = w["n"]
        pos_np, S_np = synth.make_system(n, w["s"], w["dist"], w["seed"] + 1000 * rank)
    pos_h = torch.from_numpy(pos_np).pin_memory()
    S_h = torch.from_numpy(S_np).pin_memory()
    pos_d, S_d = pos_h.to(dev), S_h.to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    main = measure_form(args, w, args.precision, dev, world, rank, pos_h, S_h, pos_d, S_d, flush)
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic (seeded; %s)" % w["dist"], "config": config_of(w, args)}
    line.update({k: main[k] for k in ("rel_err", "e2e", "roofline", "phase_ms", "clocks",
                                      "gpu_launches", "wall_s_timed", "tree")})
    if args.precision == "fp64" and not args.no_mixed:
        mx = measure_form(args, w, "fp32", dev, world, rank, pos_h, S_h, pos_d, S_d, flush)
        line["mixed_fp32"] = {k: mx[k] for k in ("value", "ms_per_step", "rel_err", "e2e",
                                                 "roofline", "phase_ms", "gpu_launches")}
        line["mixed_fp32"]["error_ratio_vs_fp64"] = (mx["rel_err"]["field_rel_rms"]
                                                     / main["rel_err"]["field_rel_rms"])
        m3 = measure_form(args, w, "3xtf32", dev, world, rank, pos_h, S_h, pos_d, S_d, flush)
        line["mixed_3xtf32"] = {k: m3[k] for k in ("value", "ms_per_step", "rel_err", "e2e",
                                                   "roofline", "roofline_m2l", "phase_ms",
                                                   "gpu_launches")}
        line["mixed_3xtf32"]["error_ratio_vs_fp64"] = (m3["rel_err"]["field_rel_rms"]
                                                       / main["rel_err"]["field_rel_rms"])
    if args.precision == "fp64" and not args.no_bh and "batch" not in w:
        line["bh"] = measure_bh(args, w, dev, world, pos_d, S_d, flush)
    if args.precision == "fp64" and not args.no_mixed_orders and "batch" not in w:
        line["mixed_orders"] = measure_mixed_orders(args, w, dev, world, flush)
    if not args.no_graph:
        line["graph"] = measure_graph(args, w, args.graph_precision or args.precision, dev, world,
                                      pos_d, S_h, S_d, flush)
    if world == 1 and not args.no_configs and "batch" not in w:
        forms = ("fp64", "fp32", "3xtf32")
        line["plummer_4m_p8"] = measure_config(args, "dipole_plummer_4m_p8", forms, dev, flush)
        line["quadrupole_batch_4096_p5"] = measure_config(args, "quadrupole_batch_4096_p5", forms,
                                                          dev, flush)
    if world == 1 and args.serving_requests > 0 and "batch" not in w:
        line["serving"] = run_serving(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        full = args.cpu_baseline_sample <= 0 or "batch" in w
        dt, k, cores = oracle_sample(w, None if full else args.cpu_baseline_sample)
        line["cpu_baseline"] = {
            "value": k / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": ("oracle FMM (C, FP64, OpenMP): tree, lists and the FMM result of every one of "
                       "the %d particles, one run, %.1f s" % (k, dt)) if full else
                      ("oracle FMM on the full tree and lists, FMM result for %d sampled particles "
                       "(full upward pass, ancestor-chain downward pass, L2P + P2P); %.1f s" % (k, dt))}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="dipole_1m_p6", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--err-samples", type=int, default=4096)
    ap.add_argument("--oracle-sample", type=int, default=65536,
                    help="sampled particles per step of --impl reference")
    ap.add_argument("--cpu-baseline-sample", type=int, default=0,
                    help="sampled particles of the main line's cpu_baseline; 0 (default) evaluates "
                         "the whole workload once (about 20 s on 16 cores at 1M particles)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 4M Plummer p=8 and 4,096-system quadrupole batch sub-objects")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "fp32", "3xtf32"], default="fp64")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the extra FP32 and 3xTF32 form measurements in the same run")
    ap.add_argument("--no-graph", action="store_true",
                    help="skip the repeated-geometry measurement (autotune + graph replay)")
    ap.add_argument("--graph-precision", choices=["fp64", "fp32", "3xtf32"], default=None,
                    help="form of the graph measurement (default: --precision)")
    ap.add_argument("--no-bh", action="store_true",
                    help="skip the Barnes-Hut line (FP64, same workload, theta_BH = theta / 2)")
    ap.add_argument("--bh-theta", type=float, default=None)
    ap.add_argument("--no-mixed-orders", action="store_true",
                    help="skip the charge + dipole (orders 0..1) line")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests in the serving measurement (0 = skip)")
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-precision", choices=["fp64", "fp32", "3xtf32"], default="3xtf32")
    ap.add_argument("--fp64-peak-tflops", type=float, default=1.259)
    ap.add_argument("--fp64-peak-source", default="152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz "
                    "(nominal 1.25 TFLOP/s FP64 of the part)")
    args = ap.parse_args(argv)
    w = dict(synth.WORKLOADS[args.workload])
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
