#!/usr/bin/env python
"""Benchmark: chi(i tau) time per tau point and useful TFLOP/s on GB300.

Workload: the 298-atom armchair-ribbon-shaped chain (200 C + 98 H, 3090
primary / 7176 RI functions, 20 tau points in [0.01, 50] a.u., filter
threshold 1e-9), seeded synthetic inputs (synth).  One step = chi(i tau_j) for
one tau point through the C ABI (steps cycle through the tau grid); inputs
(3c tensor 11 GB, orbitals) are resident in HBM before the timed region.

value  = useful TFLOP/s of the mixed-precision form (default FP16x3: two scaled
         binary16 slices, 3 tensor-core products; flops of the surviving
         atom-block products of Eq. 3's steps A, B, C; split products,
         padding and skipped work not counted), whole job.
Also reported: ms per tau point; the other forms (FP64, FP32, BF16x3,
BF16x6) on one tau point with their sampled errors; the rooflines of the two
tensor-core kernels (steps A/B and step C) against the measured tensor peak,
and of the CUDA-core forms against the FFMA/DFMA throughput measured here
(--peaks prints those alone); the error of the timed form against the FP64
block oracle at every tau point; the learned screen at the same threshold
(time, skipped tasks, error); an end-to-end figure through host buffers; and
the CPU oracle on a bounded sample, whose useful flops are the oracle's own
count (tests/golden/flops_ribbon298.json).

Multi-GPU: tau points are independent; rank r takes steps r, r + N, ... of
the tau cycle (no collective on the data path): weak scaling.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ribbon300"
N_PRODUCTS = {"fp32": 1, "bf16x3": 3, "bf16x6": 6, "fp16x3": 3, "fp64": 1}
SPLIT_FORMS = ("bf16x3", "bf16x6", "fp16x3")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2] if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def tau_index(i: int, world: int, rank: int, n_tau: int) -> int:
    """tau point of step i on rank `rank`: the ranks take interleaved points of
    the tau cycle (independent problems, no exchange)."""
    return (i * world + rank) % n_tau


def job_totals(t_local: float, flops_local: float, device) -> tuple[float, float]:
    """Whole-job time (max over ranks) and useful flops (sum over ranks); the
    local values when no process group of more than one rank is running."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_local, flops_local
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ff = torch.tensor([flops_local], dtype=torch.float64, device=device)
    dist.all_reduce(ff, op=dist.ReduceOp.SUM)
    return tt.item(), ff.item()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_sample(case, steps: int, useful_flops_per_tau: float):
    """Time the CPU oracle (as it stands) on a bounded sample of one tau point:
    M slices and N slices of single RI atoms and single atom-block
    contractions; scale to one full tau point by the counts of a full
    evaluation (n_atoms M slices, n_atoms N slices, n_atoms(n_atoms+1)/2
    blocks)."""
    from oracle import chi as oc

    bo = oc.BlockOracle(case)
    n_at = case.system.n_atoms
    j = len(case.tau) // 2
    bo.greens(j)
    t_m, t_n, t_b = [], [], []
    blocks = {}
    for i in range(max(1, steps)):
        p = (n_at // 2 + 37 * i) % n_at
        t0 = time.perf_counter()
        m = bo.m_slice(j, p)
        t1 = time.perf_counter()
        n = bo.n_slice(j, p)
        t2 = time.perf_counter()
        cache = {("m", j, p): m, ("n", j, p): n}
        blocks[p] = bo.block(j, p, p, cache)
        t3 = time.perf_counter()
        t_m.append(t1 - t0)
        t_n.append(t2 - t1)
        t_b.append(t3 - t2)
    tm = sum(t_m) / len(t_m)
    tn = sum(t_n) / len(t_n)
    tb = sum(t_b) / len(t_b)
    t_tau = n_at * (tm + tn) + n_at * (n_at + 1) / 2 * tb
    return {
        "value": useful_flops_per_tau / t_tau / 1e12,
        "unit": "TFLOP/s",
        "cores": os.cpu_count(),
        "kind": "oracle",
        "ms_per_tau_estimate": t_tau * 1e3,
        "sample": (f"tau index {j}: {len(t_m)} RI-atom M slice(s), N slice(s) and diagonal "
                   f"block contraction(s) of the numpy FP64 block oracle "
                   f"(mean {tm:.2f} s, {tn:.2f} s, {tb:.3f} s), scaled to one tau point by "
                   f"{n_at} M + {n_at} N slices and {n_at * (n_at + 1) // 2} blocks"),
        "sample_seconds": sum(t_m) + sum(t_n) + sum(t_b),
        "tau_index": j,
        "blocks": blocks,
    }


def run_reference(args):
    """The CPU FP64 oracle as the reference arm (rank 0 only)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    from synth import make_case

    case = make_case(WORKLOAD)
    flops_tau = _useful_flops_oracle_side(case, len(case.tau) // 2)
    for _ in range(args.warmup):
        cpu_oracle_sample(case, 1, flops_tau)
    t0 = time.perf_counter()
    res = cpu_oracle_sample(case, args.steps, flops_tau)
    wall = time.perf_counter() - t0
    line = {
        "impl": "reference",
        "metric": "chi(i tau) useful TFLOP/s (time per tau point), mixed vs FP64 at <=1e-6 rel err",
        "value": res["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(1, args.steps),
        "ms_per_tau": res["ms_per_tau_estimate"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "armchair-ribbon-298 (3090 AO / 7176 RI, 20 tau, thr 1e-9)",
                   "form": "CPU FP64 oracle (numpy)"},
        "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": res["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _useful_flops_oracle_side(case, tau_index: int) -> float:
    """Useful flops of one tau point as the oracle counts them from its own
    filtered blocks (oracle.chi.useful_flops_blocks; the flops of the atom-block
    products whose operands survive the filter), read from the count that
    tests/golden/make_flops_ribbon298.py wrote for the benchmark workload."""
    path = os.path.join(ROOT, "tests", "golden", "flops_ribbon298.json")
    with open(path) as f:
        rec = json.load(f)["per_tau"][str(tau_index)]
    return rec["flops_a"] + rec["flops_b"] + rec["flops_c"]


def alu_peaks():
    """Measured FFMA and DFMA throughput of this GPU (libgwpeaks.so), TFLOP/s."""
    import ctypes

    from paper_2104_09857_gb300 import build as b

    lib = ctypes.CDLL(b.build_peaks())
    lib.gw_fma_peak.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]
    out = {}
    for name, fp64, iters in (("fp32", 0, 20000), ("fp64", 1, 400)):
        tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
        rc = lib.gw_fma_peak(fp64, iters, ctypes.byref(tf), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError(f"gw_fma_peak({name}) failed: {rc}")
        out[name] = {"tflops": tf.value, "ms": ms.value, "iters": iters}
    out["how"] = ("FMA chains, 8 independent per thread, 8 CTAs x 256 threads per SM, best of "
                  "3 launches timed with CUDA events (paper_2104_09857_gb300/peaks/fma_peaks.cu)")
    return out


def _roof(flops, seconds, prec, peaks, peak_src, kernel, traffic, alu=None):
    """Roofline object of one kernel: achieved = useful flops / its device
    time over the timed region (the same per average launch)."""
    achieved = flops / seconds / 1e12 if seconds > 0 else None
    if prec in SPLIT_FORMS:
        # binary16 and bf16 share the dense tensor rate (kind::f16)
        peak = peaks["bf16_tflops_sustained"] / N_PRODUCTS[prec]
        note = (f"{peak_src} bf16 sustained (= f16 rate) / {N_PRODUCTS[prec]} products per useful "
                f"product")
        bound = "tensor"
    else:
        peak = alu[prec]["tflops"] if alu else None
        note = (f"measured {'FFMA' if prec == 'fp32' else 'DFMA'} throughput of this GPU "
                f"(libgwpeaks)") if peak else "not measured"
        bound = "alu"
    return {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if (achieved and peak) else None,
            "traffic": traffic, "traffic_unit": "bytes per launch",
            "peak_note": note}


def _traffic(prec, step_flops):
    """DRAM bytes per launch of the two tensor-core kernels on the bench
    workload, from the one-pass ncu counters of a small case of the same
    kernels (profiles/traffic_fp16x3_ribbon120.json), scaled to a full launch
    by the useful flops each launch processes: X and Y written, panels and G
    read, and step C's operand reads all grow with that work.  Empty when the
    record was taken on another kernel source or form."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic_fp16x3_ribbon120.json")
    src = os.path.join(ROOT, "paper_2104_09857_gb300", "csrc", "k_tc.cu")
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return {}
    if rec.get("k_tc_sha256") != sha or rec.get("form") != prec or not step_flops:
        return {}
    nb = max(1.0, step_flops["batches"])
    ab = (rec["step_a_bytes"] / rec["step_a_flops"] * step_flops["a"] / nb +
          rec["step_b_bytes"] / rec["step_b_flops"] * step_flops["b"] / nb) / 2.0
    c = rec["step_c_bytes"] / rec["step_c_flops"] * step_flops["c"] / nb
    return {"ab": ab, "c": c}


def _block_errors(got_blocks, ref_blocks):
    """(relative Frobenius error, element error over max |ref|) of a sample."""
    import numpy as np

    num = sum(float(np.sum((g - r) ** 2)) for g, r in zip(got_blocks, ref_blocks))
    den = sum(float(np.sum(r ** 2)) for r in ref_blocks)
    emax = max(float(np.abs(g - r).max()) for g, r in zip(got_blocks, ref_blocks))
    rmax = max(float(np.abs(r).max()) for r in ref_blocks)
    return ((num / den) ** 0.5 if den > 0 else None), (emax / rmax if rmax > 0 else None)


def _diag_blocks(chi2d, ri, atoms):
    return [chi2d[ri[p]:ri[p + 1], ri[p]:ri[p + 1]].cpu().numpy() for p in atoms]


def _train_screen(Context, device, thr, precision):
    """Train the learned screen on task logs of the benzene ring (the first
    configuration) and two short ribbons of the benchmark's family, and
    calibrate its margin on held-out tasks.  Returns (params, margin, info)."""
    import numpy as np

    from paper_2104_09857_gb300 import _lib
    from synth import make_case

    feats, tgts = [], []
    for name, nt in (("benzene", 6), ("ribbon28", 4), ("ribbon60", 3)):
        c = make_case(name, n_tau=nt, thr=1e-9)
        with Context(device) as lc:
            lc.load_case(c)
            f, t = _lib.gw_mlp_log(lc.ctx, 0, nt, thr, _lib.PRECISIONS[precision])
        feats.append(f)
        tgts.append(t)
    x = np.concatenate(feats)
    y = np.concatenate(tgts)
    keep = y > -39.0
    x, y = x[keep], y[keep]
    idx = np.random.default_rng(3).permutation(len(y))
    n_tr = int(0.8 * len(y))
    tr, va = idx[:n_tr], idx[n_tr:]
    with Context(device) as tc:
        _lib.gw_mlp_init(tc.ctx, 17)
        t0 = time.perf_counter()
        losses = _lib.gw_mlp_train(tc.ctx, x[tr], y[tr], epochs=400, batch=0, lr=3e-3, seed=5)
        t_train = time.perf_counter() - t0
        pv = _lib.gw_mlp_predict(tc.ctx, x[va])
        params = _lib.gw_mlp_get_params(tc.ctx)
    margin = float(np.max(y[va] - pv)) + 0.25
    return params, margin, {"samples": int(len(y)), "loss_first": float(losses[0]),
                            "loss_last": float(losses[-1]), "train_s": t_train,
                            "margin": margin, "trained_on": "benzene, ribbon28, ribbon60 task logs"}


def _per_tau_parity(case, run_tau, out, ri, prec, taus):
    """Error of the timed form at the given tau points, each on the diagonal
    chi block of one RI atom (atom j of a seeded permutation) that the FP64
    block oracle computes from its own M and N slices."""
    import numpy as np
    import torch

    from oracle import chi as oc

    bo = oc.BlockOracle(case)
    perm = np.random.default_rng(20210420).permutation(case.system.n_atoms)
    per_tau, oracle_blocks = [], {}
    for j in taus:
        a = int(perm[j])
        ref = bo.block(j, a, a, {})
        oracle_blocks[j] = (a, ref)
        run_tau(j)
        torch.cuda.synchronize()
        rel, el = _block_errors(_diag_blocks(out[0], ri, [a]), [ref])
        per_tau.append({"tau_index": j, "atom": a, "rel_frobenius": rel, "rel_element": el})
    res = {"form": prec, "reference": "numpy FP64 block oracle", "per_tau": per_tau,
           "max_rel_frobenius": max(p["rel_frobenius"] for p in per_tau),
           "max_rel_element": max(p["rel_element"] for p in per_tau)}
    return res, oracle_blocks


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__ as g

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    g.build()
    from paper_2104_09857_gb300 import Context
    from synth import make_case

    peaks, peak_src = _peaks()
    alu = alu_peaks() if args.alu_peaks else None
    prec = args.precision
    t_gen = time.perf_counter()
    case = make_case(args.workload)
    t_gen = time.perf_counter() - t_gen
    n_tau = len(case.tau)
    stream = torch.cuda.current_stream()
    ctx = Context(local, stream)
    if args.batch_atoms > 0:
        ctx.set_option("batch_atoms", args.batch_atoms)
    if args.batch_bytes > 0:
        ctx.set_option("batch_bytes", args.batch_bytes)
    ctx.load_case(case)
    nri = ctx.nri
    out = torch.empty((1, nri, nri), dtype=torch.float64, device=f"cuda:{local}")

    def step(j, precision, screening=None):
        if screening is None:
            ctx.chi_tau(case.thr, precision, j, 1, out=out)
        else:
            ctx.chi_tau(case.thr, precision, j, 1, out=out, screening=screening)
        return ctx.stats()

    # schedule search of the tensor-core route (before the warm-up; the
    # context keeps the chosen knobs)
    tune = None
    if args.autotune and prec in SPLIT_FORMS:
        from paper_2104_09857_gb300 import _lib as _l

        trials = _l.gw_autotune(ctx.ctx, n_tau // 2, case.thr, _l.PRECISIONS[prec])
        best = min(trials, key=lambda t: t["ms"])
        tune = {"tau_index": n_tau // 2, "trials": trials,
                "chosen": {k: best[k] for k in ("panel_staged", "c_split_k", "batch_bytes",
                                                "mu_chunk_atoms")},
                "start_ms": trials[0]["ms"], "chosen_ms": best["ms"]}
    # warm-up (W steps on the first tau points of this rank's cycle)
    for w in range(args.warmup):
        step(tau_index(w, world, rank, n_tau), prec)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    agg = {"flops_useful": 0.0, "flops_c": 0.0, "ms_step_c_kernel": 0.0, "kernel_launches": 0,
           "flops_issued": 0.0, "c_launches": 0, "ms_step_ab": 0.0, "ms_greens": 0.0,
           "flops_a": 0.0, "flops_b": 0.0, "n_batches": 0}
    for i in range(args.steps):
        st = step(tau_index(i, world, rank, n_tau), prec)
        for k in agg:
            agg[k] += st[k]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    t_local = ms / 1e3
    flops_local = agg["flops_useful"]
    t_job, flops_job = job_totals(t_local, flops_local, f"cuda:{local}")
    value = flops_job / t_job / 1e12
    ms_per_tau = t_job * 1e3 / max(1, args.steps)  # per tau point on one GPU

    # rooflines of the two tensor-core kernels: steps A/B (k_tc_persistent
    # PanelJob, two launches per batch) and step C (ChiJob, one per batch);
    # "roofline" is the one that takes more time
    nb = max(1, agg["n_batches"])
    traffic = _traffic(prec, {"a": agg["flops_a"], "b": agg["flops_b"], "c": agg["flops_c"],
                              "batches": float(nb)})
    roof_ab = _roof(agg["flops_a"] + agg["flops_b"], agg["ms_step_ab"] / 1e3, prec, peaks, peak_src,
                    "steps A/B (panel job; time includes the two G gathers)", traffic.get("ab"), alu)
    roof_c = _roof(agg["flops_c"], agg["ms_step_c_kernel"] / 1e3, prec, peaks, peak_src,
                   "step C (chi job)", traffic.get("c"), alu)
    for r, n_l in ((roof_ab, 2 * nb), (roof_c, nb)):
        r["launches"] = n_l
    if agg["ms_step_ab"] >= agg["ms_step_c_kernel"]:
        roof, roof_other = roof_ab, roof_c
    else:
        roof, roof_other = roof_c, roof_ab

    result = {
        "metric": "chi(i tau) useful TFLOP/s (time per tau point), mixed vs FP64 at <=1e-6 rel err",
        "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_job * 1e3 / max(1, args.steps),
        "ms_per_tau": ms_per_tau, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x3": "bf16x3", "bf16x6": "bf16x6",
                                       "fp16x3": "f16x3", "fp64": "f64"}[prec],
        "data": "synthetic",
        "config": {"workload": ("armchair-ribbon-298 (200 C + 98 H, 3090 AO / 7176 RI, "
                                "20 tau in [0.01, 50] a.u., thr 1e-9)") if args.workload == WORKLOAD
                   else f"{case.system.name} ({case.system.nao_total} AO / "
                        f"{case.system.nri_total} RI, {len(case.tau)} tau, thr {case.thr:g})",
                   "form": prec, "l2": "inputs and per-step operands larger than L2 (11 GB 3c)",
                   "parallelism": f"tau-sharded replicas x{world}"},
        "roofline": roof,
        "roofline_other": roof_other,
        "step_flops": {"a": agg["flops_a"] / max(1, args.steps), "b": agg["flops_b"] / max(1, args.steps),
                       "c": agg["flops_c"] / max(1, args.steps), "batches": agg["n_batches"] / max(1, args.steps)},
        "step_ms": {"greens": agg["ms_greens"] / max(1, args.steps),
                    "ab_kernels": agg["ms_step_ab"] / max(1, args.steps),
                    "c_kernel": agg["ms_step_c_kernel"] / max(1, args.steps)},
        "gpu_launches": int(agg["kernel_launches"]),
        "clocks": clk,
    }
    if alu:
        result["alu_peaks"] = alu
    if tune:
        result["autotune"] = tune

    if rank == 0 and world == 1 and args.workload == WORKLOAD:
        from oracle import chi as oc

        ri = np.concatenate([[0], np.cumsum(case.system.n_ri)])
        jm = n_tau // 2
        # CPU oracle on a bounded sample of tau index jm; its diagonal blocks
        # are the sample every form below is checked on
        flops_oracle = _useful_flops_oracle_side(case, jm)
        res = cpu_oracle_sample(case, args.cpu_samples, flops_oracle)
        result["cpu_baseline"] = {k: v for k, v in res.items()
                                  if k not in ("sample_seconds", "tau_index", "blocks")}
        atoms_m = sorted(res["blocks"])
        refs_m = [res["blocks"][p] for p in atoms_m]
        # every form at tau index jm: time, useful TFLOP/s, sampled error
        forms = {}
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for form in args.forms.split(","):
            if not form:
                continue
            step(jm, form)  # first call of a form builds its operands
            torch.cuda.synchronize()
            e0.record(stream)
            st = step(jm, form)
            e1.record(stream)
            torch.cuda.synchronize()
            f_ms = e0.elapsed_time(e1)
            rel, el = _block_errors(_diag_blocks(out[0], ri, atoms_m), refs_m)
            forms[form] = {"ms_per_tau": f_ms, "useful_tflops": st["flops_useful"] / f_ms / 1e9,
                           "rel_frobenius": rel, "rel_element": el,
                           "roofline_step_c": _roof(st["flops_c"], st["ms_step_c_kernel"] / 1e3, form,
                                                    peaks, peak_src, "step C", None, alu)}
            if form == "fp64":
                forms[form]["speedup_timed_form_over_fp64"] = f_ms / ms_per_tau
        forms["tau_index"] = jm
        forms["sample"] = f"diagonal chi blocks of RI atoms {atoms_m} at tau index {jm}"
        forms["useful_flops_library"] = st["flops_useful"]
        forms["useful_flops_oracle"] = flops_oracle
        result["forms"] = forms
        # per-tau parity of the timed form: one diagonal block per tau point
        oracle_blocks = {}
        if args.parity_taus > 0:
            result["parity"], oracle_blocks = _per_tau_parity(
                case, lambda j: step(j, prec), out, ri, prec, list(range(min(args.parity_taus, n_tau))))
        # learned screening at the bench threshold: time, skipped tasks,
        # per-tau error on the same oracle blocks
        if args.learned:
            params, margin, info = _train_screen(Context, local, case.thr, prec)
            from paper_2104_09857_gb300 import _lib

            _lib.gw_mlp_set_params(ctx.ctx, params)
            ctx.set_option("mlp_margin", margin)
            lt = []
            l_ms = 0.0
            skipped = seen = 0
            fl_u = fl_i = fl_i_plain = 0.0
            for j in range(n_tau):
                st_plain = step(j, prec)
                fl_i_plain += st_plain["flops_issued"]
                torch.cuda.synchronize()
                e0.record(stream)
                st = step(j, prec, screening=_lib.GW_SCREEN_MLP)
                e1.record(stream)
                torch.cuda.synchronize()
                l_ms += e0.elapsed_time(e1)
                skipped += st["tasks_skipped"]
                seen += st["tasks_seen"]
                fl_u += st["flops_useful"]
                fl_i += st["flops_issued"]
                if j in oracle_blocks:
                    a, ref = oracle_blocks[j]
                    rel, el = _block_errors(_diag_blocks(out[0], ri, [a]), [ref])
                    lt.append({"tau_index": j, "rel_frobenius": rel, "rel_element": el})
            result["learned"] = {
                "ms_per_tau": l_ms / n_tau, "ms_per_tau_norm_bound": ms_per_tau,
                "tasks_skipped": skipped, "tasks_seen": seen,
                "skipped_fraction": skipped / seen if seen else None,
                "flops_issued_fraction": fl_i / fl_i_plain if fl_i_plain else None,
                "useful_tflops_credited": fl_u / (l_ms / 1e3) / 1e12 if l_ms else None,
                "per_tau": lt,
                "max_rel_frobenius": max((p["rel_frobenius"] for p in lt), default=None),
                "training": info}
        # end to end through host buffers: upload inputs, chi, download
        if args.e2e_steps > 0:
            t3 = case.t3c
            pin_data = torch.from_numpy(t3.data).pin_memory()
            pin_blk = torch.from_numpy(np.ascontiguousarray(t3.blocks)).pin_memory()
            pin_c = torch.from_numpy(case.C).pin_memory()
            host_out = torch.empty((1, nri, nri), dtype=torch.float64).pin_memory()
            s = case.system
            e_fl = 0.0
            t0 = time.perf_counter()
            for i in range(args.e2e_steps):
                ctx.set_basis(s.xyz, s.n_ao, s.n_ri)
                ctx.set_3c_tensor(pin_blk.numpy(), pin_data.numpy())
                ctx.set_greens(pin_c.numpy(), case.eps, case.n_occ, case.mu_fermi, case.tau)
                ctx.chi_tau(case.thr, prec, (i * 7) % n_tau, 1, out=host_out.numpy())
                e_fl += ctx.stats()["flops_useful"]
            torch.cuda.synchronize()
            t_e = time.perf_counter() - t0
            result["e2e"] = {"value": e_fl / t_e / 1e12, "unit": "TFLOP/s",
                             "h2d_bytes_per_step": int(t3.data.nbytes + t3.blocks.nbytes +
                                                       case.C.nbytes + case.eps.nbytes +
                                                       case.tau.nbytes),
                             "d2h_bytes_per_step": int(nri * nri * 8),
                             "ms_per_step": t_e * 1e3 / args.e2e_steps}
        result["setup"] = {"generate_s": t_gen}
    elif rank == 0 and world == 1 and args.parity_taus > 0:
        # other workloads: sampled parity at tau points spread over the grid
        ri = np.concatenate([[0], np.cumsum(case.system.n_ri)])
        taus = sorted({int(round(x)) for x in np.linspace(0, n_tau - 1, min(args.parity_taus, n_tau))})
        result["parity"], _ = _per_tau_parity(case, lambda j: step(j, prec), out, ri, prec, taus)
        result["setup"] = {"generate_s": t_gen}
    ctx.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_sigma_batch(args):
    """The batched self-energy workload: Sigma^c(+-i tau) of HOMO and LUMO for
    64 molecules of 10-150 atoms (rings and ribbon segments, 20 tau points,
    thr 1e-9, synthetic NSD W) through gw_sigma_tau_batch, the split form
    against the plain FP64 form, with per-molecule errors against the block
    oracle on a sample of molecules."""
    import numpy as np
    import torch

    import __graft_entry__ as g

    g.build()
    from oracle import sigma as osg
    from paper_2104_09857_gb300 import Context, _lib
    from synth import case_from_system, molecule_set
    from synth.chain_inputs import synthetic_w

    mols = molecule_set(64, 10, 150, 20210425)
    ctxs, ws, orbs, sizes = [], [], [], []
    t0 = time.perf_counter()
    for i, m in enumerate(mols):
        c = case_from_system(m, 20, 1e-9, 20210425 + i)
        ctx = Context(0)
        ctx.load_case(c)
        ctxs.append(ctx)
        ws.append(synthetic_w(c.system.nri_total, c.tau, 100 + i))
        orbs.append([c.n_occ - 1, c.n_occ])
        sizes.append((c.system.n_atoms, c.system.nao_total, c.system.nri_total))
        del c
    t_gen = time.perf_counter() - t0
    handles = [c.ctx for c in ctxs]
    # dense product flops of Eq. 10 per tau point: Y = B W and Z = Y B^T per orbital
    flops_tau = sum(2 * len(o) * (ao * ri * ri + ao * ao * ri) for o, (_, ao, ri) in zip(orbs, sizes))
    res = {}
    outs = {}
    for prec in (args.precision, "fp64"):
        _lib.gw_sigma_tau_batch(handles, ws, orbs, 1e-9, _lib.PRECISIONS[prec])  # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = _lib.gw_sigma_tau_batch(handles, ws, orbs, 1e-9, _lib.PRECISIONS[prec])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        outs[prec] = out
        res[prec] = {"s_per_call": dt, "ms_per_tau": dt * 1e3 / 20, "tflops_dense_products": 20 * flops_tau / dt / 1e12}
    for c in ctxs:
        c.close()
    # per-molecule error on a sample spread over the sizes (oracle on the host)
    order = np.argsort([s_[0] for s_ in sizes])
    pick = sorted({int(order[int(round(x))]) for x in np.linspace(0, 63, args.sigma_check)})
    taus = [0, 9, 19]
    errs = []
    for i in pick:
        c = case_from_system(mols[i], 20, 1e-9, 20210425 + i)
        ref = osg.sigma_blocks(c, ws[i], orbs[i], taus)
        sc = np.abs(ref).max()
        errs.append({"molecule": i, "atoms": sizes[i][0],
                     "err_" + args.precision: float(np.abs(outs[args.precision][i][:, taus] - ref).max() / sc),
                     "err_fp64": float(np.abs(outs["fp64"][i][:, taus] - ref).max() / sc)})
    line = {"metric": "batched Sigma^c(i tau) of HOMO/LUMO, 64 molecules, time per tau point",
            "value": res[args.precision]["ms_per_tau"], "unit": "ms per tau point (all 64 molecules)",
            "higher_is_better": False, "n_gpus": 1, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "64 molecules, 10-150 atoms (rings and ribbon segments), "
                                   f"{sum(s_[1] for s_ in sizes)} AO / {sum(s_[2] for s_ in sizes)} RI in all, "
                                   "20 tau, thr 1e-9, HOMO and LUMO"},
            "forms": res, "speedup_split_over_fp64": res["fp64"]["s_per_call"] / res[args.precision]["s_per_call"],
            "dense_product_flops_per_tau": flops_tau, "errors_vs_oracle": errs,
            "max_err_split": max(e["err_" + args.precision] for e in errs),
            "max_err_fp64": max(e["err_fp64"] for e in errs), "setup_s": t_gen}
    print(json.dumps(line), flush=True)


def run_learned_cluster(args):
    """Learned screening on the 500-atom disordered cluster (thr 1e-9): the
    norm-bound screen against the learned one on the timed form at a few tau
    points, with skipped tasks, time, and the error of both against the FP64
    block oracle on sampled diagonal blocks.  The tensor is kept in FP32 on the
    device and the split panels are streamed (the whole set would need about
    405 GB)."""
    import numpy as np
    import torch

    import __graft_entry__ as g

    g.build()
    from paper_2104_09857_gb300 import Context, _lib
    from synth import make_case

    prec = args.precision
    t0 = time.perf_counter()
    case = make_case("cluster500")
    t_gen = time.perf_counter() - t0
    params, margin, info = _train_screen(Context, 0, case.thr, prec)
    stream = torch.cuda.current_stream()
    ctx = Context(0, stream)
    ctx.set_option("tensor_fp32", 1)
    ctx.set_option("batch_bytes", args.batch_bytes if args.batch_bytes > 0 else 20e9)
    ctx.load_case(case)
    _lib.gw_mlp_set_params(ctx.ctx, params)
    ctx.set_option("mlp_margin", margin)
    nri = ctx.nri
    out = torch.empty((1, nri, nri), dtype=torch.float64, device="cuda:0")
    ri = np.concatenate([[0], np.cumsum(case.system.n_ri)])
    taus = [int(t) for t in args.cluster_taus.split(",")]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    from oracle import chi as oc

    bo = oc.BlockOracle(case)
    perm = np.random.default_rng(20210420).permutation(case.system.n_atoms)
    rows = []
    for j in taus:
        a = int(perm[j])
        rec = {"tau_index": j, "tau": float(case.tau[j]), "atom": a}
        got = {}
        for name, scr in (("norm_bound", _lib.GW_SCREEN_BOUND), ("learned", _lib.GW_SCREEN_MLP)):
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.chi_tau(case.thr, prec, j, 1, out=out, screening=scr)
            e1.record(stream)
            torch.cuda.synchronize()
            st = ctx.stats()
            got[name] = _diag_blocks(out[0], ri, [a])
            rec[name] = {"ms": e0.elapsed_time(e1), "useful_tflops": st["flops_useful"] / e0.elapsed_time(e1) / 1e9,
                         "flops_issued": st["flops_issued"], "tasks_seen": st["tasks_seen"],
                         "tasks_skipped": st["tasks_skipped"], "n_batches": st["n_batches"]}
        ref = bo.block(j, a, a, {})
        for name in got:
            rel, el = _block_errors(got[name], [ref])
            rec[name].update({"rel_frobenius": rel, "rel_element": el})
        rel, el = _block_errors(got["learned"], got["norm_bound"])
        rec["learned_vs_norm_bound"] = {"rel_frobenius": rel, "rel_element": el}
        rows.append(rec)
    ctx.close()
    line = {"metric": "learned vs norm-bound screening of chi(i tau), 500-atom disordered cluster",
            "unit": "ms per tau point", "n_gpus": 1, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"cluster-500 ({case.system.nao_total} AO / {case.system.nri_total} RI, "
                                   "0.1 atoms/A^3, thr 1e-9)", "tensor": "FP32 on the device",
                       "panels": "streamed per batch"},
            "per_tau": rows, "training": info, "setup_s": t_gen}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16x3", "bf16x6", "fp16x3", "fp64"],
                    default="fp16x3")
    ap.add_argument("--forms", default="fp64,fp32,bf16x3,bf16x6",
                    help="other forms timed on one tau point and checked on the oracle sample")
    ap.add_argument("--parity-taus", type=int, default=20,
                    help="tau points of the timed form checked against the oracle (one block each)")
    ap.add_argument("--learned", type=int, default=1,
                    help="train the learned screen and time it on every tau point")
    ap.add_argument("--alu-peaks", type=int, default=1,
                    help="measure the FFMA/DFMA throughput the FP32/FP64 rooflines divide by")
    ap.add_argument("--peaks", action="store_true",
                    help="only measure and print the FFMA/DFMA throughput of this GPU")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-samples", type=int, default=2)
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic case (smaller ones serve profiling); the bench line is %(default)s")
    ap.add_argument("--batch-atoms", type=int, default=0,
                    help="upper limit on sigma-atoms per operand batch (0: byte budget only)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="search the tensor-core schedule (gw_autotune) before the warm-up")
    ap.add_argument("--batch-bytes", type=float, default=0,
                    help="device bytes for one batch's X and Y operands (0: the library default)")
    ap.add_argument("--sigma-check", type=int, default=6,
                    help="batched self-energy workload: molecules checked against the oracle")
    ap.add_argument("--cluster-taus", default="1,3",
                    help="500-atom cluster workload: tau indices (of 6) timed and checked")
    args = ap.parse_args()
    if args.workload == "cluster500":
        run_learned_cluster(args)
        return
    if args.workload == "molecules64":
        run_sigma_batch(args)
        return
    if args.peaks:
        import __graft_entry__ as g

        g.build()
        print(json.dumps(alu_peaks()), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
