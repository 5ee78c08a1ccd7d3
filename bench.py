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
Also reported: ms per tau point, the FP64 form on a subset of tau points,
the rooflines of the two tensor-core kernels (steps A/B and step C), a
sampled error against the FP64 block oracle, an end-to-end figure through
host buffers, and the CPU oracle on a bounded sample.

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
FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # FP32 lanes x 2 flop x max SM clock
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
    flops_tau = _useful_flops_oracle_side(case)
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


def _useful_flops_oracle_side(case) -> float:
    """Useful flops of one tau point counted from the stored 3c blocks alone,
    for a tau at which no Green's-function block is filtered (true for this
    workload away from the largest tau): steps A and B do
    2 nao n_l n_s n_P per stored block orientation; step C does
    2 n_m n_s n_p n_q for every (m, s, p <= q) with p in the RI window of s
    and q in the RI window of m (the windows of nonzero intermediates)."""
    import numpy as np

    s = case.system
    t3 = case.t3c
    blk = t3.blocks
    na = s.n_ao[blk[:, 0]].astype(float)
    nb = s.n_ao[blk[:, 1]].astype(float)
    npp = s.n_ri[blk[:, 2]].astype(float)
    w = na * nb * npp * np.where(blk[:, 0] == blk[:, 1], 1.0, 2.0)
    fa = 2.0 * s.nao_total * w.sum()
    n_at = s.n_atoms
    win = np.zeros((n_at, n_at), dtype=bool)
    win[blk[:, 0], blk[:, 2]] = True
    win[blk[:, 1], blk[:, 2]] = True
    x = win * s.n_ri[None, :].astype(float)            # x[s, p]
    ysuf = np.cumsum(x[:, ::-1], axis=1)[:, ::-1]      # ysuf[m, p] = sum_{q >= p} x[m, q]
    pairs = x @ ysuf.T                                 # [s, m]
    nao = s.n_ao.astype(float)
    fc = 2.0 * float(nao @ pairs @ nao)
    return 2.0 * fa + fc


def _roof(flops, seconds, prec, peaks, peak_src, kernel, traffic):
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
        peak = FFMA_PEAK_TFLOPS if prec == "fp32" else None
        note = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz" if peak else "FP64 ALU"
        bound = "alu"
    return {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if (achieved and peak) else None,
            "traffic": traffic, "traffic_unit": "bytes per launch",
            "peak_note": note}


def _traffic(prec):
    """DRAM bytes per launch of the tensor-core kernels from the committed ncu
    summary, if it was taken on the current kernel source and form."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic_fp16x3_ribbon298.json")
    src = os.path.join(ROOT, "paper_2104_09857_gb300", "csrc", "k_tc.cu")
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return {}
    if rec.get("k_tc_sha256") != sha or rec.get("form") != prec:
        return {}
    return {"ab": rec.get("panel_job_bytes_per_launch"), "c": rec.get("chi_job_bytes_per_launch")}


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
    prec = args.precision
    t_gen = time.perf_counter()
    case = make_case(args.workload)
    t_gen = time.perf_counter() - t_gen
    n_tau = len(case.tau)
    stream = torch.cuda.current_stream()
    ctx = Context(local, stream)
    if args.batch_atoms > 0:
        ctx.set_option("batch_atoms", args.batch_atoms)
    ctx.load_case(case)
    nri = ctx.nri
    out = torch.empty((1, nri, nri), dtype=torch.float64, device=f"cuda:{local}")

    def step(j, precision):
        ctx.chi_tau(case.thr, precision, j, 1, out=out)
        return ctx.stats()

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
    traffic = _traffic(prec)
    roof_ab = _roof(agg["flops_a"] + agg["flops_b"], agg["ms_step_ab"] / 1e3, prec, peaks, peak_src,
                    "steps A/B (panel job; time includes the two G gathers)", traffic.get("ab"))
    roof_c = _roof(agg["flops_c"], agg["ms_step_c_kernel"] / 1e3, prec, peaks, peak_src,
                   "step C (chi job)", traffic.get("c"))
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
        "step_ms": {"greens": agg["ms_greens"] / max(1, args.steps),
                    "ab_kernels": agg["ms_step_ab"] / max(1, args.steps),
                    "c_kernel": agg["ms_step_c_kernel"] / max(1, args.steps)},
        "gpu_launches": int(agg["kernel_launches"]),
        "clocks": clk,
    }

    if rank == 0 and world == 1:
        # FP64 form on a subset of tau points
        if args.fp64_taus > 0:
            f_fl, f_ms = 0.0, 0.0
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            for i in range(args.fp64_taus):
                j = (n_tau // 2 + i) % n_tau
                e0.record(stream)
                st = step(j, "fp64")
                e1.record(stream)
                torch.cuda.synchronize()
                f_ms += e0.elapsed_time(e1)
                f_fl += st["flops_useful"]
            result["fp64"] = {"ms_per_tau": f_ms / args.fp64_taus,
                              "useful_tflops": f_fl / (f_ms / 1e3) / 1e12,
                              "taus_timed": args.fp64_taus,
                              "speedup_mixed_over_fp64": (f_ms / args.fp64_taus) / ms_per_tau}
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
        # CPU oracle, bounded sample; its diagonal chi blocks also give a
        # sampled error of the timed form at that tau point
        if args.cpu_samples > 0:
            per_tau = flops_job / max(1, args.steps * world)
            res = cpu_oracle_sample(case, args.cpu_samples, per_tau)
            result["cpu_baseline"] = {k: v for k, v in res.items()
                                      if k not in ("sample_seconds", "tau_index", "blocks")}
            step(res["tau_index"], prec)
            torch.cuda.synchronize()
            ri = np.concatenate([[0], np.cumsum(case.system.n_ri)])
            num = den = 0.0
            emax = rmax = 0.0
            for p, ref in res["blocks"].items():
                got = out[0, ri[p]:ri[p + 1], ri[p]:ri[p + 1]].cpu().numpy()
                num += float(np.sum((got - ref) ** 2))
                den += float(np.sum(ref ** 2))
                emax = max(emax, float(np.abs(got - ref).max()))
                rmax = max(rmax, float(np.abs(ref).max()))
            result["parity"] = {"form": prec, "tau_index": res["tau_index"],
                                "blocks": [[int(p), int(p)] for p in res["blocks"]],
                                "rel_frobenius": (num / den) ** 0.5 if den > 0 else None,
                                "rel_element": emax / rmax if rmax > 0 else None,
                                "reference": "numpy FP64 block oracle"}
        result["setup"] = {"generate_s": t_gen}
    ctx.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16x3", "bf16x6", "fp16x3", "fp64"],
                    default="fp16x3")
    ap.add_argument("--fp64-taus", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-samples", type=int, default=1)
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic case (smaller ones serve profiling); the bench line is %(default)s")
    ap.add_argument("--batch-atoms", type=int, default=0,
                    help="upper limit on sigma-atoms per operand batch (0: byte budget only)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
