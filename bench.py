"""Benchmark of the sparse-wavefunction UCC hot path on one GB300.

A step is one full evaluation on the 64-spin-orbital workload: the ordered
product of UCC factors applied to the reference with eps pruning (Eq. 3,
Methods section), E = <psi|H|psi>/<psi|psi>, and dE/dtheta for every factor
by the adjoint sweep.  The JSON line reports

  value  = forward det-rotations per second of full-evaluation time (each
           linked determinant pair rotated by one factor is one det-rotation;
           the count is the oracle's and the kernel's, which agree exactly),
  e2e    = the same metric through the public C-ABI call with host buffers
           (theta uploaded from pinned host memory, E and dE/dtheta read back
           every step),
  evals_per_s, apply-only det-rotations/s, the roofline of the dominant kernel,
  clocks sampled during the timed region, and the CPU oracle timed on a
  bounded prefix of the same workload (cpu_baseline).

``--impl reference`` times the CPU oracle (the repository's plain reference
implementation; the paper ships no code) on a bounded prefix sample of the same
workload and prints the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "UCC det-rotations/s; energy+adjoint-gradient evals/s at 64 qubits vs plain"
UNIT = "det-rotations/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg4", help="cfg4 (default) or cfgN[:prefix] for exploration")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    return ap.parse_args()


def workload(spec):
    from paper_2301_05726_gb300 import synth
    name, _, pre = spec.partition(":")
    cfg = int(name.replace("cfg", ""))
    prob = synth.config_problem(cfg)
    if pre:
        prob = prob.prefix(int(pre))
    return prob


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region (read from its
    output pipe by a thread)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.reader = None

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.reader = threading.Thread(target=lambda: self.lines.extend(self.proc.stdout), daemon=True)
        self.reader.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.reader.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in list(self.lines):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_time(prob, n_factors, with_grad=True):
    """One oracle evaluation (apply + energy + adjoint) of the first n_factors factors:
    (forward rotations, seconds)."""
    import oracle
    sub = prob.prefix(min(n_factors, prob.n_exc))
    o = oracle.Oracle(sub)
    t0 = time.perf_counter()
    _, _, cnt = o.apply()
    if with_grad:
        o.gradient()
    return cnt["rotations"], time.perf_counter() - t0


def oracle_prefix(prob, seconds, with_grad=True):
    """The longest factor prefix whose oracle evaluation should take at most ~`seconds`: prefixes grow
    by 1.5x while the cost of the next one, extrapolated from the growth of the last two (the map and so
    the cost per factor grow with the prefix), stays within the budget.
    Returns (prefix, its forward rotations, its seconds)."""
    pre, prev = 16, None
    while True:
        rot, dt = oracle_time(prob, pre, with_grad)
        nxt = min(prob.n_exc, max(pre + 1, int(pre * 1.5)))
        if pre >= prob.n_exc:
            return pre, rot, dt
        growth = max(1.5, dt / prev) if prev else 4.0
        if dt * growth > seconds:
            return pre, rot, dt
        pre, prev = nxt, dt


def oracle_sample(prob, seconds, with_grad=True, n_factors=None):
    """Time the CPU oracle on a prefix of the workload sized to ~`seconds` (or on the first n_factors).
    Returns (forward rotations per eval second, evals/s, prefix, seconds)."""
    if n_factors is None:
        nf, rot, dt = oracle_prefix(prob, seconds, with_grad)
    else:
        nf = n_factors
        rot, dt = oracle_time(prob, nf, with_grad)
    return rot / dt, 1.0 / dt, nf, dt


def run_reference(args, prob):
    import torch  # noqa: F401  (same environment as the other arm)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    nf_fixed = oracle_prefix(prob, per_step)[0]  # one calibration; every step then runs the same prefix
    rates = []
    desc = None
    for s in range(args.warmup + args.steps):
        r, evals, nf, dt = oracle_sample(prob, per_step, n_factors=nf_fixed)
        if s >= args.warmup:
            rates.append(r)
            desc = f"{prob.name} first {nf} of {prob.n_exc} factors: apply + energy + adjoint, {dt:.1f}s"
    val = sorted(rates)[len(rates) // 2]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": prob.name, "n_so": prob.n_so, "n_elec": prob.n_elec, "n_factors": prob.n_exc,
                       "eps": prob.eps},
            "cpu_baseline": {"kind": "oracle", "value": val, "unit": UNIT, "cores": 1, "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def flush_l2(buf):
    buf.add_(1.0)


# DRAM traffic per algorithmic byte of a kernel, from one ncu capture of every launch of one evaluation
# of the 1000-factor prefix (profiles/k_reverse_traffic_64so_prefix1000.md); a launch's traffic is taken
# as this ratio times its algorithmic bytes.  To be re-measured (or removed) whenever the kernel changes.
TRAFFIC_PER_ALGORITHMIC_BYTE = {"k_reverse": 1.75}


def _roofline(kernel, bytes_, ms, launches, hbm, peak_kind):
    ach = bytes_ / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    ratio = TRAFFIC_PER_ALGORITHMIC_BYTE.get(kernel)
    traffic = ratio * bytes_ / max(1, launches) if ratio else None
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
            "kernel": kernel, "peak_kind": peak_kind, "launches": launches,
            "avg_launch_ms": ms / max(1, launches), "algorithmic_bytes": bytes_, "total_ms": ms}


def run_ours(args, prob):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2301_05726_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2301_05726_gb300.api import UCCContext

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = UCCContext(prob)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MB > L2
    theta_host = torch.tensor(prob.theta, dtype=torch.float64).pin_memory()
    grad_host = torch.empty(prob.n_exc, dtype=torch.float64).pin_memory()
    grad_dev = torch.empty(prob.n_exc, dtype=torch.float64, device=dev)

    def step_device():
        E, _ = ctx.gradient(out=grad_dev)
        return E

    for _ in range(args.warmup):
        flush_l2(flush)
        step_device()
    torch.cuda.synchronize()

    # Device-timed region: inputs resident, CUDA events on the library's stream.
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    times = []
    tot = {}
    for _ in range(args.steps):
        flush_l2(flush)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        step_device()
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        for k, v in ctx.stats().items():
            tot[k] = tot.get(k, 0) + v
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = sum(times) / len(times)
    n_steps = len(times)
    # Replicas: the slowest rank's step time, the work of all ranks.
    from paper_2301_05726_gb300.replicas import combine_step
    ms, rot_all = combine_step(ms, tot["rotations"] / n_steps, device=dev)
    rot_per_eval = tot["rotations"] / n_steps
    value = rot_all / (ms / 1e3)

    # End to end through the public API with host buffers.
    e2e_times = []
    for _ in range(0 if args.no_e2e else max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_theta(theta_host.numpy())
        E, g = ctx.gradient()
        grad_host.copy_(torch.from_numpy(g))
        e2e_times.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * sum(e2e_times) / len(e2e_times) if e2e_times else float("nan")

    # "Plain": per-theta central differences on the GPU need 2K + 1 energy
    # evaluations (apply + energy); one is measured, the total extrapolated.
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.apply()
    ctx.energy()
    torch.cuda.synchronize()
    energy_eval_s = time.perf_counter() - t0
    plain_s = (2 * prob.n_exc + 1) * energy_eval_s

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    hbm, peak_kind = peaks()
    fwd_bytes = 8.0 * (tot["scanned"] + tot["recompute_scanned"]) + \
        48.0 * (tot["rotations"] + tot["recompute_rotations"]) + 32.0 * (tot["created"] + tot["recompute_created"])
    # per stored determinant: key + amplitude read, sigma written; per connected stored pair (visited once):
    # the partner amplitude read and one sigma update
    sig_bytes = 24.0 * tot["n_det"] + 16.0 * tot["sigma_hits"]
    # per pair as in the forward step plus lam of both members; the scan term counts the entries of psi_k
    # (the forward step's scan), not the dropped entries the sweep carries until it compacts
    rev_bytes = 8.0 * tot["scanned"] + 80.0 * tot["reverse_pairs"]
    kernels = {
        "k_forward": _roofline("k_forward", fwd_bytes, tot["forward_kernel_ms"], tot["forward_launches"], hbm,
                               peak_kind),
        "k_sigma": _roofline("k_sigma", sig_bytes, tot["energy_ms"], n_steps, hbm, peak_kind),
        "k_reverse": _roofline("k_reverse", rev_bytes, tot["reverse_kernel_ms"], tot["reverse_launches"], hbm,
                               peak_kind),
    }
    dom = max(kernels.values(), key=lambda r: r["total_ms"])
    roof = {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel", "peak_kind",
                                "avg_launch_ms")}
    cpu = None
    if not args.no_cpu_baseline:
        r, evals, nf, dt = oracle_sample(prob, args.cpu_seconds)
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{prob.name}: first {nf} of {prob.n_exc} factors, apply + energy + adjoint in {dt:.1f}s"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": prob.name, "n_so": prob.n_so, "n_elec": prob.n_elec, "n_factors": prob.n_exc,
                   "eps": prob.eps, "n_max": prob.n_max, "n_cut": prob.n_cut, "n_det": tot["n_det"] // n_steps,
                   "l2": "table larger than L2 + 256 MB flush per step",
                   "parallelism": "replicas" if world > 1 else "single"},
        "evals_per_s": world * 1e3 / ms,
        "apply_det_rotations_per_s": tot["rotations"] / (tot["apply_ms"] / 1e3) if tot["apply_ms"] > 0 else None,
        "phase_ms": {"forward": tot["apply_ms"] / n_steps, "energy": tot["energy_ms"] / n_steps,
                     "reverse_incl_recompute": tot["reverse_ms"] / n_steps},
        "vs_plain": {"plain": "per-theta central differences on the GPU, 2K+1 energy evaluations",
                     "energy_eval_s": energy_eval_s, "plain_gradient_s_extrapolated": plain_s,
                     "adjoint_gradient_s": ms / 1e3, "speedup": plain_s / (ms / 1e3)},
        "e2e": {"value": rot_all / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": 48 * prob.n_exc, "d2h_bytes_per_step": 8 * prob.n_exc + 8},
        "gpu_launches": int(tot["kernel_launches"]),
        "counts_per_step": {k: int(tot[k] // n_steps) for k in (
            "rotations", "created", "dropped_new", "dropped_old", "cut", "scanned", "rebuilds", "tape_entries",
            "sigma_probes", "sigma_hits", "reverse_pairs", "reverse_scanned", "recompute_rotations")},
        "roofline": roof,
        "kernels": {k: {x: v[x] for x in ("achieved", "frac", "launches", "avg_launch_ms", "total_ms")}
                    for k, v in kernels.items()},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    prob = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, prob)
    else:
        run_ours(args, prob)


if __name__ == "__main__":
    main()
