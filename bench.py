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
    ap.add_argument("--plain-components", type=int, default=2,
                    help="theta components timed by central differences on the main workload")
    ap.add_argument("--no-n1", action="store_true", help="skip the 40-spin-orbital adjoint/batched vs plain leg")
    ap.add_argument("--n1-fd-components", type=int, default=2)
    ap.add_argument("--n1-batch", type=int, default=2, help="theta vectors in the 40-spin-orbital batched leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-job batched leg")
    ap.add_argument("--no-wide", action="store_true", help="skip the 72-spin-orbital leg")
    ap.add_argument("--no-ncut", action="store_true", help="skip the fixed-parameter cut sweep")
    ap.add_argument("--n-max", type=int, default=None,
                    help="exploration: the workload's N_MAX (with --n-cut; default: the workload's own cut)")
    ap.add_argument("--n-cut", type=int, default=None)
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


# The CPU oracle's sample of the 64-spin-orbital workload, the same in the CPU-baseline leg and in the
# reference arm: its first 40 factors (apply + energy + adjoint, a few seconds on one core).
ORACLE_PREFIX = 40

# Bytes the library uploads per factor when theta comes from the host (the factor table entry: masks,
# Jordan-Wigner parity terms, cos, sin and 1/cos).
FACTOR_BYTES = 56


def host_info():
    """The host the oracle runs on: logical CPUs and the CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": os.uname().machine}


def oracle_leg(prob, repeats):
    """The oracle on the fixed prefix, `repeats` times: (median rate, median seconds, description)."""
    nf = min(ORACLE_PREFIX, prob.n_exc)
    runs = [oracle_time(prob, nf) for _ in range(repeats)]
    runs.sort(key=lambda r: r[1])
    rot, dt = runs[len(runs) // 2]
    desc = (f"{prob.name}: first {nf} of {prob.n_exc} factors (cut n_max={prob.n_max}, n_cut={prob.n_cut}), "
            f"apply + energy + adjoint, median of {repeats}: {dt:.2f} s")
    return rot / dt, dt, desc


def workload_config(prob):
    return {"workload": prob.name, "n_so": prob.n_so, "n_elec": prob.n_elec, "n_factors": prob.n_exc,
            "eps": prob.eps, "n_max": prob.n_max, "n_cut": prob.n_cut}


def run_reference(args, prob):
    import torch  # noqa: F401  (same environment as the other arm)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    rates, desc = [], None
    for s in range(args.warmup + args.steps):
        r, dt, desc = oracle_leg(prob, 1)
        if s >= args.warmup:
            rates.append(r)
    val = sorted(rates)[len(rates) // 2]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(prob), parallelism="single"),
            "cpu_baseline": {"kind": "oracle", "value": val, "unit": UNIT, "cores": 1, "sample": desc,
                             "host": host_info()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def flush_l2(buf):
    buf.add_(1.0)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per entry a launch scans, from one ncu capture
# of three launches of that kernel alone on a 1,000-factor prefix of the 64-so workload (about 8.6e6
# entries per launch, far larger than L2; the summary under profiles/ gives the command); a full-size
# launch's traffic is taken as this figure times the entries it scans.  A kernel is left out (traffic
# reported as null) once its code has changed since its capture.
TRAFFIC_PER_SCANNED_ENTRY = {"k_reverse": 47.3}


def _roofline(kernel, bytes_, ms, launches, hbm, peak_kind, scanned=0):
    ach = bytes_ / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    per = TRAFFIC_PER_SCANNED_ENTRY.get(kernel)
    traffic = per * scanned / max(1, launches) if per and scanned else None
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
            "kernel": kernel, "peak_kind": peak_kind, "launches": launches,
            "avg_launch_ms": ms / max(1, launches), "algorithmic_bytes": bytes_, "total_ms": ms}


def byte_models(tot):
    """Algorithmic bytes of the timed steps for the three kernels, in two models.

    pair model: every rotation is charged a full pair (both members' amplitudes read and written and a
    slot probe, 48 B; the reverse step also both adjoints, 80 B), whether or not the partner is stored.
    member model: a rotation whose partner is absent (created, or computed below eps and never stored)
    touches only its own member (16 B forward: amplitude read and write; 32 B reverse: amplitude and
    adjoint read and written); a stored pair is charged as in the pair model.  Both charge 8 B per key
    scanned and 32 B per created entry (key and amplitude written, slot claimed).  The energy: by
    buckets (route 2) a 32 B record written and read per core (sigma_probes counts the records) and 40 B
    per determinant (key and amplitude read by the record passes, sigma written and read back); per
    connection (route 1) 24 B per determinant and 16 B per connected stored pair."""
    scanned = tot["scanned"] + tot["recompute_scanned"]
    rot = tot["rotations"] + tot["recompute_rotations"]
    cre = tot["created"] + tot["recompute_created"]
    lone = min(rot, tot["created"] + tot["dropped_new"] + tot["recompute_created"])
    both = rot - lone
    rev_lone = min(tot["reverse_pairs"], tot["dropped_new"])
    rev_both = tot["reverse_pairs"] - rev_lone
    if tot.get("energy_route_last") == 2:
        sig = 64.0 * tot["sigma_probes"] + 40.0 * tot["n_det"]
    else:
        sig = 24.0 * tot["n_det"] + 16.0 * tot["sigma_hits"]
    return {
        "pair": {"k_forward": 8.0 * scanned + 48.0 * rot + 32.0 * cre, "energy": sig,
                 "k_reverse": 8.0 * tot["scanned"] + 80.0 * tot["reverse_pairs"]},
        "member": {"k_forward": 8.0 * scanned + 16.0 * lone + 48.0 * both + 32.0 * cre, "energy": sig,
                   "k_reverse": 8.0 * tot["scanned"] + 32.0 * rev_lone + 80.0 * rev_both},
    }


def plain_fd(ctx, prob, m, h=1e-6, seed=7):
    """Per-theta central differences on the GPU through the public API, timed on m randomly chosen
    components (2m energy evaluations: theta uploaded, apply, energy), and the extrapolation to all
    2K + 1 evaluations of a full gradient."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    comps = rng.choice(prob.n_exc, size=min(m, prob.n_exc), replace=False)
    th = np.array(prob.theta, dtype=np.float64)
    fd = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in comps:
        e = []
        for sgn in (1.0, -1.0):
            tt = th.copy()
            tt[k] += sgn * h
            ctx.set_theta(tt)
            ctx.apply()
            e.append(ctx.energy()[0])
        fd.append((e[0] - e[1]) / (2 * h))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ctx.set_theta(th)
    n_eval = 2 * len(comps)
    return {"components": [int(k) for k in comps], "energy_evaluations": n_eval, "seconds": dt,
            "s_per_energy_evaluation": dt / n_eval,
            "extrapolated_gradient_s": dt / n_eval * (2 * prob.n_exc + 1)}, np.array(fd)


def timed_gradients(ctx, n, out=None):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        E, g = ctx.gradient(out=out)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / n, E, g


def n1_leg(args):
    """The 40-spin-orbital workload (12 electrons, 9,954 factors, eps = 1e-8, the cut, gradient with
    sqrt(K) checkpointing): one adjoint gradient against per-theta central differences (timed on a
    random subset of components), and the batched form on several theta vectors."""
    import math
    import numpy as np
    from paper_2301_05726_gb300 import synth
    from paper_2301_05726_gb300.api import UCCContext, batch_run
    prob = synth.config_problem(3)
    stride = int(math.ceil(math.sqrt(prob.n_exc)))
    ctx = UCCContext(prob)
    ctx.set_options(checkpoint_stride=stride)
    ctx.gradient()  # warm-up
    t_adj, E, g = timed_gradients(ctx, 1)
    st = ctx.stats()
    plain, fd = plain_fd(ctx, prob, args.n1_fd_components)
    comps = plain["components"]
    out = {"workload": prob.name, "n_so": prob.n_so, "n_elec": prob.n_elec, "n_factors": prob.n_exc,
           "eps": prob.eps, "n_max": prob.n_max, "n_cut": prob.n_cut, "checkpoint_stride": stride,
           "n_det": st["n_det"], "adjoint_gradient_s": t_adj, "plain": plain,
           "speedup_adjoint_vs_plain": plain["extrapolated_gradient_s"] / t_adj, "target": 20.0}
    # Batched form: B theta vectors of the same problem (each its own context) in one call.
    B = args.n1_batch
    if B > 0:
        rng = np.random.default_rng(11)
        jobs = []
        for b in range(B):
            th = prob.theta * (1.0 + 0.01 * rng.standard_normal(prob.n_exc))
            c = UCCContext(prob.with_theta(th))
            c.set_options(checkpoint_stride=stride)
            jobs.append(c)
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch_run(jobs, prob.eps, with_grad=True)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        out["batched"] = {"jobs": B, "seconds": tb, "gradient_s_per_job": tb / B,
                          "speedup_vs_plain": plain["extrapolated_gradient_s"] / (tb / B)}
        for c in jobs:
            c.close()
    ctx.close()
    return out


def batch_leg(args):
    """The 256-job workload (16-36 spin-orbitals, 4-12 electrons, theta ~ N(0, 0.02), eps = 1e-8), each
    job with the paper's production cut (N_MAX = 8,000, N_CUT = 5,000): energies and adjoint gradients
    of all jobs through one ucc_batch_run call (persistent launches), and the same for a sample of jobs
    against the one-job path."""
    import torch
    from paper_2301_05726_gb300 import synth
    from paper_2301_05726_gb300.api import UCCContext, batch_run

    def jobs(ids):
        out = []
        for j in ids:
            p = synth.batch_job_problem(j)
            p.n_max, p.n_cut = BATCH_N_MAX, BATCH_N_CUT
            out.append(p)
        return out

    probs = jobs(range(256))
    ctxs = [UCCContext(p) for p in probs]
    batch_run(ctxs, 1e-8, with_grad=True)  # warm-up (tunes probe width and tiles once)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E, _ = batch_run(ctxs, 1e-8, with_grad=True)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    st = [c.stats() for c in ctxs]
    rot = sum(x["rotations"] for x in st)
    out = {"workload": "256 jobs, 16-36 so, 4-12 e, eps 1e-8, cut n_max=8000 n_cut=5000",
           "factors": sum(p.n_exc for p in probs), "seconds": tb, "evals_per_s": len(probs) / tb,
           "det_rotations_per_s": rot / tb, "probe_width": st[0]["probe_width"], "tiles": st[0]["batch_tiles"],
           "phase_ms": {"forward": st[0]["apply_ms"], "energy": st[0]["energy_ms"], "reverse": st[0]["reverse_ms"]},
           "jobs_cut": sum(x["cut"] > 0 for x in st)}
    for c in ctxs:
        c.close()
    # a sample of jobs: the batch vs one job at a time (the one-job path, host-driven cuts)
    sample = list(range(0, 256, 32))
    sp = jobs(sample)
    sc = [UCCContext(p) for p in sp]
    batch_run(sc, 1e-8, with_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch_run(sc, 1e-8, with_grad=True)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    for c in sc:
        c.gradient(eps=1e-8)
    torch.cuda.synchronize()
    t_s = time.perf_counter() - t0
    rot_s = sum(c.stats()["rotations"] for c in sc)
    for c in sc:
        c.close()
    # The sample batched alone is latency-bound (its longest job sets the time); the throughput
    # comparison sets the whole batch against the one-job path's rate on the sample, both per
    # evaluation and per det-rotation (the sample's jobs are smaller or larger than the average).
    out["sample_vs_one_by_one"] = {
        "jobs": sample, "batched_s": t_b, "one_by_one_s": t_s, "speedup": t_s / t_b,
        "one_by_one_evals_per_s": len(sample) / t_s, "one_by_one_det_rotations_per_s": rot_s / t_s,
        "throughput_speedup_evals": out["evals_per_s"] / (len(sample) / t_s),
        "throughput_speedup_det_rotations": out["det_rotations_per_s"] / (rot_s / t_s)}
    return out


# The paper's production truncation (Methods section), carried by every job of the batched workload.
BATCH_N_MAX, BATCH_N_CUT = 8000, 5000


def wide_leg(args):
    """A 72-spin-orbital problem shaped like the paper's CH2O/cc-pVDZ frozen-core case (36 spatial orbitals,
    12 electrons, the 5,000 largest doubles and all singles, the production cut N_MAX = 8,000 / N_CUT =
    5,000, eps = 1e-8): two-word determinant keys.  One full evaluation (apply, energy, adjoint)."""
    import torch
    from paper_2301_05726_gb300 import synth
    from paper_2301_05726_gb300.api import UCCContext
    p = synth.make_problem(7200, 36, 6, 6, 0.02, eps=1e-8, m_doubles=5000, name="72so_12e_md5000_cut8000")
    p.n_max, p.n_cut = BATCH_N_MAX, BATCH_N_CUT
    ctx = UCCContext(p)
    ctx.gradient()  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E, _ = ctx.gradient()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = ctx.stats()
    ctx.close()
    return {"workload": p.name, "n_so": p.n_so, "n_elec": p.n_elec, "n_factors": p.n_exc, "key_words": 2,
            "eval_s": dt, "det_rotations_per_s": st["rotations"] / dt, "n_det": st["n_det"], "cut": st["cut"]}


NCUT_SWEEP = (1000, 2000, 3000, 4000, 5000, 20000, 100000, 500000)


def ncut_leg(args):
    """Energy of fixed parameters as the cut grows (Results, discussion of Fig. 3c): a 64-spin-orbital,
    10-electron problem shaped like the paper's NH3/cc-pCVDZ study (the 5,000 largest doubles and all
    singles), evaluated at N_CUT = 1,000-5,000 with N_MAX = 8,000 (the optimisation-time settings), then
    with the wavefunction allowed to grow (N_MAX = 1.6 N_CUT).  One context; apply and energy per cut."""
    import torch
    from paper_2301_05726_gb300 import synth
    from paper_2301_05726_gb300.api import UCCContext
    p = synth.fig3_problem()
    ctx = UCCContext(p)
    ctx.apply()  # warm-up at the problem's own cut
    ctx.energy()
    rows = []
    for n_cut in NCUT_SWEEP:
        n_max = 8000 if n_cut <= 5000 else 8 * n_cut // 5
        ctx.set_options(n_max=n_max, n_cut=n_cut)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.apply()
        E, n2 = ctx.energy()
        dt = time.perf_counter() - t0
        st = ctx.stats()
        rows.append({"n_max": n_max, "n_cut": n_cut, "E": E, "norm2": n2, "n_det": st["n_det"], "cut": st["cut"],
                     "s": dt})
    ctx.close()
    return {"workload": p.name, "n_so": p.n_so, "n_elec": p.n_elec, "n_factors": p.n_exc, "eps": p.eps,
            "sweep": rows}


def run_ours(args, prob):
    import numpy as np
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
        st = ctx.stats()
        for k, v in st.items():
            tot[k] = tot.get(k, 0) + v
        tot["energy_route_last"] = st["energy_route"]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = sum(times) / len(times)
    n_steps = len(times)
    # Replicas: the slowest rank's step time, the work of all ranks.
    from paper_2301_05726_gb300.replicas import combine_step
    ms, rot_all = combine_step(ms, tot["rotations"] / n_steps, device=dev)
    value = rot_all / (ms / 1e3)
    g_dev = grad_dev.cpu().numpy()

    # End to end through the public API with host buffers (a few steps).
    e2e_times = []
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_theta(theta_host.numpy())
        E, g = ctx.gradient()
        grad_host.copy_(torch.from_numpy(g))
        e2e_times.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * sum(e2e_times) / len(e2e_times) if e2e_times else float("nan")

    # "Plain": per-theta central differences on the GPU (2K + 1 energy evaluations per gradient), timed on
    # a random subset of components through the public API and extrapolated.
    plain = None
    if args.plain_components > 0:
        plain, fd = plain_fd(ctx, prob, args.plain_components)
        plain["adjoint_gradient_s"] = ms / 1e3
        plain["speedup_adjoint_vs_plain"] = plain["extrapolated_gradient_s"] / (ms / 1e3)
    ctx.close()

    n1 = None
    if rank == 0 and not args.no_n1:
        n1 = n1_leg(args)
    batched = None
    if rank == 0 and not args.no_batch:
        batched = batch_leg(args)
    wide = None
    if rank == 0 and not args.no_wide:
        wide = wide_leg(args)
    ncut = None
    if rank == 0 and not args.no_ncut:
        ncut = ncut_leg(args)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    hbm, peak_kind = peaks()
    models = byte_models(tot)
    kernel_ms = {"k_forward": (tot["forward_kernel_ms"], tot["forward_launches"], tot["scanned"]),
                 "energy": (tot["energy_ms"], n_steps, 0),
                 "k_reverse": (tot["reverse_kernel_ms"], tot["reverse_launches"], tot["reverse_scanned"])}
    kernels = {m: {k: _roofline(k, models[m][k], t, n, hbm, peak_kind, sc) for k, (t, n, sc) in kernel_ms.items()}
               for m in models}
    dom = max(kernels["member"].values(), key=lambda r: r["total_ms"])
    roof = {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel", "peak_kind",
                                "avg_launch_ms")}
    roof["byte_model"] = "member (a rotation whose partner is absent is charged its own member only)"
    roof["frac_pair_model"] = kernels["pair"][dom["kernel"]]["frac"]
    cpu = None
    if not args.no_cpu_baseline:
        r, dt, desc = oracle_leg(prob, 3)
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, "host": host_info()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(prob), n_det=tot["n_det"] // n_steps,
                       l2="table larger than L2 + 256 MB flush per step",
                       parallelism="replicas" if world > 1 else "single"),
        "evals_per_s": world * 1e3 / ms,
        "apply_det_rotations_per_s": tot["rotations"] / (tot["apply_ms"] / 1e3) if tot["apply_ms"] > 0 else None,
        "phase_ms": {"forward": tot["apply_ms"] / n_steps, "energy": tot["energy_ms"] / n_steps,
                     "reverse_incl_recompute": tot["reverse_ms"] / n_steps,
                     "forward_kernels": tot["forward_kernel_ms"] / n_steps,
                     "reverse_kernels": tot["reverse_kernel_ms"] / n_steps,
                     "cuts": tot["cut_ms"] / n_steps, "other_rebuilds": tot["rebuild_ms"] / n_steps,
                     # the step minus the device time of every library kernel inside it (the factor
                     # steps, energy, cuts and rebuilds): host round trips and launch gaps
                     "host_gaps": (ms - (tot["forward_kernel_ms"] + tot["energy_ms"] + tot["reverse_kernel_ms"]
                                         + tot["cut_ms"] + tot["rebuild_ms"]) / n_steps)},
        "vs_plain": plain,
        "n1_40so": n1,
        "batched": batched,
        "wide_72so": wide,
        "ncut_sweep_64so": ncut,
        "e2e": {"value": rot_all / (e2e_ms / 1e3), "unit": UNIT, "steps": len(e2e_times),
                "h2d_bytes_per_step": FACTOR_BYTES * prob.n_exc, "d2h_bytes_per_step": 8 * prob.n_exc + 8},
        "gpu_launches": int(tot["kernel_launches"]),
        "counts_per_step": {k: int(tot[k] // n_steps) for k in (
            "rotations", "created", "dropped_new", "dropped_old", "cut", "scanned", "rebuilds", "tape_entries",
            "sigma_probes", "sigma_hits", "reverse_pairs", "reverse_scanned", "recompute_rotations",
            "forward_launches", "reverse_launches")},
        "roofline": roof,
        "kernels": {m: {k: {x: v[x] for x in ("achieved", "frac", "launches", "avg_launch_ms", "total_ms")}
                        for k, v in ks.items()} for m, ks in kernels.items()},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    prob = workload(args.workload)
    if args.n_max is not None:
        prob.n_max = args.n_max
        prob.n_cut = args.n_cut if args.n_cut is not None else args.n_max * 5 // 8
    if args.impl == "reference":
        run_reference(args, prob)
    else:
        run_ours(args, prob)


if __name__ == "__main__":
    main()
