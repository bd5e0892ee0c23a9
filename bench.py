#!/usr/bin/env python3
"""Throughput of the otVMC hot path: trajectory-steps per second on GB300.

A step is one trajectory step (App. C: two evaluations -- Metropolis sampling, local
estimators, observables, S and D, regularised solve -- and the predictor-corrector update)
of every trajectory of the batch, on synthetic quenches of the long-range transverse-field
Ising chain (64 spins, Jastrow P = 2080, 4096 samples, 256 trajectories per GPU, decay and
dephasing, dt = 0.005, midpoint) from the coherent state along +x.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank drives one GPU with its own 256 trajectories (global ids
rank*256 ...): weak scaling, no collective on the data path.  Rank 0 prints one JSON line.
--impl reference times the CPU FP64 oracle (the only reference this method has) on a
bounded sample of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trajectory-steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) of the Gram kernel per trajectory-evaluation, from an ncu capture of
# one launch of 32 trajectories (E4M3 O with its 33 extra rows: 279.5 MB read, 239.7 MB
# written), chain64_jastrow shape
GRAM_DRAM_BYTES_PER_TRAJ = (279.5e6 + 239.7e6) / 32
# nominal dense FP8 / BF16 tensor rate (4.5 / 2.25 PFLOP/s): the FP8 peak is the measured BF16
# peak times this
FP8_PER_BF16 = 2.0
# DRAM bytes (read + write) of the block-column update kernel per trajectory-evaluation, from an
# ncu capture of all 64 update launches of one evaluation of 32 trajectories (four groups of 8;
# 30.90 MB per launch with the factor in two FP16 pieces), chain64_jastrow shape
UPDATE_DRAM_BYTES_PER_TRAJ_EVAL = 30.90e6 * 64 / 32
# tensor-core products the Cholesky update and panel kernels issue per product of the method (the
# factor in two FP16 pieces h + m: h.h, h.m and m.h)
NPROD_CHOL = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chain64_jastrow")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--ntraj", type=int, default=None, help="trajectories per GPU (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-rbm-path", action="store_true")
    ap.add_argument("--no-rbm-workloads", action="store_true")
    ap.add_argument("--no-jastrow-workloads", action="store_true")
    ap.add_argument("--no-equal-error", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shape")
    ap.add_argument("--snr-full-size", action="store_true",
                    help="time the SNR regulariser at P = 2080 on 8 trajectories instead of 2")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(sm)}


def workload(args):
    import synth
    w = synth.WORKLOADS[args.workload]
    ntraj = args.ntraj or w.ntraj
    return w, ntraj


def build_model(w):
    import numpy as np
    import paper_2506_23928_gb300 as pkg
    from paper_2506_23928_gb300 import abi
    J = pkg.lattice_couplings(w.extent, w.J, w.alpha, w.kac, w.pbc)
    model = pkg.Model(J, w.h, np.full(w.n, w.kappa), np.full(w.n, w.gamma))
    if w.ansatz == "lj":
        return model, pkg.Ansatz(model, kind=abi.OTVMC_LJ, d=w.lj_d, pbc=w.pbc)
    return model, pkg.Ansatz(model)


def run_desc(w, ntraj, traj0, step0, n_steps, precision, seed, reg=None):
    from paper_2506_23928_gb300 import abi
    return abi.RunDesc(ntraj=ntraj, traj0=traj0, ns=w.ns, n_steps=n_steps, step0=step0, n_sweep=w.n_sweep, dt=w.dt,
                       scheme=abi.OTVMC_HEUN if w.scheme == "heun" else abi.OTVMC_MIDPOINT, precision=precision,
                       reg=abi.OTVMC_REG_SHIFT if reg is None else reg, eps=w.eps, snr_thresh=4.0, seed=seed,
                       measure_every=1, measure_final=0, use_graph=0)


def rbm_path(stream, fp64_value, peaks_, autotune=True):
    """The mixed batched RBM path on the chain64_rbm shape (N = 64, M = 128 hidden units,
    P = 8384 > ns: the T path), on a reduced batch that fits beside the main run: 16
    trajectories at ns = 2048 (the smallest of the workload's sample counts), hidden weights
    drawn N(0, 0.01) in real and imaginary part, a = b = 0, no observables in the timed steps.
    Timed with T formed from the factorised kernel (the default) and from materialised O on
    the tensor cores (split BF16); the second also gives the T-GEMM's tensor throughput.
    Reported next to the plain FP64 per-trajectory Jastrow path of the same GPU."""
    import numpy as np
    import torch
    import synth
    import paper_2506_23928_gb300 as pkg
    from paper_2506_23928_gb300 import abi
    from paper_2506_23928_gb300.abi import check
    w = synth.WORKLOADS["chain64_rbm"]
    T, ns, seed, steps = 16, 2048, 7, 2
    J = pkg.lattice_couplings(w.extent, w.J, w.alpha, w.kac, w.pbc)
    model = pkg.Model(J, w.h, np.full(w.n, w.kappa), np.full(w.n, w.gamma))
    ans = pkg.Ansatz(model, kind=abi.OTVMC_RBM, n_hidden=w.n_hidden)
    P, M = ans.P, w.n_hidden
    g = synth.rng(11)
    th0 = np.zeros((T, P), complex)
    th0[:, w.n + M:] = g.normal(0, 0.01, (T, w.n * M)) + 1j * g.normal(0, 0.01, (T, w.n * M))

    def desc(step0):
        return abi.RunDesc(ntraj=T, traj0=0, ns=ns, n_steps=1, step0=step0, n_sweep=w.n_sweep, dt=w.dt,
                           scheme=abi.OTVMC_MIDPOINT, precision=abi.OTVMC_PREC_MIXED, reg=abi.OTVMC_REG_SHIFT,
                           eps=w.eps, snr_thresh=4.0, seed=seed, measure_every=0, measure_final=0, use_graph=0)

    shape = {}

    def measure(mode, tune):
        check(abi.otvmc_ansatz_set_rbm_t_build(ans.handle, mode))
        theta = torch.from_numpy(th0.view(np.float64).copy()).cuda().reshape(T, P, 2)
        spins = torch.zeros((T, ns, 1), dtype=torch.int64, device="cuda")
        check(abi.otvmc_init_chains(ans.handle, T, 0, ns, seed, spins, stream))
        nb = abi.otvmc_run_workspace_bytes(ans.handle, desc(0))
        nbt = abi.otvmc_autotune_workspace_bytes(ans.handle, desc(0)) if tune else 0
        work = torch.zeros(max(nb, nbt), dtype=torch.uint8, device="cuda")
        check(abi.otvmc_run_trajectories(ans.handle, desc(0), theta, spins, None, work, nb, stream))
        torch.cuda.synchronize()
        if tune:
            st, pipes, groups, tms = abi.otvmc_autotune_run(ans.handle, desc(0), theta, spins, work, nbt, stream)
            check(st)
            shape.update({"source": "otvmc_autotune_run", "sub_batches": pipes,
                          "solver_groups": groups if groups else "built-in rule", "tuning_step_ms": tms})
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            check(abi.otvmc_run_trajectories(ans.handle, desc(1 + k), theta, spins, None, work, nb, stream))
        e1.record(stream)
        torch.cuda.synchronize()
        value = T * steps / (e0.elapsed_time(e1) / 1000.0)
        # one more step with per-class kernel timing (outside the timed steps)
        abi.otvmc_profile_enable(abi.OTVMC_PROFILE_SERIAL)
        check(abi.otvmc_run_trajectories(ans.handle, desc(1 + steps), theta, spins, None, work, nb, stream))
        torch.cuda.synchronize()
        prof = abi.profile_summary()
        abi.otvmc_profile_enable(0)
        del work
        return value, {k: v[0] for k, v in prof.items()}, nb

    v_f, st_f, nb_f = measure(abi.OTVMC_RBM_T_FACTORED, autotune)
    abi.otvmc_autotune_clear()
    v_m, st_m, nb_m = measure(abi.OTVMC_RBM_T_MATERIALISED, False)
    check(abi.otvmc_ansatz_set_rbm_t_build(ans.handle, abi.OTVMC_RBM_T_FACTORED))
    rows, K = 2 * ns, 2 * P
    # BF16 product flops of the split T-GEMM: six piece products of the upper triangle of the
    # embedded T (size 2 ns) over K = 2P, for T trajectories x 2 evaluations of the profiled step
    gemm_flops = 6 * 2.0 * K * rows * (rows + 1) / 2 * T * 2
    gram_ms = st_m.get("gram")
    t_gemm = None
    if gram_ms:
        ach = gemm_flops / (gram_ms / 1000.0) / 1e12
        t_gemm = {"bound": "tensor", "achieved": ach, "peak": peaks_["bf16_tflops_sustained"], "unit": "TFLOP/s",
                  "frac": ach / peaks_["bf16_tflops_sustained"], "ms_per_step": gram_ms}
    return {"value": v_f, "unit": METRIC,
            "precision": "mixed (FP32 ratios; T factorised: integer A, FP32 B, FP64 column sums; "
                         "tensor-core Cholesky + refinement)",
            "config": {"workload": w.name, "N": w.n, "M": M, "P": P, "ns": ns, "ntraj": T,
                       "solve": "T path (2 ns)", "steps_timed": steps, "observables": "off",
                       "workspace_bytes": nb_f},
            "launch_shape": shape or None,
            "stage_ms_per_step": st_f,
            "vs_fp64_jastrow_path": (v_f / fp64_value) if fp64_value else None,
            "materialised_T": {"value": v_m, "unit": METRIC, "workspace_bytes": nb_m, "stage_ms_per_step": st_m,
                               "t_gemm_roofline": t_gemm,
                               "vs_fp64_jastrow_path": (v_m / fp64_value) if fp64_value else None}}


def rbm_workload(name, stream, fp64_value, steps=3, warmup=2):
    """A whole RBM workload at its full size on the mixed path (T formed from the factorised
    kernel): chain64_rbm = 128 trajectories whose sample counts go round-robin over
    2048 / 4096 / 8192, timed as one batch per sample count run one after another
    (`sequential`) and as one grouped call that runs the three concurrently (`grouped`, the
    line's value when it fits in memory); square16_rbm = 64 trajectories at 4096 samples.  Hidden weights N(0, 0.01) in real
    and imaginary part, a = b = 0; observables off (the RBM's pair terms cost N^2 M per sample).
    Each step is every trajectory of the workload advanced once."""
    import numpy as np
    import torch
    import synth
    import paper_2506_23928_gb300 as pkg
    from paper_2506_23928_gb300 import abi
    from paper_2506_23928_gb300.abi import check
    w = synth.WORKLOADS[name]
    ns_mix = (2048, 4096, 8192) if name == "chain64_rbm" else (w.ns,)
    counts = [len(range(k, w.ntraj, len(ns_mix))) for k in range(len(ns_mix))]
    J = pkg.lattice_couplings(w.extent, w.J, w.alpha, w.kac, w.pbc)
    model = pkg.Model(J, w.h, np.full(w.n, w.kappa), np.full(w.n, w.gamma))
    ans = pkg.Ansatz(model, kind=abi.OTVMC_RBM, n_hidden=w.n_hidden)
    check(abi.otvmc_ansatz_set_rbm_t_build(ans.handle, abi.OTVMC_RBM_T_FACTORED))
    P, M, Wd = ans.P, w.n_hidden, (w.n + 63) // 64
    seed = 20261203

    def desc(k, step0):
        return abi.RunDesc(ntraj=counts[k], traj0=sum(counts[:k]), ns=ns_mix[k], n_steps=1, step0=step0,
                           n_sweep=w.n_sweep, dt=w.dt, scheme=abi.OTVMC_MIDPOINT, precision=abi.OTVMC_PREC_MIXED,
                           reg=abi.OTVMC_REG_SHIFT, eps=w.eps, snr_thresh=4.0, seed=seed, measure_every=0,
                           measure_final=0, use_graph=0)
    nb = max(abi.otvmc_run_workspace_bytes(ans.handle, desc(k, 0)) for k in range(len(ns_mix)))
    if nb == 0:
        return {"unavailable": "run descriptor rejected"}
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    g = synth.rng(13)
    batches = []
    for k, (T, ns) in enumerate(zip(counts, ns_mix)):
        th = np.zeros((T, P), complex)
        th[:, w.n + M:] = g.normal(0, 0.01, (T, w.n * M)) + 1j * g.normal(0, 0.01, (T, w.n * M))
        theta = torch.from_numpy(th.view(np.float64).copy()).cuda().reshape(T, P, 2)
        spins = torch.zeros((T, ns, Wd), dtype=torch.int64, device="cuda")
        check(abi.otvmc_init_chains(ans.handle, T, sum(counts[:k]), ns, seed, spins, stream))
        batches.append((theta, spins))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(ns_mix) + 1)] for _ in range(steps)]
    for i in range(warmup + steps):
        marks = ev[i - warmup] if i >= warmup else None
        if marks:
            marks[0].record(stream)
        for k in range(len(ns_mix)):
            theta, spins = batches[k]
            check(abi.otvmc_run_trajectories(ans.handle, desc(k, i), theta, spins, None, work, nb, stream))
            if marks:
                marks[k + 1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(m[0].elapsed_time(m[-1]) for m in ev)
    per_ns = {str(ns_mix[k]): {"ntraj": counts[k],
                               "ms_per_step": sum(m[k].elapsed_time(m[k + 1]) for m in ev) / steps}
              for k in range(len(ns_mix))}
    # one more step with per-class kernel timing (outside the timed steps)
    abi.otvmc_profile_enable(abi.OTVMC_PROFILE_SERIAL)
    for k in range(len(ns_mix)):
        theta, spins = batches[k]
        check(abi.otvmc_run_trajectories(ans.handle, desc(k, warmup + steps), theta, spins, None, work, nb, stream))
    torch.cuda.synchronize()
    stage = {c: v[0] for c, v in abi.profile_summary().items()}
    abi.otvmc_profile_enable(0)
    del work
    torch.cuda.empty_cache()
    seq_value = w.ntraj * steps / (total_ms / 1000.0)
    grouped = None
    if len(ns_mix) > 1:
        # the same step as one grouped call: the sample counts' batches concurrently on forked
        # streams (the largest N_s at the highest stream priority), each in its own workspace
        s0 = warmup + steps + 1
        descs = lambda i: [desc(k, s0 + i) for k in range(len(ns_mix))]
        nbg = abi.otvmc_run_grouped_workspace_bytes(ans.handle, descs(0))
        free, _ = torch.cuda.mem_get_info()
        if nbg and nbg < free - (4 << 30):
            workg = torch.zeros(nbg, dtype=torch.uint8, device="cuda")
            gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for i in range(warmup + steps):
                if i >= warmup:
                    gev[i - warmup][0].record(stream)
                check(abi.otvmc_run_trajectories_grouped(ans.handle, descs(i), [b[0] for b in batches],
                                                         [b[1] for b in batches], [None] * len(ns_mix), workg, nbg,
                                                         stream))
                if i >= warmup:
                    gev[i - warmup][1].record(stream)
                torch.cuda.synchronize()
            gms = sum(a.elapsed_time(b) for a, b in gev) / steps
            grouped = {"value": w.ntraj / (gms / 1000.0), "ms_per_step": gms, "workspace_bytes": nbg,
                       "call": "otvmc_run_trajectories_grouped, one group per N_s"}
            del workg
        else:
            grouped = {"unavailable": f"grouped workspace {nbg} bytes exceeds the free memory {free}"}
        torch.cuda.empty_cache()
    del batches
    torch.cuda.empty_cache()
    value = grouped["value"] if grouped and "value" in grouped else seq_value
    return {"value": value, "unit": METRIC,
            "ms_per_step": (grouped["ms_per_step"] if grouped and "value" in grouped else total_ms / steps),
            "steps": steps, "warmup": warmup,
            "precision": "mixed (FP32 ratios; T factorised; tensor-core Cholesky + refinement)",
            "config": {"workload": name, "N": w.n, "M": M, "P": P, "ntraj": w.ntraj, "ns": list(ns_mix),
                       "solve": "T path (2 ns)", "observables": "off", "workspace_bytes": nb,
                       "launch": "one grouped call per step" if grouped and "value" in grouped
                       else "one batch per sample count, one after another"},
            "sequential": {"value": seq_value, "ms_per_step": total_ms / steps, "per_ns": per_ns},
            "grouped": grouped, "stage_ms_per_step": stage,
            "vs_fp64_jastrow_path": (value / fp64_value) if fp64_value else None}


def jastrow_workload(name, stream, precision, steps=3, warmup=2, reg=None, ntraj=None):
    """A whole Jastrow workload at its full size: every trajectory advanced by one trajectory
    step per step (observables of the predictor samples included, as in the headline step), in
    waves of contiguous trajectory ids by device-memory footprint when the batch's workspace
    exceeds the free memory (one workspace of the largest wave, reused; the waves run one after
    another).  CUDA events around each step.  reg: the regulariser (diagonal shift by default,
    or the SNR filter); ntraj: fewer trajectories than the workload's, for a costly variant."""
    import numpy as np
    import torch
    import synth
    from paper_2506_23928_gb300 import abi, waves as wv
    from paper_2506_23928_gb300.abi import check
    w = synth.WORKLOADS[name] if name in synth.WORKLOADS else synth.PAPER_WORKLOADS[name]
    model, ans = build_model(w)
    P, T, Wd = ans.P, (ntraj or w.ntraj), (w.n + 63) // 64
    seed = 20261204

    def desc(o, c, step0):
        return run_desc(w, c, o, step0, 1, precision, seed, reg)
    torch.cuda.empty_cache()
    free = torch.cuda.mem_get_info()[0]
    state = T * (P * 16 + w.ns * Wd * 8 + 9 * 8)
    budget = int(0.85 * free) - state
    plan = wv.plan(T, lambda c: abi.otvmc_run_workspace_bytes(ans.handle, desc(0, c, 0)), budget)
    nb = max(abi.otvmc_run_workspace_bytes(ans.handle, desc(o, c, 0)) for o, c in plan)
    work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    theta = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    spins = torch.zeros((T, w.ns, Wd), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(ans.handle, T, 0, w.ns, seed, spins, stream))
    cmax = max(c for _, c in plan)
    mom = torch.zeros((1, cmax, 9), dtype=torch.float64, device="cuda")
    per = []
    for i in range(warmup + steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for o, c in plan:
            check(abi.otvmc_run_trajectories(ans.handle, desc(o, c, i), theta[o:o + c], spins[o:o + c], mom, work,
                                             nb, stream))
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            per.append(e0.elapsed_time(e1))
    total_ms = sum(per)
    del work, theta, spins
    torch.cuda.empty_cache()
    return {"value": T * steps / (total_ms / 1000.0), "unit": METRIC, "ms_per_step": total_ms / steps,
            "ms_per_step_min": min(per), "ms_per_step_max": max(per), "steps": steps, "warmup": warmup,
            "precision": "mixed" if precision == abi.OTVMC_PREC_MIXED else "fp64",
            "config": {"workload": name, "N": w.n, "P": P, "ns": w.ns, "ntraj": T, "dt": w.dt, "scheme": w.scheme,
                       "eps": w.eps, "ansatz": "LJPH%d" % w.lj_d if w.ansatz == "lj" else "Jastrow",
                       "regulariser": "snr (threshold 4)" if reg == abi.OTVMC_REG_SNR else "diagonal shift",
                       "waves": [list(x) for x in plan], "workspace_bytes": nb}}


GOLDEN_CHAIN8 = os.path.join(ROOT, "tests", "golden", "chain8_lindblad.txt")


def equal_error_chain8(stream, T=256):
    """Throughput at a measured observable error: the 8-spin workload (h = 1, decay 0.1, Heun,
    dt = 0.01) to t = 1 with T trajectories, (a) on the plain FP64 Jastrow path run one
    trajectory per call, (b) on the mixed batched RBM path (16 hidden units, weights drawn
    N(0, 0.05^2), shift 1e-3) in one batch.  Each ensemble's magnetisation at t = 0.1 .. 1 is
    compared with the exact Lindblad values stored in tests/golden/chain8_lindblad.txt; the
    error is the largest |M - M_exact| over those times (standard error beside it).  A
    trajectory whose recorded magnetisation leaves the physical range by far (|M_a| > 2) has run
    into a nearly nodal state of its ansatz; it is counted (`trajectories_out_of_range`) and
    left out of that ensemble's mean."""
    import numpy as np
    import torch
    import synth
    import paper_2506_23928_gb300 as pkg
    from paper_2506_23928_gb300 import abi
    from paper_2506_23928_gb300.abi import check
    exact = np.loadtxt(GOLDEN_CHAIN8)
    w = synth.WORKLOADS["chain8_jastrow"]
    steps, every, seed = 100, 10, 11
    model, jas = build_model(w)
    M_h = 16
    rbm = pkg.Ansatz(model, kind=abi.OTVMC_RBM, n_hidden=M_h)

    def run(ans, P, th0, per_call, precision, eps):
        nm = None
        moms, ms = [], 0.0
        for t0 in range(0, T, per_call):
            c = min(per_call, T - t0)
            desc = abi.RunDesc(ntraj=c, traj0=t0, ns=w.ns, n_steps=steps, step0=0, n_sweep=w.n_sweep, dt=w.dt,
                               scheme=abi.OTVMC_HEUN, precision=precision, reg=abi.OTVMC_REG_SHIFT, eps=eps,
                               snr_thresh=4.0, seed=seed, measure_every=every, measure_final=1, use_graph=0)
            nm = abi.otvmc_run_n_meas(desc)
            theta = torch.from_numpy(np.tile(th0, (c, 1)).view(np.float64).copy()).cuda().reshape(c, P, 2)
            spins = torch.zeros((c, w.ns, 1), dtype=torch.int64, device="cuda")
            check(abi.otvmc_init_chains(ans.handle, c, t0, w.ns, seed, spins, stream))
            nb = abi.otvmc_run_workspace_bytes(ans.handle, desc)
            work = torch.zeros(nb, dtype=torch.uint8, device="cuda")
            mom = torch.zeros((nm, c, 9), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            check(abi.otvmc_run_trajectories(ans.handle, desc, theta, spins, mom, work, nb, stream))
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            moms.append(mom.cpu().numpy())
        mom = np.concatenate(moms, axis=1)
        m = mom[1:, :, :3]                                   # t = 0.1 .. 1.0
        out = (np.abs(m) > 2.0).any(axis=(0, 2))
        m = m[:, ~out]
        M = m.mean(axis=1)
        se = m.std(axis=1, ddof=1) / np.sqrt(m.shape[1])
        err = np.abs(M - exact[1:, 1:4])
        return {"value": T * steps / (ms / 1000.0), "unit": METRIC, "max_abs_dM": float(err.max()),
                "mean_abs_dM_t06_t1": float(err[5:].max(axis=1).mean()), "standard_error_max": float(se.max()),
                "ntraj": T, "trajectories_out_of_range": int(out.sum()), "trajectories_per_call": per_call}

    g = synth.rng(17)
    th_r = np.zeros(rbm.P, complex)
    th_r[w.n + M_h:] = g.normal(0, 0.05, w.n * M_h) + 1j * g.normal(0, 0.05, w.n * M_h)
    j = run(jas, jas.P, np.zeros(jas.P, complex), 1, abi.OTVMC_PREC_FP64, w.eps)
    r = run(rbm, rbm.P, th_r, T, abi.OTVMC_PREC_MIXED, 1e-3)
    return {"workload": "chain8_jastrow (N = 8, h = 1, kappa = 0.1, Heun, dt = 0.01, to t = 1)",
            "jastrow_fp64_per_trajectory": j, "rbm_mixed_batched": r,
            "rbm_error_not_larger": r["max_abs_dM"] <= j["max_abs_dM"],
            "speedup_at_no_larger_error": r["value"] / j["value"]}


def cpu_baseline(w, steps=1):
    """The oracle as it stands: one trajectory, `steps` trajectory steps, on the host cores."""
    import numpy as np
    from oracle.model import Model, couplings
    from oracle.ansatz import Jastrow
    from oracle import trajectories as tr
    m = Model(J=couplings(w.extent, w.J, w.alpha, kac=w.kac, pbc=w.pbc), h=w.h, kappa=w.kappa, gamma=w.gamma)
    t0 = time.perf_counter()
    tr.run_mc(m, Jastrow(w.n), 1, w.ns, steps, w.dt, 1, w.scheme, n_sweep=w.n_sweep, eps=w.eps)
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max((i.get("num_threads", 1) for i in threadpool_info()), default=cores)
    except Exception:
        pass
    return {"value": steps / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"1 trajectory x {steps} step(s) of {w.name} (N={w.n}, P={w.n * (w.n + 1) // 2}, "
                      f"ns={w.ns}), numpy FP64", "seconds": dt}


def run_reference(args):
    w, ntraj = workload(args)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(w, 1)
    t0 = time.perf_counter()
    res = None
    for _ in range(args.steps):
        res = cpu_baseline(w, 1)
    el = time.perf_counter() - t0
    value = args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N": w.n, "P": w.n * (w.n + 1) // 2, "ns": w.ns, "ntraj_per_step": 1,
                       "note": "each step is 1 trajectory-step of 1 trajectory (bounded CPU sample)"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"]},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2506_23928_gb300 import abi, build
    from paper_2506_23928_gb300.abi import check

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    prec = abi.OTVMC_PREC_MIXED if args.precision == "mixed" else abi.OTVMC_PREC_FP64
    w, T = workload(args)
    model, ans = build_model(w)
    P = ans.P
    seed = 20260603
    from paper_2506_23928_gb300.sharding import shard
    traj0, _ = shard(T * world, rank, world)   # weak scaling: T trajectories per rank
    W = (w.n + 63) // 64
    stream = torch.cuda.current_stream()

    theta = torch.zeros((T, P, 2), dtype=torch.float64, device="cuda")
    spins = torch.zeros((T, w.ns, W), dtype=torch.int64, device="cuda")
    check(abi.otvmc_init_chains(ans.handle, T, traj0, w.ns, seed, spins, stream))
    d1 = run_desc(w, T, traj0, 0, 1, prec, seed)
    nb = abi.otvmc_run_workspace_bytes(ans.handle, d1)
    nbh = abi.otvmc_run_host_workspace_bytes(ans.handle, d1)
    nbt = abi.otvmc_autotune_workspace_bytes(ans.handle, d1)
    work = torch.zeros(max(nb, nbh, nbt), dtype=torch.uint8, device="cuda")
    mom = torch.zeros((1, T, 9), dtype=torch.float64, device="cuda")

    def step(i):
        d = run_desc(w, T, traj0, i, 1, prec, seed)
        check(abi.otvmc_run_trajectories(ans.handle, d, theta, spins, mom, work, nb, stream))

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    # launch shape (sub-batches, solver groups) picked by the library's autotuner on this batch,
    # from a copy of the warmed-up state; no result depends on it
    launch_shape = {"source": "built-in"}
    if not args.no_autotune:
        st, pipes, groups, tms = abi.otvmc_autotune_run(ans.handle, d1, theta, spins, work, max(nb, nbh, nbt), stream)
        check(st)
        launch_shape = {"source": "otvmc_autotune_run", "sub_batches": pipes,
                        "solver_groups": groups if groups else "built-in rule", "tuning_step_ms": tms}

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    l0 = abi.otvmc_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = abi.otvmc_launch_count() - l0
    el_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks else None
    t = torch.tensor([el_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    el_ms = float(t.item())
    total_units = T * world * args.steps
    value = total_units / (el_ms / 1000.0)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        th_h = theta.cpu().pin_memory()
        sp_h = spins.cpu().pin_memory()
        mo_h = torch.zeros((1, T, 9), dtype=torch.float64).pin_memory()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            d = run_desc(w, T, traj0, args.warmup + args.steps + k, 1, prec, seed)
            check(abi.otvmc_run_trajectories_host(ans.handle, d, th_h, sp_h, mo_h, work, nbh, stream))
        torch.cuda.synchronize()
        e2e_s = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(e2e_s, op=dist.ReduceOp.MAX)
        h2d = th_h.numel() * 8 + sp_h.numel() * 8
        d2h = h2d + mo_h.numel() * 8
        e2e = {"value": total_units / float(e2e_s.item()), "unit": METRIC, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # per-kernel durations: the same steps once more, outside the timed region, with every launch
    # bracketed by CUDA events on its own stream and the solver's trajectory groups run one after
    # another (in the timed steps they overlap on forked streams, where a launch's event time
    # would include the time it shares the GPU with the other groups' kernels)
    prof_steps = max(1, min(args.steps, 2))
    abi.otvmc_profile_enable(abi.OTVMC_PROFILE_SERIAL)
    for k in range(prof_steps):
        step(args.warmup + 2 * args.steps + k)
    torch.cuda.synchronize()
    prof = abi.profile_summary()
    abi.otvmc_profile_enable(abi.OTVMC_PROFILE_OFF)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    stage_ms = {k: v[0] / prof_steps for k, v in prof.items()}
    dominant = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None
    ns = w.ns
    roof = {}
    evals = 2 * prof_steps                                            # evaluations per trajectory in the profiled steps
    NBK = 128
    jbs = list(range(0, P, NBK))
    # algorithmic work per trajectory-evaluation of each kernel class
    work = {
        # useful tensor flops of G = O^T O (upper triangle incl. diagonal), E4M3 operands
        "gram": ("tensor_fp8", 2.0 * ns * P * (P + 1) / 2),
        # bytes of the Cholesky block-column updates C = A - L L^T: the two FP16 pieces of
        # L[i >= jb, k < jb] read once, the Gram counts of the block column read (FP32) and C
        # written below the diagonal tile (two FP16 pieces).  Its arithmetic intensity, 2 x 128
        # method flops per 4 bytes of L, is far below the GPU's flop-to-byte ratio: HBM-bound
        # (the method's flops and the issued FP16 products are reported beside it).  The
        # diagonal tile of C is written in FP32.
        "chol_update": ("hbm", sum(4.0 * (P - jb) * jb + 4.0 * NBK * (P - jb) + 4.0 * NBK * max(0, P - jb - NBK)
                                   + 4.0 * NBK * NBK for jb in jbs if jb > 0)),
        # flops of the method in the panel products X = C L_dd^-T (three FP16 piece products issued each)
        "chol_trsm": ("tensor", 2.0 * sum(max(0, P - jb - NBK) * NBK * NBK for jb in jbs)),
        # bytes the triangular substitutions must read: the lower factor (FP32) once for the
        # backward pass after the factorization (its forward pass is fused into it) and twice
        # for the correction of the refinement step
        "solve": ("hbm", 3 * 4.0 * P * P / 2),
        # bytes of the refinement residual: the upper triangle of the Gram counts (FP32) once
        "chol_resid": ("hbm", 4.0 * P * (P + 1) / 2),
    }
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    for cls, (bound, per_eval) in work.items():
        if cls not in prof:
            continue
        ms, cnt = prof[cls]
        total = per_eval * T * evals
        if bound == "tensor_fp8":
            bound = "tensor"
            ach, peak, unit = total / (ms / 1000.0) / 1e12, FP8_PER_BF16 * pk["bf16_tflops_sustained"], "TFLOP/s"
            kind = f"fp8 = 2 x bf16 sustained ({pk_kind}; nominal dense ratio 4.5 / 2.25)"
        elif bound == "tensor":
            ach, peak, unit = total / (ms / 1000.0) / 1e12, pk["bf16_tflops_sustained"], "TFLOP/s"
            kind = f"bf16 sustained, {pk_kind}"
        elif bound == "alu":
            ach, peak, unit = total / (ms / 1000.0) / 1e12, fp32_peak, "TFLOP/s"
            kind = "fp32 SIMT: 152 SMs x 128 lanes x 2 x max SM clock (derived)"
        else:
            ach, peak, unit = total / (ms / 1000.0) / 1e9, pk["hbm_gbs"], "GB/s"
            kind = f"HBM copy, {pk_kind}"
        # DRAM bytes per launch from the ncu capture, scaled by the trajectories one launch covers
        per_te = {"gram": GRAM_DRAM_BYTES_PER_TRAJ, "chol_update": UPDATE_DRAM_BYTES_PER_TRAJ_EVAL}.get(cls)
        traffic = per_te * T * evals / cnt if (per_te and w.name == "chain64_jastrow") else None
        roof[cls] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                     "traffic": traffic, "peak_kind": kind, "launches": cnt, "ms_total": ms}
        if cls in ("chol_update", "chol_trsm"):
            # the method's flops (one product per FP32-level product) and what the tensor pipe
            # executes: three FP16 piece products (h.h, h.m, m.h) per method product; FP16 runs at
            # the BF16 rate, so the BF16 peak is its peak too
            fl = {"chol_update": 2.0 * sum((P - jb) * NBK * jb for jb in jbs if jb > 0)}.get(cls)
            mt = (fl * T * evals / (ms / 1000.0) / 1e12) if fl else ach
            tp = pk["bf16_tflops_sustained"]
            roof[cls]["method_tflops"] = mt
            roof[cls]["method_frac_of_bf16"] = mt / tp
            roof[cls]["issued_fp16_tflops"] = NPROD_CHOL * mt
            roof[cls]["issued_fp16_frac"] = NPROD_CHOL * mt / tp
    # the dominant kernel class among those with a roofline (largest total event time)
    dominant = max(roof, key=lambda k: roof[k]["ms_total"]) if roof else dominant
    rl = roof.get(dominant)

    fp64 = None
    if not args.no_fp64_path and prec == abi.OTVMC_PREC_MIXED:
        # the plain FP64 path (FP64 O, FP64 S, FP64 Cholesky) on a reduced slice of the batch
        Tf = 2
        thf = torch.zeros((Tf, P, 2), dtype=torch.float64, device="cuda")
        spf = spins[:Tf].clone()
        df = run_desc(w, Tf, 0, 0, 1, abi.OTVMC_PREC_FP64, seed)
        nbf = abi.otvmc_run_workspace_bytes(ans.handle, df)
        wf = torch.zeros(nbf, dtype=torch.uint8, device="cuda")
        mf = torch.zeros((1, Tf, 9), dtype=torch.float64, device="cuda")
        check(abi.otvmc_run_trajectories(ans.handle, df, thf, spf, mf, wf, nbf, stream))
        torch.cuda.synchronize()
        n_fp64 = 3
        per = []
        for k in range(n_fp64):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            df = run_desc(w, Tf, 0, 1 + k, 1, abi.OTVMC_PREC_FP64, seed)
            e0.record(stream)
            check(abi.otvmc_run_trajectories(ans.handle, df, thf, spf, mf, wf, nbf, stream))
            e1.record(stream)
            torch.cuda.synchronize()
            per.append(e0.elapsed_time(e1))
        med = statistics.median(per)
        # FP64 roofline of this path: its dominant work, per evaluation, is the S build
        # (ns P (P + 1) multiply-adds) and the Cholesky (P^3 / 3), against the FP64 rate that a
        # library DGEMM (cuBLAS through torch, 8192^3) reaches on this GPU
        fl = 2 * (2.0 * ns * P * (P + 1) / 2 + P ** 3 / 3.0)   # flops per trajectory-step
        a64 = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
        b64 = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
        torch.matmul(a64, b64)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        for _ in range(3):
            torch.matmul(a64, b64)
        g1.record()
        torch.cuda.synchronize()
        dgemm = 3 * 2.0 * 8192 ** 3 / (g0.elapsed_time(g1) / 1000.0) / 1e12
        del a64, b64
        ach = fl * Tf / (med / 1000.0) / 1e12
        fp64 = {"value": Tf / (med / 1000.0), "unit": METRIC, "ms_per_step_median": med,
                "ms_per_step_min": min(per), "ms_per_step_max": max(per), "steps": n_fp64, "warmup": 1,
                "sample": f"{Tf} trajectories x {n_fp64} steps (CUDA events, median) after 1 warm-up step, "
                          "same workload, FP64 O / S / Cholesky",
                "roofline": {"bound": "fp64", "achieved": ach, "peak": dgemm, "unit": "TFLOP/s", "frac": ach / dgemm,
                             "peak_kind": "cuBLAS DGEMM 8192^3 through torch, measured in this run",
                             "work": "S build ns P(P+1) + Cholesky P^3/3 multiply-adds per evaluation"}}
        del wf

    rbm = None
    if not args.no_rbm_path and world == 1:
        rbm = rbm_path(stream, fp64["value"] if fp64 else None, pk, not args.no_autotune)

    rbm_full = None
    if not args.no_rbm_workloads and world == 1:
        rbm_full = {name: rbm_workload(name, stream, fp64["value"] if fp64 else None)
                    for name in ("chain64_rbm", "square16_rbm")}

    jw = None
    if not args.no_jastrow_workloads and world == 1:
        del work
        torch.cuda.empty_cache()
        jw = {"chain8_jastrow": jastrow_workload("chain8_jastrow", stream, abi.OTVMC_PREC_FP64, steps=20, warmup=3),
              "chain8_jastrow_mixed": jastrow_workload("chain8_jastrow", stream, abi.OTVMC_PREC_MIXED, steps=20,
                                                       warmup=3),
              "square10_jastrow": jastrow_workload("square10_jastrow", stream, abi.OTVMC_PREC_MIXED),
              "ring100_ljph1": jastrow_workload("ring100_ljph1", stream, abi.OTVMC_PREC_MIXED),
              "ring160_ljph1": jastrow_workload("ring160_ljph1", stream, abi.OTVMC_PREC_MIXED),
              # the paper's own regulariser (the SNR filter, threshold 4) on its Fig. 3 / Fig. 2 setups
              "ring100_ljph1_snr": jastrow_workload("ring100_ljph1", stream, abi.OTVMC_PREC_MIXED, steps=2, warmup=1,
                                                    reg=abi.OTVMC_REG_SNR),
              "ring160_ljph1_snr": jastrow_workload("ring160_ljph1", stream, abi.OTVMC_PREC_MIXED, steps=2, warmup=1,
                                                    reg=abi.OTVMC_REG_SNR)}
        # the SNR filter at the benchmark's P = 2080 (O(P^3) FP64 per trajectory, one CTA each): 2
        # trajectories by default (about a minute), 8 with --snr-full-size
        jw["chain64_jastrow_snr"] = jastrow_workload("chain64_jastrow", stream, abi.OTVMC_PREC_MIXED, steps=1,
                                                     warmup=0, reg=abi.OTVMC_REG_SNR,
                                                     ntraj=8 if args.snr_full_size else 2)

    eq = None
    if not args.no_equal_error and world == 1:
        eq = equal_error_chain8(stream)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w, 1)
        cpu.pop("seconds", None)

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "mixed: e4m3 Gram (exact), fp16-piece tensor-core Cholesky + fp64 refinement, int64/fp64 fields"
            if prec == abi.OTVMC_PREC_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "N": w.n, "P": P, "ns": ns, "ntraj_per_gpu": T, "dt": w.dt,
                       "scheme": w.scheme, "n_sweep": w.n_sweep, "eps": w.eps, "precision": args.precision,
                       "parallelism": f"trajectories sharded over {world} GPU(s)",
                       "l2": "no flush: per-step working set (O, G, L of 256 trajectories, ~14 GB) exceeds L2"},
            "roofline": rl, "roofline_by_kernel": roof, "dominant_kernel": dominant,
            "kernel_timing": f"CUDA events per launch over {prof_steps} more step(s) after the timed region, "
                             "solver trajectory groups serialised (launch durations not shared)",
            "stage_ms_per_step": stage_ms, "launch_shape": launch_shape, "cpu_baseline": cpu, "fp64_path": fp64, "rbm_mixed_path": rbm,
            "rbm_workloads": rbm_full, "jastrow_workloads": jw, "equal_error": eq,
            "clocks": clk, "e2e": e2e,
            "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
