"""Benchmark of the particle BP update (predict + update per step) on GB300.

Default workload: 64 potential features (LoS + 63 surfaces, held fixed: no birth,
no pruning), 100000 particles per belief, J = 4 PAs with 4 x 4 URAs and 10
frequency bins (Nz = 160), 20 dB SNR, visibility 0.8, 200 spurious paths per step.
Metric: (particle, PA) updates per second = P * J / step time (each step updates
every particle of every belief against every PA's observation).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

One JSON line is printed by rank 0.  N > 1 runs N independent replicas (one per
GPU, weak scaling; the method has no cross-replica exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_19723_gb300 import workload as W  # noqa: E402

METRIC = "particle-measurement updates/sec and steps/sec at matched OSPA vs plain FP32 GPU"
# The paper's own figure for its Experiment 1 shape (P = 30000, J = 4, Nz = 160, ~5 PFs):
# 420 ms per step on an RTX PRO 4000 Blackwell, i.e. 30000 * 4 / 0.42 updates/s.  Context
# for the matching workload only; other workloads have no published number.
PAPER_UPDATES_PER_S = {"paper_exp1": 30000 * 4 / 0.420}
UNIT = "(particle, PA) updates/s"
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25   # GB300 dense FP64, nominal


def kappa_flops(P, S, J, Nz):
    """Algorithmic FP32 flops of one launch of the PF likelihood kernel: per (p, s, j)
    two passes over Nz elements against the S-1 (eigen-whitened, orthogonal) basis
    columns plus the residual column, 8 flops per complex multiply-add, the steering
    vector and residual element work (40 per element) and the O(S) amplitude sums."""
    per = 8 * Nz * S + 8 * Nz * (S - 1) + 40 * Nz + 16 * (S - 1)
    return float(P) * S * J * per


def kappa_tc_used(g, S, S_max):
    """Whether the PF likelihood runs on the tensor cores (k_kappa_tc) with its built-in
    tiles: a shape the kernel takes (autotune.tensor_core_shape) and a column bucket equal
    to the basis stride (S > 32 at stride 64, S > 24 at stride 32)."""
    from paper_2604_19723_gb300 import autotune
    if not autotune.tensor_core_shape(g, S_max):
        return False
    width = autotune.basis_stride(S_max)
    return S > (32 if width == 64 else 24)


def kappa_contraction_flops(P, S, J, Nz):
    """The two contractions of the PF likelihood (psi^H V over the S-1 basis columns and
    r0, then V conj(h) over the S-1 basis columns), 8 flops per complex multiply-add."""
    return float(P) * S * J * (8 * Nz * S + 8 * Nz * (S - 1))


def iota_flops(P, S, J, Nf, My, Mz):
    """Algorithmic flops of one launch of the MT likelihood kernel, per (p, j): the
    Kronecker-factored Gram (S(S+1)/2 entries, Nf + My + Mz complex multiply-adds and
    two complex products each), g = Psi^H z, the right-hand side, the Cholesky
    factorisation (S^3/6 complex multiply-adds), two triangular solves and the
    element-wise residual (three complex products and one accumulation per (s, k)).
    Counted as plain FP32 flops; the kernel runs them in float-float arithmetic."""
    Nz = Nf * My * Mz
    per = (S * (S + 1) / 2 * 8 * (Nf + My + Mz + 2) + 8 * S * Nf * (My * Mz + My + 1) + 8 * S * S
           + 8 * S ** 3 / 6 + 8 * S * S + 20 * Nz * S)
    return float(P) * J * per


# DRAM bytes of one launch of a kernel (dram__bytes_read.sum + dram__bytes_write.sum), from
# a one-pass ncu capture of that kernel alone (-c 1) running the bench command itself at
# full size.  The kernels' traffic does not scale with the particles (operand tiles read
# once per PF and then served from L2), so a record applies only to the workload and
# particle count it was taken at, and only while the kernel sources hash to the recorded
# value.
TRAFFIC_RECORDS = {
    "k_kappa_tc": {"workload": "scale_64x100k", "P": 100000, "bytes": 873119232 + 50664448,
                   "sources_sha256": "1110bf0b1cfc98075cd47b06617919570f7d65d3df893ff6bb438e748e463a97",
                   "how": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                          "--clock-control none -k regex:^k_kappa_tc$ -c 1 python bench.py --steps 2 "
                          "--warmup 1 --no-matched --no-cpu-baseline"},
}
KERNEL_SOURCES = ("paper_2604_19723_gb300/csrc/k_like.cu", "paper_2604_19723_gb300/csrc/bp_kernels.cuh",
                  "paper_2604_19723_gb300/csrc/bp_internal.cuh", "paper_2604_19723_gb300/csrc/tc_sm100.cuh")


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_for(kernel, workload, P):
    rec = TRAFFIC_RECORDS.get(kernel)
    if not rec or rec["workload"] != workload or rec["P"] != P or rec["sources_sha256"] != kernel_sources_sha256():
        return None
    return rec["bytes"]


def reduce_max(x, world, device):
    """Max of a scalar over the ranks of the process group (a no-op for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([t.strip() for t in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def make_inputs(name, steps, seed_offset=0):
    wl = W.workload(name)
    g, prm = wl["geom"], wl["params"]
    scn = W.make_scenario(g, prm, N=steps + 1, K=wl["K"], seed=wl["seed"] + seed_offset, snr_db=wl["snr_db"],
                          visibility=wl["visibility"], clutter_mean=wl["clutter_mean"])
    return wl, g, prm, scn


def sm_count(dev=0):
    """Streaming multiprocessors of the device (from its attributes)."""
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def host_cpu():
    """CPU model name and the number of online cores of this host."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model name", "CPU part") and v.strip():
                    model = v.strip()
                    if k.strip() != "CPU part":
                        break
    except OSError:
        pass
    if model is None or model.startswith("0x"):
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count() or 1}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(wl, g, prm, scn, sample_P, z_host):
    """The FP64 oracle (as it stands) on the host cores: one predict + update of a
    bounded particle sample of the same workload (same S, J, Nz)."""
    from oracle import beliefs, messages_woodbury, model
    S = wl["fixed_S"] or (wl["K"] + 1)
    st = W.state_near_truth(scn, P=sample_P, S=S, n=0, seed=wl["seed"] + 7, eta_true=float(np.mean(np.abs(z_host[0]) ** 2)) / 100,
                            pos_std=0.01, sfv_std=0.01)
    t0 = time.perf_counter()
    pred = model.predict(st, prm, g.J, seed=wl["seed"], S_max=wl["fixed_S"] or wl["S_max"])
    msg = messages_woodbury.update_messages(pred, prm, g, z_host[0].astype(np.complex128))
    beliefs.beliefs(pred, msg)
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return {"value": sample_P * g.J / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one predict+update of {sample_P} particles x S={S} x J={g.J} x Nz={g.Nz} "
                      f"(FP64 Woodbury-mode oracle, {dt:.2f} s)", **host_cpu()}


def run_reference(args, rank):
    """Reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    if args.workload == "batched":
        sc, scns = batched_inputs(args, 2)
        vals = []
        for i in range(args.warmup + args.steps):
            v, t = batched_oracle_sample(sc, scns, args.ref_particles, 2)
            if i >= args.warmup:
                vals.append(v)
        value = float(np.mean(vals))
        cores = os.cpu_count() or 1
        smp = f"one predict+update of {args.ref_particles} particles of each of the first 2 scenarios per step"
        print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f64", "data": "synthetic", "impl": "reference",
                          "config": {"workload": "batched", "scenarios": len(sc),
                                     "parallelism": "oracle on the host cores", "sample": smp},
                          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": smp,
                                           **host_cpu()},
                          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    wl, g, prm, scn = make_inputs(args.workload, args.warmup + args.steps)
    from oracle import synth
    eta = synth.noise_variance(scn)
    zs = [synth.observe(scn, n, eta, 17) for n in range(1, args.warmup + args.steps + 1)]
    from oracle import beliefs, messages_woodbury, model
    S = wl["fixed_S"] or (wl["K"] + 1)
    Ps = args.ref_particles
    st = W.state_near_truth(scn, P=Ps, S=S, n=0, seed=wl["seed"] + 7, eta_true=eta, pos_std=0.01, sfv_std=0.01)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pred = model.predict(st, prm, g.J, seed=wl["seed"], S_max=wl["fixed_S"] or wl["S_max"])
        msg = messages_woodbury.update_messages(pred, prm, g, zs[i])
        beliefs.beliefs(pred, msg)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = Ps * g.J / t
    cores = os.cpu_count() or 1
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "P": wl["P"], "S": S, "J": g.J, "Nz": g.Nz,
                      "clutter_per_step": wl["clutter_mean"], "visibility": wl["visibility"],
                      "parallelism": "oracle on the host cores",
                      "sample": f"{Ps} of the workload's {wl['P']} particles per step; value = sample updates / time"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{Ps} particles per step, FP64 Woodbury-mode oracle", **host_cpu()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_gpu(args, rank, world):
    import torch
    from paper_2604_19723_gb300 import bp
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    total_steps = args.warmup + args.steps
    wl, g, prm, scn = make_inputs(args.workload, 2 * total_steps, seed_offset=rank)
    P = args.particles or wl["P"]
    S = wl["fixed_S"] or (wl["K"] + 1)
    S_max = wl["fixed_S"] or wl["S_max"]
    stream = torch.cuda.Stream()
    x_pos, sfv, rho, cc, cs, cr = bp.scenario_arrays(scn, range(1, 2 * total_steps + 1))
    with torch.cuda.stream(stream):
        z_all, eta = bp.synthesize(g, x_pos, sfv, rho, cc, cs, cr, snr_db=wl["snr_db"], seed=wl["seed"] + 11,
                                   step0=1, stream=stream)
    stream.synchronize()
    st = W.state_near_truth(scn, P=P, S=S, n=0, seed=wl["seed"] + 5, eta_true=eta, pos_std=0.01, sfv_std=0.01)
    f = bp.Filter(g, prm, P=P, S_max=S_max, seed=wl["seed"], stream=stream)
    f.set_state(st)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for i in range(args.warmup):
        f.step(z_all[i])
    stream.synchronize()
    f.set_profiling(True)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kappa_ms, iota_ms, prof_tot, repaired = [], [], {}, []
    l0 = f.launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))              # L2 flush between timed steps (256 MB > 129 MB L2)
                ev0[i].record(stream)
                f.step(z_all[args.warmup + i])
                ev1[i].record(stream)
            pr = f.profile()                       # events recorded by the library on its stream
            repaired.append(f.estimate()["iota_repaired"])
            kappa_ms.append(pr["kappa"])
            iota_ms.append(pr["iota"])
            for k, v in pr.items():
                prof_tot[k] = prof_tot.get(k, 0.0) + v
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    launches = f.launch_count() - l0
    f.set_profiling(False)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    t_step = reduce_max(float(np.mean(step_ms)), world, "cuda")
    value = world * P * g.J / (t_step * 1e-3)

    # end to end through the public API: host (pinned) observations copied in every
    # step, estimates copied out every step
    zh = z_all[total_steps:total_steps + args.steps].cpu().pin_memory()
    zd = torch.empty_like(z_all[0])
    e2e_times = []
    torch.cuda.synchronize()
    for i in range(args.steps):
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            e_a.record(stream)
            zd.copy_(zh[i], non_blocking=True)
            f.step(zd)
            est = f.estimate()                     # synchronous D2H of the estimates
            e_b.record(stream)
        stream.synchronize()
        e2e_times.append(e_a.elapsed_time(e_b))
    t_e2e = reduce_max(float(np.mean(e2e_times)), world, "cuda")
    h2d = g.J * g.Nz * 8
    d2h = 8 * (12 + g.J + 9 * S_max + S_max * g.J)

    clocks = clk.summary()
    peaks = measured_peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    SMS = sm_count(dev)
    peak_alu = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    # roofline of the dominant kernel (by its measured time in this run)
    k_ms, i_ms = float(np.mean(kappa_ms)), float(np.mean(iota_ms))
    per_kernel = {
        "k_kappa": (k_ms, kappa_flops(P, S, g.J, g.Nz)),
        "k_iota_blk": (i_ms, iota_flops(P, S, g.J, g.Nf, g.My, g.Mz)),
    }
    def roof(name):
        ms, fl = per_kernel[name]
        a = fl / (ms * 1e-3) / 1e12
        label = name if name != "k_iota_blk" else (
            "k_iota_bulk (FP32, every particle) + k_iota_select + k_iota_blk (float-float, queued particles)"
            if S >= 24 else "k_iota (FP32) + k_iota_blk (flagged particles)")
        r = {"bound": "alu", "kernel": label, "achieved": a, "peak": peak_alu, "unit": "TFLOP/s",
             "frac": a / peak_alu, "traffic": traffic_for(name, args.workload, P), "ms_per_launch": ms,
             "peak_basis": f"FP32 FMA lanes: {SMS} SMs x {FP32_LANES_PER_SM} x 2 flop x {sm_mhz:.0f} MHz "
                           f"(median sampled; SM count from the device); derived, not in MEASURED_PEAKS.json"}
        if name == "k_iota_blk":
            # the same algorithmic flops against the nominal FP64 rate, the precision class the
            # log determinant needs (the kernel emulates it with FP32 operations)
            r["vs_fp64_nominal"] = {"peak": FP64_NOMINAL_TFLOPS, "frac": a / FP64_NOMINAL_TFLOPS}
        if name == "k_kappa" and kappa_tc_used(g, S, S_max):
            # both contractions run on the tensor cores in 3xTF32: each algorithmic flop is
            # three TF32 MMA flops, against the measured bf16 rate (sustained: the kernel runs
            # inside a long step) times the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)
            tf32 = peaks.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25)
            eff = tf32 / 3.0
            fc = kappa_contraction_flops(P, S, g.J, g.Nz)
            ac = fc / (ms * 1e-3) / 1e12
            r = {"bound": "tensor", "kernel": "k_kappa_tc (tcgen05 3xTF32, both contractions)", "achieved": ac,
                 "peak": eff, "unit": "TFLOP/s", "frac": ac / eff,
                 "traffic": traffic_for("k_kappa_tc", args.workload, P),
                 "ms_per_launch": ms,
                 "peak_basis": f"3xTF32 effective: MEASURED_PEAKS bf16_tflops_sustained {peaks.get('bf16_tflops_sustained')} "
                               f"x 1.1/2.25 (nominal TF32/BF16) / 3 products",
                 "cuda_core_part": {"flops": fl - fc, "achieved": (fl - fc) / (ms * 1e-3) / 1e12, "peak": peak_alu,
                                    "note": "element-wise float-float residual and amplitude sums on the FP32 lanes, "
                                            "whole-kernel time"}}
        return r
    dominant = max(per_kernel, key=lambda n: per_kernel[n][0])
    other = "k_iota_blk" if dominant == "k_kappa" else "k_kappa"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_step, "steps_per_s": 1e3 / t_step,
           "higher_is_better": True, "scaling": "weak",
           "vs_baseline": (value / PAPER_UPDATES_PER_S[args.workload]
                           if args.workload in PAPER_UPDATES_PER_S and P == wl["P"] else None),
           "dtype": "f32",
           "data": "synthetic (generative signal model of the paper, seeded)",
           "config": {"workload": args.workload, "P": P, "S": S, "J": g.J, "Nz": g.Nz,
                      "clutter_per_step": wl["clutter_mean"], "visibility": wl["visibility"],
                      "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
           "stage_ms": {k: v / args.steps for k, v in prof_tot.items()},
           "roofline": roof(dominant),
           "roofline_next_kernel": roof(other),
           "e2e": {"value": world * P * g.J / (t_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": t_e2e},
           "gpu_launches": int(launches), "clocks": clocks,
           "iota_floatfloat_particles_per_step": float(np.mean(repaired)) if repaired else 0.0}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, g, prm, scn, args.cpu_particles, z_all[:1].cpu().numpy())
    f.close()
    # the matched-accuracy comparison rides on the headline line only (default workload
    # at its full particle count)
    if rank == 0 and world == 1 and not args.no_matched and args.workload == "scale_64x100k" and P == wl["P"]:
        out["matched_accuracy"] = matched_accuracy()
    if rank == 0:
        print(json.dumps(out))


def matched_accuracy(runs=2, steps=40, P_learned=10000, P_transition=100000):
    """Steps/s at matched accuracy on the 64-PF workload (64 PFs, J = 4, Nz = 160, map in
    place at time 0, the same observations): the learned MT proposal at P_learned particles
    against the plain transition proposal at P_transition, the network trained here on the
    GPU on 2^20 rows simulated from the scene's model.  Accuracy: MT position RMSE and the
    map's OSPA (c = 1 m, p = 2) over the declared PFs; device time per step from CUDA events.
    A short form of the comparison `python -m paper_2604_19723_gb300.learned --c5` runs
    (10 runs x 200 steps)."""
    try:
        from paper_2604_19723_gb300 import learned
        res = learned.c5(runs=runs, steps=steps, P=P_learned, P_transition=P_transition, samples=1 << 20)
        keep = ("rmse", "rmse_runs_min_max", "ospa", "ospa_final", "ospa_runs_min_max", "median_err", "mean_ess",
                "ms_per_step", "steps_per_s", "failed_steps")
        return {"workload": "scale_64x100k, map in place at time 0", "runs": runs, "steps": steps,
                "learned": dict(P=P_learned, **{k: res["learned"][k] for k in keep}),
                "transition": dict(P=P_transition, **{k: res["transition"][k] for k in keep}),
                "rmse_unit": "m", "ospa": {"c_m": res["ospa_c_m"], "p": res["ospa_p"]},
                "train_samples": res["samples"], "train_s": res["train_s"], "final_loss": res["loss"][-1][1]}
    except Exception as e:   # the headline line must not depend on this comparison
        return {"error": f"{type(e).__name__}: {e}"}


# ---------------------------------------------------------------- batched scenarios
def batched_inputs(args, steps):
    """Scenario shapes, truths and the observations of `steps` steps, synthesised on the
    GPU per scenario and concatenated per step in scenario order."""
    sc = W.batched_scenarios(args.scenarios, seed=21)
    scns = []
    for d in sc:
        scns.append(W.make_scenario(d["geom"], d["params"], N=steps + 1, K=d["S"] - 1, seed=d["seed"],
                                    snr_db=20.0, visibility=0.8, clutter_mean=0.0))
    return sc, scns


def batched_oracle_sample(sc, scns, sample_P, n_scen):
    """The FP64 oracle on the host cores: one predict + update of sample_P particles of
    each of the first n_scen scenarios (their own S, J, Nz); updates/s of the sample."""
    from oracle import beliefs, messages_woodbury, model, synth
    done, t = 0, 0.0
    for d, scn in list(zip(sc, scns))[:n_scen]:
        eta = synth.noise_variance(scn)
        z = synth.observe(scn, 1, eta, d["seed"] + 17)
        st = W.state_near_truth(scn, P=sample_P, S=d["S"], n=0, seed=d["seed"] + 7, eta_true=eta,
                                pos_std=0.01, sfv_std=0.01)
        t0 = time.perf_counter()
        pred = model.predict(st, d["params"], d["geom"].J, seed=d["seed"], S_max=d["S"])
        msg = messages_woodbury.update_messages(pred, d["params"], d["geom"], z)
        beliefs.beliefs(pred, msg)
        t += time.perf_counter() - t0
        done += sample_P * d["geom"].J
    return done / t, t


def run_batched(args, rank, world):
    """Many independent scenarios of uneven sizes per step (bp_batch_*): concurrent
    streams with shared workspaces and graph replay, against the same scenarios run as
    the plain path (one stream, launched directly, one scenario after another)."""
    import torch
    from paper_2604_19723_gb300 import bp
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    total = args.warmup + args.steps
    sc, scns = batched_inputs(args, 2 * total)
    stream = torch.cuda.Stream()
    n = len(sc)
    tup = [(d["geom"], d["params"], d["P"], d["S"], d["S"], d["seed"] + 1000003 * rank) for d in sc]
    updates = sum(d["P"] * d["geom"].J for d in sc)

    def make_z(b):
        z = torch.zeros((2 * total, b.z_floats()), dtype=torch.float32, device="cuda")
        for i, (d, scn) in enumerate(zip(sc, scns)):
            x_pos, sfv, rho, cc, cs, cr = bp.scenario_arrays(scn, range(1, 2 * total + 1))
            with torch.cuda.stream(stream):
                zi, _ = bp.synthesize(d["geom"], x_pos, sfv, rho, cc, cs, cr, snr_db=20.0, seed=d["seed"] + 11,
                                      step0=1, stream=stream)
            stream.synchronize()
            o = b.z_offset(i)
            z[:, o:o + 2 * zi.shape[1] * zi.shape[2]] = torch.view_as_real(zi).reshape(2 * total, -1)
        torch.cuda.synchronize()
        return z

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(b, z, members):
        for i in range(args.warmup):
            with torch.cuda.stream(stream):
                b.step(z[i])
        stream.synchronize()
        l0 = sum(m.launch_count() for m in members)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev) as clk:
            for i in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(float(i))
                    ev0[i].record(stream)
                    b.step(z[args.warmup + i])
                    ev1[i].record(stream)
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
        launches = sum(m.launch_count() for m in members) - l0
        ms = [a.elapsed_time(c) for a, c in zip(ev0, ev1)]
        return reduce_max(float(np.mean(ms)), world, "cuda"), launches, clk.summary()

    t_init = time.perf_counter()
    b = bp.Batch(tup, n_streams=args.streams, shared_workspace=True, use_graph=True, stream=stream)
    t_init = time.perf_counter() - t_init
    z = make_z(b)
    tuned = None
    if not args.no_autotune:
        # launch configuration picked by measurement on a sample of the scenarios
        from paper_2604_19723_gb300 import autotune
        b.close()
        tuned = autotune.tune_batch(tup, z, sample=min(n, 64), steps=2, warmup=1, stream=stream)
        args.streams, use_graph = tuned["best"]
        t_init = time.perf_counter()
        b = bp.Batch(tup, n_streams=args.streams, shared_workspace=True, use_graph=use_graph, stream=stream)
        t_init = time.perf_counter() - t_init
    tiles, tile_res = None, {}
    if not args.no_tile_tune:
        # kernel tile shapes per shape class, measured on single filters rebuilt from the
        # members' states (the batch's graphs are captured again with them)
        from paper_2604_19723_gb300 import autotune
        t0 = time.perf_counter()
        tile_res = autotune.tune_batch_tiles(b, tup, z[0], reps=1)
        tiles = {"classes": len(tile_res), "seconds": time.perf_counter() - t0,
                 "choices": {k: {"scenarios": v["scenarios"], "best": {f: x for f, x in v["best"].items() if x}}
                             for k, v in tile_res.items()}}
    members = [b.member(i) for i in range(n)]
    t_step, launches, clocks = timed(b, z, members)
    dev_bytes = b.device_bytes()

    # end to end through the public API: the step's observations copied in from pinned
    # host memory, every scenario's MT estimate read back
    zh = z[total:total + args.steps].cpu().pin_memory()
    zd = torch.empty_like(z[0])
    e2e = []
    torch.cuda.synchronize()
    for i in range(args.steps):
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            e_a.record(stream)
            zd.copy_(zh[i], non_blocking=True)
            b.step(zd)
            for m in members:
                m.estimate()
            e_b.record(stream)
        stream.synchronize()
        e2e.append(e_a.elapsed_time(e_b))
    t_e2e = reduce_max(float(np.mean(e2e)), world, "cuda")
    del members
    b.close()

    # the plain path on the same scenarios: one stream, direct launches
    seq_ms = None
    if not args.no_sequential:
        b1 = bp.Batch(tup, n_streams=1, shared_workspace=True, use_graph=False, stream=stream)
        if args.sequential_tiles:
            for v in tile_res.values():
                for i in v["members"]:
                    b1.set_tiles(i, **v["best"])
        m1 = [b1.member(i) for i in range(n)]
        seq_ms, _, _ = timed(b1, z, m1)
        del m1
        b1.close()

    peaks = measured_peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    SMS = sm_count(dev)
    peak_alu = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    fl = sum(kappa_flops(d["P"], d["S"], d["geom"].J, d["geom"].Nz) +
             iota_flops(d["P"], d["S"], d["geom"].J, d["geom"].Nf, d["geom"].My, d["geom"].Mz) for d in sc)
    ach = fl / (t_step * 1e-3) / 1e12
    value = world * updates / (t_step * 1e-3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_step, "steps_per_s": 1e3 / t_step,
           "scenario_steps_per_s": world * n * 1e3 / t_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (generative signal model of the paper, seeded)",
           "config": {"workload": "batched", "scenarios": n, "S": "U{1..64}", "P": "U{256..16384}",
                      "Nz": "U{5..300} (one antenna below 16, else 2x2 URA)", "J": 4,
                      "particle_PA_updates_per_step": updates, "streams": min(args.streams, n),
                      "graph": bool(tuned["best"][1]) if tuned else True, "shared_workspace": True,
                      "autotune": tuned, "tiles": tiles, "device_GB": dev_bytes / 1e9,
                      "init_s": t_init, "l2": "flushed between timed steps (256 MB write)",
                      "parallelism": f"replicas x{world}"},
           "sequential": ({"ms_per_step": seq_ms, "value": world * updates / (seq_ms * 1e-3),
                           "speedup": seq_ms / t_step,
                           "how": "same scenarios, one stream, direct launches, " +
                                  ("the tuned tiles" if args.sequential_tiles and tile_res else "built-in tiles")}
                          if seq_ms else None),
           "roofline": {"bound": "alu", "kernel": "k_kappa + k_iota/k_iota_blk of every scenario (whole step time)",
                        "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s", "frac": ach / peak_alu,
                        "traffic": None,
                        "peak_basis": f"FP32 FMA lanes: {SMS} SMs x {FP32_LANES_PER_SM} x 2 flop x {sm_mhz:.0f} MHz"},
           "e2e": {"value": world * updates / (t_e2e * 1e-3), "unit": UNIT,
                   "h2d_bytes_per_step": int(4 * z.shape[1]),
                   "d2h_bytes_per_step": int(sum(8 * (13 + 4 + 9 * d["S"] + 4 * d["S"]) + 4 for d in sc)),
                   "ms_per_step": t_e2e},
           "gpu_launches": int(launches), "clocks": clocks}
    if rank == 0 and not args.no_cpu_baseline:
        v, t = batched_oracle_sample(sc, scns, args.cpu_particles // 4, 4)
        cores = os.cpu_count() or 1
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"one predict+update of {args.cpu_particles // 4} particles of each of the "
                                         f"first 4 scenarios (FP64 Woodbury-mode oracle, {t:.2f} s)", **host_cpu()}
    if rank == 0:
        print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="scale_64x100k")
    ap.add_argument("--particles", type=int, default=0)
    ap.add_argument("--cpu-particles", type=int, default=1024)
    ap.add_argument("--ref-particles", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-matched", action="store_true", help="skip the learned-proposal matched-accuracy comparison")
    ap.add_argument("--scenarios", type=int, default=4096, help="batched workload: number of scenarios")
    ap.add_argument("--streams", type=int, default=32, help="batched workload: concurrent streams")
    ap.add_argument("--no-sequential", action="store_true", help="batched workload: skip the one-stream run")
    ap.add_argument("--no-tile-tune", action="store_true", help="batched workload: built-in kernel tile shapes")
    ap.add_argument("--sequential-tiles", action="store_true",
                    help="batched workload: the one-stream run uses the tuned tiles too")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched workload: use --streams with graphs instead of the measured best configuration")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.workload == "batched":
        run_batched(args, rank, world)
    else:
        run_gpu(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
