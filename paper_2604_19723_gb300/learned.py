"""Learned MT proposal: training on the GPU and its gain over the transition proposal.

The proposal network (bp_mlp_*, BF16 tensor-core kernels) is trained by its own Adam
steps on samples that bp_lp_dataset simulates from the model of a workload (its
geometry, surfaces, amplitudes and noise variance), then attached to filters with
bp_set_mt_proposal.  The importance weights keep every filter's posterior exact, so
the network can only change how well P particles cover it: `compare` runs the same
observations with and without the network and reports the MT posterior's effective
sample size and position error.

Runs from the command line:  python -m paper_2604_19723_gb300.learned --runs 4 --steps 50 --P 2000
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time
from typing import Dict

import numpy as np

from . import bp
from . import workload as W
from .ospa import ospa

OSPA_C = 1.0   # cut-off of the map's OSPA distance [m]; order p = 2


def scenario_model(name: str, seed: int):
    """Geometry, parameters, surfaces, moduli and noise variance of a workload's scene."""
    wl = W.workload(name)
    g, prm = wl["geom"], wl["params"]
    scn = W.make_scenario(g, prm, N=2, K=wl["K"], seed=seed, snr_db=wl["snr_db"])
    x_pos, sfv, rho, cc, cs, cr = bp.scenario_arrays(scn, [1])
    _, eta = bp.synthesize(g, x_pos, sfv, rho, cc, cs, cr, snr_db=wl["snr_db"], seed=seed, step0=1)
    return g, prm, scn.sfv_true, scn.rho_abs, eta


def train_proposal(name: str = "paper_exp1_proposal", n_samples: int = 1 << 17, steps: int = 2000,
                   batch: int = 4096, lr: float = 1e-3, seed: int = 7, data_seed: int = 1,
                   coherent: bool = True) -> Dict:
    """Simulates n_samples training rows (amplitude phases common to all PAs, or per PA
    with coherent False) and runs `steps` Adam steps on random batches; returns the
    network and the loss history (mean per row, every 100 steps)."""
    import torch
    g, prm, sfv, rho_abs, eta = scenario_model(name, data_seed)
    t0 = time.perf_counter()
    X, T = bp.lp_dataset(g, prm, sfv, rho_abs, eta, n_samples, seed=seed, coherent=coherent)
    t_data = time.perf_counter() - t0
    net = bp.Mlp(W.mlp_init(seed))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    t0 = time.perf_counter()
    for s in range(steps):
        idx = torch.randint(0, n_samples, (batch,), device="cuda", generator=gen)
        net.train_step(X[idx], T[idx], lr, loss)
        if s % 100 == 0 or s == steps - 1:
            hist.append((s, float(loss.item()) / batch))
    net.sync()
    return dict(net=net, loss=hist, data_s=t_data, train_s=time.perf_counter() - t0, eta=eta)


def run(name: str, net, runs: int, steps: int, P: int, seed: int) -> Dict:
    """The filter over `steps` steps of `runs` scenes (map in place at time 0), with the
    network attached or (net None) with the transition proposal.  Each step's device
    time comes from CUDA events recorded on the filter's stream around bp_predict +
    bp_update; the estimate is read outside them."""
    import torch
    wl = W.workload(name)
    g, prm = wl["geom"], wl["params"]
    err, ess = np.full((runs, steps), np.nan), np.full((runs, steps), np.nan)
    osp = np.full((runs, steps), np.nan)
    step_ms = []
    wall = 0.0
    stream = torch.cuda.Stream()
    for r in range(runs):
        scn = W.make_scenario(g, prm, N=steps, K=wl["K"], seed=seed + r, snr_db=wl["snr_db"],
                              visibility=wl["visibility"], clutter_mean=wl["clutter_mean"])
        x_pos, sfv, rho, cc, cs, cr = bp.scenario_arrays(scn, range(1, steps + 1))
        with torch.cuda.stream(stream):
            z, eta = bp.synthesize(g, x_pos, sfv, rho, cc, cs, cr, snr_db=wl["snr_db"], seed=seed + r + 7, step0=1,
                                   stream=stream)
        stream.synchronize()
        f = bp.Filter(g, prm, P=P, S_max=wl["S_max"], seed=seed + r, stream=stream)
        f.set_state(W.state_near_truth(scn, P=P, S=wl["K"] + 1, n=0, seed=seed + r + 3, eta_true=eta,
                                       pos_std=0.02, vel_std=0.05, sfv_std=0.02))
        if net is not None:
            f.set_mt_proposal(net)
        t0 = time.perf_counter()
        try:
            for n in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                f.step(z[n])
                e1.record(stream)
                try:
                    e = f.estimate()
                except bp.BPError:
                    break
                step_ms.append(e0.elapsed_time(e1))
                err[r, n] = np.linalg.norm(e["x_hat"][:3] - scn.x_true[n + 1, :3])
                ess[r, n] = e["ess_x"]
                decl = [s for s in range(1, e["S"]) if e["declared"][s]]
                osp[r, n] = ospa(e["phi_hat"][decl, :3].reshape(-1, 3), scn.sfv_true, OSPA_C, 2.0)
        finally:
            wall += time.perf_counter() - t0
            f.close()
    return dict(err=err, ess=ess, ospa=osp, wall_s=wall, step_ms=step_ms)


def compare(name: str = "paper_exp1_proposal", runs: int = 4, steps: int = 50, P: int = 2000, seed: int = 500,
            train: Dict = None, P_transition: int = None, P_more=()) -> Dict:
    """The same scenes with the learned proposal at P particles (and at every count in
    P_more) and with the transition proposal at P_transition (default P)."""
    train = train or train_proposal(name)
    with_net = run(name, train["net"], runs, steps, P, seed)
    more = {int(q): run(name, train["net"], runs, steps, int(q), seed) for q in P_more}
    plain = run(name, None, runs, steps, P_transition or P, seed)

    def stats(d):
        e = d["err"]
        ms = float(np.mean(d["step_ms"])) if d["step_ms"] else float("nan")
        run_rmse = np.sqrt(np.nanmean(e ** 2, axis=1))
        run_ospa = np.nanmean(d["ospa"], axis=1)
        return dict(rmse=float(np.sqrt(np.nanmean(e ** 2))), median_err=float(np.nanmedian(e)),
                    rmse_runs_min_max=[float(np.nanmin(run_rmse)), float(np.nanmax(run_rmse))],
                    ospa=float(np.nanmean(d["ospa"])), ospa_final=float(np.nanmean(d["ospa"][:, -1])),
                    ospa_runs_min_max=[float(np.nanmin(run_ospa)), float(np.nanmax(run_ospa))],
                    mean_ess=float(np.nanmean(d["ess"])), median_ess=float(np.nanmedian(d["ess"])),
                    failed_steps=int(np.sum(np.isnan(e))), ms_per_step=ms, steps_per_s=1e3 / ms,
                    wall_s=d["wall_s"])

    return dict(workload=name, runs=runs, steps=steps, P=P, P_transition=P_transition or P, loss=train["loss"],
                train_s=train["train_s"], data_s=train["data_s"], ospa_c_m=OSPA_C, ospa_p=2,
                learned=stats(with_net), learned_more={q: stats(d) for q, d in more.items()},
                transition=stats(plain))


def c5(runs: int = 10, steps: int = 200, P: int = 10000, P_transition: int = 100000, samples: int = 1 << 20,
       train_steps: int = 2000, seed: int = 900, P_more=()) -> Dict:
    """The learned-proposal comparison at the 64-PF scale (64 PFs held fixed, J = 4,
    Nz = 160, 200 spurious paths per step): the network trained on `samples` rows simulated
    from the scene's model, the learned proposal at P particles against the transition
    proposal at P_transition, map scored by OSPA over the declared PFs and the MT by RMSE."""
    tr = train_proposal("scale_64x100k", n_samples=samples, steps=train_steps)
    res = compare("scale_64x100k", runs=runs, steps=steps, P=P, seed=seed, train=tr, P_transition=P_transition,
                  P_more=P_more)
    res["samples"] = samples
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="paper_exp1_proposal")
    ap.add_argument("--runs", type=int, default=4)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--P", type=int, default=2000)
    ap.add_argument("--samples", type=int, default=None, help="training rows (2^17; 2^20 with --c5)")
    ap.add_argument("--P-more", type=int, nargs="*", default=[], help="--c5: further particle counts of the learned arm")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--P-transition", type=int, default=None, help="particles of the transition-proposal runs")
    ap.add_argument("--c5", action="store_true", help="the 64-PF comparison (10000 vs 100000 particles by default)")
    a = ap.parse_args(argv)
    if a.c5:
        res = c5(runs=a.runs, steps=a.steps, P=a.P if a.P != 2000 else 10000, samples=a.samples or (1 << 20),
                 train_steps=a.train_steps, P_more=a.P_more)
        res.pop("loss", None)
        print(json.dumps(res))
        return
    tr = train_proposal(a.workload, a.samples or (1 << 17), a.train_steps, lr=a.lr)
    res = compare(a.workload, a.runs, a.steps, a.P, train=tr, P_transition=a.P_transition)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
