"""Monte Carlo evaluation of the SLAM variants against the posterior CRLBs (Sec. VII).

The variants of Sec. VII:
  * NZM: the method as derived (non-zero-mean amplitude prior), on coherent data
    (amplitude phases common to all PAs);
  * ZM: the zero-mean amplitude prior (mu == 0), on coherent data;
  * NZM-NC: NZM on noncoherent data (amplitude phases drawn independently per PA and
    step).

One run: a scenario of the Experiment 1 shape with its own amplitude phases and noise,
observations synthesised on the GPU (bp_synthesize), the filter stepped over N steps
through the C ABI.  Per step the MT position error and, per true surface, the error of
the SFV estimate of the declared PF associated with it by the Hungarian method (missed
detections and false alarms are not counted, as for the paper's mapping RMSE).

Bound: per step the Bayesian snapshot FIM J_B,n is the mean of the classic FIM over the
runs' true states (bp_pcrlb_fim: coherent for coherent data, noncoherent otherwise), the
recursion (bp_pcrlb_recursion) gives PEB and MEB.  The amplitudes of the bound absorb the
path loss and the carrier phase of each component (Sec. S-VII):
rho~ = rho lambda / (4 pi |r'|) exp(-j 2 pi |r'| / lambda).
Readings: J_{1|0} is the inverse of the diagonal prior covariance of the state at time
0 (uniform MT prior box, uniform birth box for the SFVs, phases uniform on a circle,
broad moduli and noise variance); nuisance parameters carry no memory (pseudo variances
sigma_phi = sigma_a = sigma_eta = 1e3).

Runs from the command line:  python -m paper_2604_19723_gb300.evaluate --runs 10 --steps 200
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time
from typing import Dict, List

import numpy as np

from . import bp
from . import workload as W

VARIANTS = {
    # name: (zero_mean, coherent data)
    "nzm": (0, True),
    "zm": (1, True),
    "nzm_nc": (0, False),
}

NUISANCE_SIGMA = 1e3

# starts of a run: "prior" is the paper's (MT from the uniform prior box, the LoS alone,
# every other PF born on the way); the others start near the truth at time 0 with the
# given standard deviations (position, velocity, SFV position) and S0 PFs (None: the LoS
# and one PF per true surface, i.e. the tracking phase with the map in place)
INIT_STD = {
    "truth": (0.02, 0.05, 0.02, 1),
    "truth_map": (0.02, 0.05, 0.02, None),
}


def associate(est: np.ndarray, truth: np.ndarray) -> np.ndarray:
    """Hungarian association of SFV estimates (m, 3) to true SFVs (K, 3); returns the
    error of each true surface, NaN where no estimate is associated."""
    from scipy.optimize import linear_sum_assignment
    K = truth.shape[0]
    err = np.full(K, np.nan)
    if est.shape[0] == 0 or K == 0:
        return err
    cost = np.linalg.norm(est[:, None, :] - truth[None, :, :], axis=-1)
    r, c = linear_sum_assignment(cost)
    err[c] = cost[r, c]
    return err


def rmse(err: np.ndarray, axis: int = 0) -> np.ndarray:
    """Root mean square over the runs, ignoring NaN (unassociated) entries."""
    e2 = np.asarray(err, float) ** 2
    cnt = np.sum(np.isfinite(e2), axis=axis)
    s = np.nansum(e2, axis=axis)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(cnt > 0, np.sqrt(s / np.maximum(cnt, 1)), np.nan)


def component_ranges(geom: W.Geometry, p: np.ndarray, sfv: np.ndarray) -> np.ndarray:
    """|r'| per PA and component (LoS first): the distance from the PA to the MT or to
    the virtual MT H p + s mirrored at the SFV s (Sec. II)."""
    K = sfv.shape[0]
    d = np.zeros((geom.J, K + 1))
    for j in range(geom.J):
        d[j, 0] = np.linalg.norm(p - geom.p_pa[j])
        for k in range(K):
            s = sfv[k]
            H = np.eye(3) - 2.0 * np.outer(s, s) / (s @ s)
            d[j, k + 1] = np.linalg.norm(H @ p + s - geom.p_pa[j])
    return d


def bound_amplitudes(scn: W.Scenario, n: int) -> np.ndarray:
    """rho~ (J, K+1) of the truth at step n (path loss and carrier phase absorbed)."""
    g = scn.geom
    lam = g.c / g.fc
    d = component_ranges(g, scn.x_true[n, :3], scn.sfv_true)
    rho = scn.rho_abs[None, :] * np.exp(1j * scn.rho_phase[n]) * scn.visible[n]
    return rho * lam / (4.0 * np.pi * d) * np.exp(-2j * np.pi * d / lam)


def prior_information(params: W.Params, K: int, J: int, coherent: bool, init: str = "prior") -> np.ndarray:
    """J_{1|0}: inverse of a diagonal covariance of the state at time 0, the one the runs
    start from (uniform boxes for "prior", the near-truth spreads otherwise)."""
    dim = bp.pcrlb_dim(K, J, coherent)
    var = np.full(dim, NUISANCE_SIGMA ** 2)
    lo, hi = np.asarray(params.p_min, float), np.asarray(params.p_max, float)
    var[0:3] = np.maximum((hi - lo) ** 2 / 12.0, 1e-6)
    var[3:6] = np.maximum((2.0 * np.asarray(params.v_max, float)) ** 2 / 12.0, 1e-6)
    blo, bhi = np.asarray(params.birth_min, float), np.asarray(params.birth_max, float)
    bv = np.maximum((bhi - blo) ** 2 / 12.0, 1e-6)
    if init in INIT_STD:
        pos_std, vel_std, sfv_std, S0 = INIT_STD[init]
        var[0:3], var[3:6] = pos_std ** 2, vel_std ** 2
        if S0 is None:
            bv = np.full(3, sfv_std ** 2)
    for k in range(K):
        var[6 + 3 * k:9 + 3 * k] = bv
    nph = (K + 1) if coherent else (K + 1) * J
    var[6 + 3 * K:6 + 3 * K + nph] = math.pi ** 2 / 3.0
    return np.diag(1.0 / var)


def transition(params: W.Params, K: int, J: int, coherent: bool):
    """F and Q of the bound's global state: NCV for the MT, random walk (sigma_sfv) for
    the SFVs, no memory for the nuisance parameters (Sec. S-VII)."""
    dim = bp.pcrlb_dim(K, J, coherent)
    T, q = params.T, params.sigma_v ** 2
    F = np.zeros((dim, dim))
    Q = np.zeros((dim, dim))
    nd = params.motion_dims
    for a in range(3):
        F[a, a] = F[3 + a, 3 + a] = 1.0
        F[a, 3 + a] = T
        if a < nd:
            Q[a, a] = q * T ** 4 / 4.0
            Q[a, 3 + a] = Q[3 + a, a] = q * T ** 3 / 2.0
            Q[3 + a, 3 + a] = q * T ** 2
    for i in range(6, 6 + 3 * K):
        F[i, i] = 1.0
        Q[i, i] = params.sigma_sfv ** 2
    for i in range(6 + 3 * K, dim):
        Q[i, i] = NUISANCE_SIGMA ** 2
    if nd == 2:
        # planar motion: z and v_z are held; a tiny process noise keeps the
        # predicted covariance invertible
        Q[2, 2] = Q[5, 5] = 1e-12
    return F, Q


@dataclasses.dataclass
class RunResult:
    pos_err: np.ndarray        # (N,)
    map_err: np.ndarray        # (N, K) NaN where no declared PF is associated
    S: np.ndarray              # (N,) PFs after the update (LoS included)
    declared: np.ndarray       # (N,) declared PFs besides the LoS
    eta: float                 # noise variance of the synthetic data
    failed: int = -1           # step at which the filter reported a numerical failure


def run_filter(name: str, variant: str, P: int, N: int, seed: int, init: str = "prior", net=None):
    """One run of a variant on the named workload's shape (Philox key and truth from seed);
    returns (RunResult, Scenario)."""
    zm, coherent = VARIANTS[variant]
    wl = W.workload(name)
    g, prm = wl["geom"], dataclasses.replace(wl["params"], zero_mean=zm)
    scn = W.make_scenario(g, prm, N=N, K=wl["K"], seed=seed, snr_db=wl["snr_db"],
                          visibility=wl["visibility"], clutter_mean=wl["clutter_mean"], coherent=coherent)
    x_pos, sfv, rho, cc, cs, cr = bp.scenario_arrays(scn, range(1, N + 1))
    z, eta = bp.synthesize(g, x_pos, sfv, rho, cc, cs, cr, snr_db=wl["snr_db"], seed=seed + 7, step0=1)
    K = scn.sfv_true.shape[0]
    f = bp.Filter(g, prm, P=P, S_max=wl["S_max"], seed=seed)
    if init in INIT_STD:
        pos_std, vel_std, sfv_std, S0 = INIT_STD[init]
        f.set_state(W.state_near_truth(scn, P=P, S=K + 1 if S0 is None else S0, n=0, seed=seed + 3, eta_true=eta,
                                       pos_std=pos_std, vel_std=vel_std, sfv_std=sfv_std))
    elif init != "prior":
        raise ValueError(init)
    if net is not None:
        f.set_mt_proposal(net)
    pos, mp = np.full(N, np.nan), np.full((N, K), np.nan)
    S, dec = np.zeros(N, np.int32), np.zeros(N, np.int32)
    failed = -1
    try:
        for n in range(N):
            f.step(z[n])
            try:
                e = f.estimate()
            except bp.BPError:
                failed = n          # a numerical failure ends the run; its errors stay NaN
                break
            pos[n] = np.linalg.norm(e["x_hat"][:3] - scn.x_true[n + 1, :3])
            sel = np.nonzero(e["declared"][1:])[0] + 1
            mp[n] = associate(e["phi_hat"][sel, :3], scn.sfv_true)
            S[n], dec[n] = e["S"], len(sel)
    finally:
        f.close()
    return RunResult(pos, mp, S, dec, eta, failed), scn


def bound(scns: List[W.Scenario], etas: List[float], coherent: bool, init: str = "prior"):
    """PEB (N,) and MEB (N, K) for the runs' truths (mean FIM over the runs per step)."""
    s0 = scns[0]
    g, prm, N = s0.geom, s0.params, s0.N
    K = s0.sfv_true.shape[0]
    eta = float(np.mean(etas))
    Js = np.zeros((N, bp.pcrlb_dim(K, g.J, coherent), bp.pcrlb_dim(K, g.J, coherent)))
    for n in range(1, N + 1):
        x = np.stack([s.x_true[n] for s in scns])
        sfv = np.stack([s.sfv_true for s in scns])
        rho = np.stack([bound_amplitudes(s, n) for s in scns])
        Js[n - 1] = bp.pcrlb_fim(g, x, sfv, rho, eta, coherent)
    F, Q = transition(prm, K, g.J, coherent)
    return bp.pcrlb_recursion(F, Q, prior_information(prm, K, g.J, coherent, init), Js, K)


def evaluate(name: str = "paper_exp1_proposal", variants=("nzm", "zm", "nzm_nc"), runs: int = 10, steps: int = 200,
             P: int = None, seed: int = 100, init: str = "truth_map", net=None) -> Dict:
    """RMSE of the MT position and of each surface's SFV per step, with PEB and MEB; with
    a proposal network (bp.Mlp, or a dict coherent-data flag -> bp.Mlp) every run draws
    its MT particles from the learned proposal."""
    wl = W.workload(name)
    P = P or wl["P"]
    out = dict(workload=name, runs=runs, steps=steps, P=P, init=init, learned=net is not None, variants={})
    for v in variants:
        t0 = time.perf_counter()
        vnet = net.get(VARIANTS[v][1]) if isinstance(net, dict) else net
        res, scns = zip(*[run_filter(name, v, P, steps, seed + r, init, vnet) for r in range(runs)])
        wall = time.perf_counter() - t0
        peb, meb = bound(list(scns), [r.eta for r in res], VARIANTS[v][1], init)
        pos = np.stack([r.pos_err for r in res])
        mp = np.stack([r.map_err for r in res])
        out["variants"][v] = dict(
            rmse_pos=rmse(pos).tolist(), median_pos=np.nanmedian(pos, axis=0).tolist(), peb=peb.tolist(),
            rmse_map=rmse(mp).tolist(), meb=meb.tolist(),
            detected=np.mean(np.isfinite(mp), axis=0).tolist(),
            mean_S=np.mean([r.S for r in res], axis=0).tolist(),
            mean_declared=np.mean([r.declared for r in res], axis=0).tolist(),
            final_err=[float(r.pos_err[-1]) for r in res],
            failed=[int(r.failed) for r in res],
            wall_s=wall)
    return out


def summary(res: Dict, at=(10, 50, 100, 200)) -> str:
    """A plain-text table of RMSE against the bounds at a few steps."""
    lines = [f"workload {res['workload']}, {res['runs']} runs, P = {res['P']}, init {res['init']}"
             f"{', learned MT proposal' if res.get('learned') else ''}",
             "variant  step  RMSE_pos[m]  median[m]  PEB[m]   RMSE_map (surfaces 1..K) [m]   MEB [m]   PFs"]
    for v, d in res["variants"].items():
        for n in at:
            if n > len(d["rmse_pos"]):
                continue
            i = n - 1
            rm = " ".join(f"{x:.4f}" for x in d["rmse_map"][i])
            mb = " ".join(f"{x:.4f}" for x in d["meb"][i])
            lines.append(f"{v:7s} {n:5d}  {d['rmse_pos'][i]:.4f}      {d['median_pos'][i]:.4f}     {d['peb'][i]:.4f}"
                         f"   {rm}   {mb}   {d['mean_S'][i]:.1f}")
        fe = np.asarray(d["final_err"])
        lines.append(f"{v:7s} runs failed: {sum(1 for x in d['failed'] if x >= 0)}, final error > 0.5 m: "
                     f"{int(np.sum(~(fe <= 0.5)))}, wall {d['wall_s']:.1f} s")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="paper_exp1_proposal")
    ap.add_argument("--variants", default="nzm,zm,nzm_nc")
    ap.add_argument("--runs", type=int, default=10)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--P", type=int, default=None)
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--init", default="truth_map", choices=["prior"] + sorted(INIT_STD))
    ap.add_argument("--json", default=None, help="write the full per-step result here")
    ap.add_argument("--learned", action="store_true", help="draw MT particles from a trained proposal network")
    a = ap.parse_args(argv)
    net = None
    if a.learned:
        # one network per kind of data: coherent for NZM and ZM, noncoherent for NZM-NC
        from . import learned
        kinds = {VARIANTS[v][1] for v in a.variants.split(",")}
        net = {c: learned.train_proposal(a.workload, coherent=c)["net"] for c in kinds}
    res = evaluate(a.workload, tuple(a.variants.split(",")), a.runs, a.steps, a.P, a.seed, a.init, net)
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(res, fh)
    print(summary(res))


if __name__ == "__main__":
    main()
