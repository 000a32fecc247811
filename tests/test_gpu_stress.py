"""The mixed-precision stress workload: 32 PFs, Nz = 1024 (16 frequencies, 8 x 8 URA),
SNR 30 dB, 500 unmodelled spurious paths per step, against the FP64 oracle through the
C ABI, with every output's error printed (and recorded in the design notes).

At 30 dB and Nz = 1024 the quadratic forms reach ~Nz (1 + SNR) ~ 1e6 noise units, the
regime where FP32 log-likelihoods lose their digits; this shape also takes the 32-column
tensor-core PF likelihood with pass-1 rounds of a quarter frequency (the 8 x 8 URA's 64
elements per frequency), and the 32-row variant of the FP32 MT kernel.

  * test_stress_shape_stagewise: the full stage-wise parity at P = 1000 (ragged over the
    256-particle tiles), the oracle evaluating every particle (Woodbury form).
  * test_stress_full_size_sampled: 262144 particles, the launch configuration the bench
    uses; the message table over every particle (streamed, process pool), the existence
    tests, and the per-particle messages on a sample, as in test_gpu_fullsize.py.
"""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import beliefs, messages_woodbury, model, synth
from oracle import messages_dense
from paper_2604_19723_gb300 import workload as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import bp  # noqa: E402

W_TOL = 1e-4
P_TOL = 1e-5
M_TOL = 1e-4


def rel_weight_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(b), 1e-300))


def rel_weight_err_log(log_a, log_b):
    wa = np.exp(log_a - np.max(log_a))
    wb = np.exp(log_b - np.max(log_b))
    wa, wb = wa / wa.sum(), wb / wb.sum()
    return float(np.max(np.abs(wa - wb)) / np.max(wb))


def stress_case(P, seed_offset=0):
    wl = W.workload("stress_32x262k")
    g, prm, S = wl["geom"], wl["params"], wl["fixed_S"]
    scn = W.make_scenario(g, prm, N=3, K=wl["K"], seed=wl["seed"] + seed_offset, snr_db=wl["snr_db"],
                          visibility=wl["visibility"], clutter_mean=wl["clutter_mean"])
    eta = synth.noise_variance(scn)
    # the observation as the C ABI takes it (complex64), for both sides
    z = synth.observe(scn, 1, eta, wl["seed"] + 100).astype(np.complex64).astype(np.complex128)
    st = W.state_near_truth(scn, P=P, S=S, n=0, seed=wl["seed"] + 5, eta_true=eta, pos_std=0.01, sfv_std=0.01)
    pred = model.predict(st, prm, g.J, seed=wl["seed"], S_max=wl["S_max"])
    return wl, g, prm, scn, z, pred


def gpu_update(pred, g, prm, z, P, S_max, seed):
    f = bp.Filter(g, prm, P=P, S_max=S_max, seed=seed)
    f.set_predicted(pred.n, pred.S, pred.x, pred.phi, pred.eta, pred.w_beta, pred.w_alpha, pred.w_xi, pred.zeta)
    f.update(torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda())
    torch.cuda.synchronize()
    return f


def test_stress_shape_stagewise():
    P = 1000
    wl, g, prm, scn, z, pred = stress_case(P, seed_offset=1)
    f = gpu_update(pred, g, prm, z, P, wl["S_max"], wl["seed"])
    msg = messages_woodbury.update_messages(pred, prm, g, z)
    bel = beliefs.beliefs(pred, msg)
    est = beliefs.estimate(pred, bel, prm)
    tab = f.diag_table(pred.S)
    gw = f.diag_weights(pred.S)
    ll = f.diag_loglik(pred.S)
    di = f.diag_iota()
    ge = f.estimate()
    f.close()
    rep = {}
    for key in ("m", "mw", "mu3", "mu4"):
        ref = getattr(msg.table, key)
        rep["table_" + key] = float(np.max(np.abs(tab[key] - ref)) / max(np.max(np.abs(ref)), 1e-300))
    rep["p_pr"] = float(np.max(np.abs(gw["p_pr"] - bel.p_pr)))
    rep["p_s"] = float(np.max(np.abs(gw["p_s"] - bel.p_s)))
    rep["w_x"] = rel_weight_err(gw["w_x"], bel.w_x)
    rep["w_eta"] = max(rel_weight_err(gw["w_eta"][j], bel.w_eta[j]) for j in range(g.J))
    rep["w_y"] = max(rel_weight_err(gw["w_y"][s], bel.w_y[s]) for s in range(pred.S) if bel.p_s[s] > 1e-12)
    rep["x_hat"] = float(np.max(np.abs(ge["x_hat"] - est.x_hat)))
    rep["eta_hat_rel"] = float(np.max(np.abs(ge["eta_hat"] - est.eta_hat) / est.eta_hat))
    live = [s for s in range(pred.S) if est.p_s[s] > 1e-3]
    rep["phi_hat_pos"] = float(max(np.max(np.abs(ge["phi_hat"][s, :3] - est.phi_hat[s, :3])) for s in live))
    rep["phi_hat_gamma_rel"] = float(max(abs(ge["phi_hat"][s, 3] - est.phi_hat[s, 3]) / abs(est.phi_hat[s, 3])
                                         for s in live))
    sel = np.zeros(P, bool)
    sel[di["selected"]] = True
    d = np.abs(ll["log_iota"] - msg.log_iota.sum(0))
    ref_i = msg.log_iota.sum(0)
    rep["log_iota_selected"] = float(np.max(d[sel] / (1e-4 + 1e-8 * np.abs(ref_i[sel])))) * 1e-4
    rep["log_iota_fp32_over_bound"] = float(np.max(d[~sel] / di["err"][~sel])) if (~sel).any() else 0.0
    lo = msg.log_omega1 - msg.log_omega0
    rep["llr_omega"] = float(np.max(np.abs(ll["llr_omega"] - lo)))
    print(rep)
    for key in ("m", "mw", "mu3", "mu4"):
        assert rep["table_" + key] < 1e-5, rep
    assert rep["p_pr"] < P_TOL and rep["p_s"] < P_TOL, rep
    assert rep["w_x"] < W_TOL and rep["w_eta"] < W_TOL and rep["w_y"] < W_TOL, rep
    assert rep["x_hat"] < M_TOL and rep["eta_hat_rel"] < M_TOL, rep
    assert rep["phi_hat_pos"] < M_TOL and rep["phi_hat_gamma_rel"] < M_TOL, rep
    assert rep["log_iota_selected"] < 1e-4 and rep["log_iota_fp32_over_bound"] <= 1.0, rep


@pytest.fixture(scope="module")
def pool():
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    try:
        with ctx.Pool(max(1, min(16, os.cpu_count() or 1))) as p:
            yield p
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def sub_pred(pred, idx):
    return model.Predicted(n=pred.n, S=pred.S, x=pred.x[:, idx], phi=pred.phi[:, :, idx], eta=pred.eta[:, idx],
                           w_beta=pred.w_beta[idx], w_alpha=pred.w_alpha[:, idx], w_xi=pred.w_xi[:, idx],
                           zeta=pred.zeta, is_new=pred.is_new)


def test_stress_full_size_sampled(pool):
    wl = W.workload("stress_32x262k")
    P = wl["P"]
    wl, g, prm, scn, z, pred = stress_case(P)
    tab = messages_dense.message_table_streamed(pred, prm, g, chunk=4096, pool=pool)
    f = gpu_update(pred, g, prm, z, P, wl["S_max"], wl["seed"])
    gt = f.diag_table(pred.S)
    ll = f.diag_loglik(pred.S)
    gw = f.diag_weights(pred.S)
    di = f.diag_iota()
    f.close()
    rep = {}
    for key in ("m", "mw", "mu3", "mu4"):
        ref = getattr(tab, key)
        rep["table_" + key] = float(np.max(np.abs(gt[key] - ref)) / max(np.max(np.abs(ref)), 1e-300))
    # the sample: particles the GPU evaluated in float-float, a spread, the ragged last one
    idx = np.unique(np.r_[di["selected"][:96], np.linspace(0, P - 1, 24).astype(int), P - 1])
    sp = sub_pred(pred, idx)
    mwb = messages_woodbury.messages_from_table(sp, tab, g, z)
    # PR existence tests and p_s^(j): functions of the table alone
    o1, o0 = mwb.log_omega1, mwb.log_omega0
    lo = o1 - o0
    rep["llr_omega"] = float(np.max(np.abs(ll["llr_omega"] - lo)))
    rep["p_pr"] = float(np.max(np.abs(gw["p_pr"] - beliefs.pr_existence(pred.zeta, o1, o0))))
    li = mwb.log_iota.sum(0)
    sel = np.isin(idx, di["selected"])
    d = np.abs(ll["log_iota"][idx] - li)
    # float-float values to 1e-4 absolute plus 1e-8 relative (particles far below the best,
    # with weights of zero, are queued only when their FP32 bound is not finite)
    rep["log_iota_selected"] = float(np.max(d[sel] / (1e-4 + 1e-8 * np.abs(li[sel])))) * 1e-4
    rep["log_iota_fp32_over_bound"] = float(np.max(d[~sel] / di["err"][idx][~sel]))
    lwb = np.log(pred.w_beta[idx])
    lw_all = np.log(pred.w_beta) + ll["log_iota"]
    rel = lwb + li - lw_all.max()
    k = int(np.argmax(np.where(sel, d, -1.0)))
    rep["worst_selected_rel"] = float(rel[k])
    rep["selected_weighted_err"] = float(np.max(np.exp(rel[sel]) * d[sel]))
    rep["selected_within_3"] = float(np.max(np.where(rel[sel] > -3.0, d[sel], 0.0)))
    rep["w_x_sample"] = rel_weight_err_log(lwb + ll["log_iota"][idx], lwb + li)
    # PF and noise likelihoods on the sample (weights normalised over it)
    dk = (mwb.log_kappa1 - mwb.log_kappa0[:, :, None]).sum(1)
    rep["w_y_sample"] = max(rel_weight_err_log(np.log(pred.w_alpha[s, idx]) + ll["delta_kappa"][s, idx],
                                               np.log(pred.w_alpha[s, idx]) + dk[s]) for s in range(pred.S))
    rep["w_eta_sample"] = max(rel_weight_err_log(np.log(pred.w_xi[j, idx]) + ll["log_nu"][j, idx],
                                                 np.log(pred.w_xi[j, idx]) + mwb.log_nu[j]) for j in range(g.J))
    print(rep)
    for key in ("m", "mw", "mu3", "mu4"):
        assert rep["table_" + key] < 1e-5, rep
    assert np.all(np.abs(ll["llr_omega"] - lo) < 1e-4 + 1e-7 * np.abs(lo)), rep
    assert rep["p_pr"] < P_TOL, rep
    assert rep["log_iota_selected"] < 1e-4 and rep["log_iota_fp32_over_bound"] <= 1.0, rep
    assert rep["w_x_sample"] < W_TOL and rep["w_y_sample"] < W_TOL and rep["w_eta_sample"] < W_TOL, rep
    # properties at full size
    assert np.all(np.isfinite(gw["w_x"])) and abs(gw["w_x"].sum() - 1.0) < 1e-12
    assert np.all((gw["p_s"] >= 0) & (gw["p_s"] <= 1 + 1e-12))
    assert np.allclose(gw["w_y"][:pred.S].sum(axis=1), gw["p_s"][:pred.S], rtol=1e-10, atol=1e-15)
