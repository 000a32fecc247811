"""Parity at the full size of the 64-PF workload (64 PFs x 100000 particles, J = 4,
Nz = 160), through the same C ABI call and launch configuration the benchmark times.

The message table is a sum over every particle, so the oracle computes it in full
(chunked, in a spawn process pool).  The per-particle log-likelihoods are then
checked on a sample of particles, which the oracle evaluates one by one with the
dense (explicit covariance) definition.  The sample holds the particles nearest the
true state (chosen from the seeded state, where the weight is), particles spread
over the whole range, and the ragged last one.  The bound is the stated one on
normalised weights, max_p |dw_p| / max_p w_p < 1e-4, with the weights normalised
over the sample (a particle far from the truth has a log-likelihood 1e3-1e4 below
the best one, FP32 rounding of 1e-7 relative on that scale, and a weight that is
zero to any precision).  Everything else is checked through properties that hold
at any size.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import messages_dense, model, synth
from paper_2604_19723_gb300 import workload as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import bp  # noqa: E402,F401

W_TOL = 1e-4


def sub_pred(pred, idx):
    return model.Predicted(n=pred.n, S=pred.S, x=pred.x[:, idx], phi=pred.phi[:, :, idx], eta=pred.eta[:, idx],
                           w_beta=pred.w_beta[idx], w_alpha=pred.w_alpha[:, idx], w_xi=pred.w_xi[:, idx],
                           zeta=pred.zeta, is_new=pred.is_new)


def rel_weight_err(log_a, log_b):
    """max |dw| / max w of the weights exp(log_a), exp(log_b) normalised over the sample."""
    wa = np.exp(log_a - np.max(log_a))
    wb = np.exp(log_b - np.max(log_b))
    wa, wb = wa / wa.sum(), wb / wb.sum()
    return float(np.max(np.abs(wa - wb)) / np.max(wb))


@pytest.fixture(scope="module")
def pool():
    # one BLAS thread per worker (the children read these at import)
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


def test_full_size_64pf_sampled(pool):
    wl = W.workload("scale_64x100k")
    g, prm, P, S, S_max = wl["geom"], wl["params"], wl["P"], wl["fixed_S"], wl["S_max"]
    scn = W.make_scenario(g, prm, N=3, K=wl["K"], seed=wl["seed"], snr_db=wl["snr_db"],
                          visibility=wl["visibility"], clutter_mean=wl["clutter_mean"])
    eta = synth.noise_variance(scn)
    # the observation as the C ABI takes it (complex64), for both sides: its rounding alone
    # moves |r|^2 / eta_bar by ~1e-2 at this residual energy
    z = synth.observe(scn, 1, eta, wl["seed"] + 100).astype(np.complex64).astype(np.complex128)
    st = W.state_near_truth(scn, P=P, S=S, n=0, seed=wl["seed"] + 5, eta_true=eta, pos_std=0.01, sfv_std=0.01)
    pred = model.predict(st, prm, g.J, seed=wl["seed"], S_max=S_max)
    tab = messages_dense.message_table_streamed(pred, prm, g, chunk=4096, pool=pool)

    f = bp.Filter(g, prm, P=P, S_max=S_max, seed=wl["seed"])
    f.set_predicted(pred.n, pred.S, pred.x, pred.phi, pred.eta, pred.w_beta, pred.w_alpha, pred.w_xi, pred.zeta)
    zd = torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda()
    f.update(zd)
    torch.cuda.synchronize()
    gt = f.diag_table(pred.S)
    ll = f.diag_loglik(pred.S)
    gw = f.diag_weights(pred.S)
    di = f.diag_iota()
    f.close()

    # message table over all 100000 particles (FP32 chunk sums, FP64 across chunks)
    for key in ("m", "mw", "mu3", "mu4"):
        ref = getattr(tab, key)
        err = np.max(np.abs(gt[key] - ref)) / max(np.max(np.abs(ref)), 1e-300)
        assert err < 1e-5, (key, err)
    assert np.allclose(gt["eta_bar"], tab.eta_bar, rtol=1e-12)

    # MT likelihoods: the MT posterior is sharply peaked, so the oracle scores the 200
    # particles nearest the truth and the 16 it weighs highest are compared (with a
    # spread of other particles, whose weights are negligible)
    dist = np.linalg.norm(pred.x[:3].astype(np.float64).T - scn.x_true[1, :3], axis=1)
    cand = np.argsort(dist)[:200]
    spc = sub_pred(pred, cand)
    psic = messages_dense.all_steering(spc, g)
    lic = np.log(pred.w_beta[cand]) + sum(messages_dense.log_iota(spc, tab, psic, z, j) for j in range(g.J))
    top = cand[np.argsort(-lic)[:16]]
    idx_i = np.unique(np.r_[top, np.linspace(0, P - 1, 8).astype(int), P - 1])
    spi = sub_pred(pred, idx_i)
    li = sum(messages_dense.log_iota(spi, tab, messages_dense.all_steering(spi, g), z, j) for j in range(g.J))
    lwb = np.log(pred.w_beta[idx_i])
    e = rel_weight_err(lwb + ll["log_iota"][idx_i], lwb + li)
    assert e < W_TOL, e
    # the log iota sums themselves, particle by particle (not only through the weights,
    # which a sharply peaked posterior would forgive): the particles evaluated in
    # float-float agree to 1e-4; every other one lies within its FP32 error bound and
    # its weight error e^(lw - max lw) (e^|d| - 1) stays below e^-23 of the largest
    sel = np.zeros(P, bool)
    sel[di["selected"]] = True
    d_i = np.abs(ll["log_iota"][idx_i] - li)
    lw_all = np.log(pred.w_beta) + ll["log_iota"]
    best = int(np.argmax(lw_all))                 # the largest weight (float-float, within 1e-4)
    rel = lwb + li - lw_all[best]
    s_i = sel[idx_i]
    print(dict(selected=int(sel.sum()), sample_selected=int(s_i.sum()), sel_err=float(d_i[s_i].max())))
    assert sel[best]
    assert np.all(d_i[s_i] < 1e-4), d_i[s_i]
    assert np.all(d_i[~s_i] <= di["err"][idx_i][~s_i])
    assert np.all(np.exp(rel[~s_i]) * np.expm1(d_i[~s_i]) <= np.exp(-23.0))

    # PF and noise likelihoods: particles nearest the truth, a spread, the ragged last one
    idx = np.unique(np.r_[np.argsort(dist)[:24], np.linspace(0, P - 1, 16).astype(int), P - 1])
    sp = sub_pred(pred, idx)
    psi = messages_dense.all_steering(sp, g)
    for s in range(pred.S):
        dk = np.zeros(len(idx))
        for j in range(g.J):
            l1, l0 = messages_dense.log_kappa(sp, tab, psi, z, s, j)
            dk += l1 - l0
        lwa = np.log(pred.w_alpha[s, idx])
        e = rel_weight_err(lwa + ll["delta_kappa"][s, idx], lwa + dk)
        assert e < W_TOL, (s, e)
    for j in range(g.J):
        # the FP32-accumulated table shifts log nu by a near-common offset (~1e-7 relative)
        ln = messages_dense.log_nu(sp, tab, z, j)
        lwx = np.log(pred.w_xi[j, idx])
        e = rel_weight_err(lwx + ll["log_nu"][j, idx], lwx + ln)
        assert e < W_TOL, (j, e)
    for s in range(pred.S):
        for j in range(g.J):
            l1, l0 = messages_dense.log_omega(tab, z, s, j)
            assert abs(ll["llr_omega"][s, j] - (l1 - l0)) < 1e-4 + 1e-7 * abs(l1 - l0), (s, j)

    # properties of the normalised beliefs at full size
    assert np.all(np.isfinite(gw["w_x"])) and abs(gw["w_x"].sum() - 1.0) < 1e-12
    for j in range(g.J):
        assert abs(gw["w_eta"][j].sum() - 1.0) < 1e-12
    assert np.all((gw["p_s"] >= 0) & (gw["p_s"] <= 1 + 1e-12))
    assert np.allclose(gw["w_y"][:pred.S].sum(axis=1), gw["p_s"][:pred.S], rtol=1e-10, atol=1e-15)
