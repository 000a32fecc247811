"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Stage-wise from identical inputs (the seeded generator of
paper_2604_19723_gb300.workload), so that FP32 rounding of one stage does not
feed the next.  Tolerances: 1e-5 absolute on existence
probabilities, 1e-4 relative on normalised weights (max_p |dw_p| / max_p w_p),
1e-4 on posterior means (m, m/s; relative for gamma, mu, eta).
"""
import math

import numpy as np
import pytest

from oracle import beliefs, messages_dense, messages_woodbury, model, resample, rng, synth
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


def setup_case(geom_kw, K, S, P, seed, pos_std=0.005, snr_db=20.0, params=None, uniform=True, J=None):
    g = W.make_geometry(**geom_kw)
    prm = params or W.Params()
    scn = W.make_scenario(g, prm, N=3, K=K, seed=seed, snr_db=snr_db)
    eta = synth.noise_variance(scn)
    # the observation as the C ABI takes it (complex64), for both sides
    z = synth.observe(scn, 1, eta, seed + 100).astype(np.complex64).astype(np.complex128)
    st = W.state_near_truth(scn, P=P, S=S, n=0, seed=seed + 1, eta_true=eta, pos_std=pos_std,
                            sfv_std=pos_std, uniform_weights=uniform)
    return g, prm, scn, eta, z, st


def gpu_update_from(pred, g, prm, z, P, S_max, seed):
    f = bp.Filter(g, prm, P=P, S_max=S_max, seed=seed)
    f.set_predicted(pred.n, pred.S, pred.x, pred.phi, pred.eta, pred.w_beta, pred.w_alpha, pred.w_xi, pred.zeta)
    zd = torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda()
    f.update(zd)
    torch.cuda.synchronize()
    return f


CASES = [
    # (geometry, K true surfaces, S PFs, P, seed, pos_std)
    (dict(J=1, Nf=10, My=4, Mz=4), 4, 5, 512, 11, 0.005),         # one PA, Nz = 160, LoS + 4 walls
    (dict(J=4, Nf=10, My=4, Mz=4), 4, 5, 700, 12, 0.003),         # paper shape, ragged P
    (dict(J=2, Nf=6, My=3, Mz=2), 3, 4, 333, 13, 0.01),           # odd sizes, Nz = 36
    (dict(J=3, Nf=10, My=4, Mz=4), 10, 12, 300, 14, 0.004),       # S bucket 16
    (dict(J=4, Nf=10, My=4, Mz=4), 63, 64, 256, 15, 0.005),       # 64 PFs: float-float likelihoods for all particles
]


def s_max_for(S):
    return 16 if S <= 16 else 64


@pytest.mark.parametrize("case", CASES)
def test_predict_parity(case):
    geom_kw, K, S, P, seed, pos = case
    g, prm, scn, eta, z, st = setup_case(geom_kw, K, S, P, seed, pos)
    f = bp.Filter(g, prm, P=P, S_max=s_max_for(S), seed=seed)
    f.set_state(st)
    f.predict()
    gp = f.get_predicted()
    op = model.predict(st, prm, g.J, seed=seed, S_max=s_max_for(S))
    assert gp["S"] == op.S
    scale = np.maximum(np.abs(op.x.astype(float)), 1.0)
    assert np.max(np.abs(gp["x"] - op.x) / scale) < 1e-6
    assert np.max(np.abs(gp["eta"] - op.eta) / op.eta) < 1e-6
    ph_g, ph_o = gp["phi"].astype(float), op.phi.astype(float)
    for k in range(6):
        sc = np.maximum(np.abs(ph_o[:, k]), 1e-3 if k >= 3 else 1.0)
        assert np.max(np.abs(ph_g[:, k] - ph_o[:, k]) / sc) < 2e-6, k
    assert np.allclose(gp["w_alpha"], op.w_alpha, rtol=1e-14, atol=0)
    assert np.allclose(gp["zeta"], op.zeta, rtol=1e-14, atol=0)
    f.close()


@pytest.mark.parametrize("case", CASES)
def test_update_parity(case):
    geom_kw, K, S, P, seed, pos = case
    g, prm, scn, eta, z, st = setup_case(geom_kw, K, S, P, seed, pos)
    pred = model.predict(st, prm, g.J, seed=seed, S_max=s_max_for(S))
    f = gpu_update_from(pred, g, prm, z, P, s_max_for(S), seed)
    msg = messages_woodbury.update_messages(pred, prm, g, z)
    bel = beliefs.beliefs(pred, msg)
    est = beliefs.estimate(pred, bel, prm)
    # message table
    tab = f.diag_table(pred.S)
    for key in ("m", "mw", "mu3", "mu4"):
        ref = getattr(msg.table, key)
        err = np.max(np.abs(tab[key] - ref)) / max(np.max(np.abs(ref)), 1e-300)
        assert err < 1e-5, (key, err)
    assert np.allclose(tab["W"], msg.table.W, rtol=1e-12)
    assert np.allclose(tab["eta_bar"], msg.table.eta_bar, rtol=1e-12)
    # existence probabilities
    gw = f.diag_weights(pred.S)
    assert np.max(np.abs(gw["p_pr"] - bel.p_pr)) < P_TOL, np.max(np.abs(gw["p_pr"] - bel.p_pr))
    assert np.max(np.abs(gw["p_s"] - bel.p_s)) < P_TOL, np.max(np.abs(gw["p_s"] - bel.p_s))
    # normalised weights
    assert rel_weight_err(gw["w_x"], bel.w_x) < W_TOL, rel_weight_err(gw["w_x"], bel.w_x)
    for j in range(g.J):
        assert rel_weight_err(gw["w_eta"][j], bel.w_eta[j]) < W_TOL
    for s in range(pred.S):
        e = rel_weight_err(gw["w_y"][s], bel.w_y[s])
        assert e < W_TOL, (s, e)
    # posterior means
    ge = f.estimate()
    assert np.max(np.abs(ge["x_hat"] - est.x_hat)) < M_TOL
    assert np.max(np.abs(ge["eta_hat"] - est.eta_hat) / est.eta_hat) < M_TOL
    for s in range(pred.S):
        if est.p_s[s] > 1e-3:
            assert np.max(np.abs(ge["phi_hat"][s, :3] - est.phi_hat[s, :3])) < M_TOL
            assert abs(ge["phi_hat"][s, 3] - est.phi_hat[s, 3]) <= M_TOL * max(abs(est.phi_hat[s, 3]), 1e-12)
    f.close()


@pytest.mark.parametrize("S, los_existence", [(25, 1e-24), (25, 0.5)])
def test_update_parity_near_duplicate_pfs(S, los_existence):
    """A map that carries several PFs per surface (six per wall here, 5 mm apart), the
    state the filter passes through while births outnumber surfaces, optionally with a
    LoS whose existence has decayed to 1e-24.  The Gram matrix B = I + M^H M / eta_bar of
    the table stage then has one large eigenvalue per surface and a cluster of
    eigenvalues within 1e-6 of 1; its eigen-decomposition must resolve the pairs of the
    large eigenvalues to FP64 accuracy (an early convergence test on the total
    off-diagonal energy left them at 1e-2 relative: PR existence tests off by 0.1-3 nats
    and NaN)."""
    g, prm, scn, eta, z, st = setup_case(dict(J=4, Nf=10, My=4, Mz=4), 4, S, 700, 16, 0.005)
    st.w_y[0] *= los_existence / st.w_y[0].sum()
    pred = model.predict(st, prm, g.J, seed=16, S_max=64)
    f = gpu_update_from(pred, g, prm, z, 700, 64, 16)
    msg = messages_woodbury.update_messages(pred, prm, g, z)
    bel = beliefs.beliefs(pred, msg)
    ll = f.diag_loglik(pred.S)
    lo = msg.log_omega1 - msg.log_omega0
    gw = f.diag_weights(pred.S)
    d_llr = np.abs(ll["llr_omega"] - lo)
    d_pr = np.abs(gw["p_pr"] - bel.p_pr)
    d_ps = np.abs(gw["p_s"] - bel.p_s)
    d_w = [rel_weight_err(gw["w_y"][s], bel.w_y[s]) for s in range(pred.S) if bel.p_s[s] > 1e-12]
    report = dict(llr=d_llr.max(), p_pr=d_pr.max(), p_s=d_ps.max(), w_x=rel_weight_err(gw["w_x"], bel.w_x),
                  w_y=max(d_w))
    print(report)
    assert np.all(np.isfinite(ll["llr_omega"]))
    # the test's terms are FP64 arithmetic on the FP32-accumulated table (2e-7 relative),
    # of size |m|^2/eta_bar ~ 1e3-1e4 and cancelling to O(1) for a PF whose m-vector lies
    # almost in the span of its duplicates': 1e-4 absolute (+1e-7 relative) on the log
    # ratio, hence |d p| <= p (1 - p) |d llr| <= 2.5e-5 on the PR existence
    assert np.all(d_llr < 1e-4 + 1e-7 * np.abs(lo)), report
    assert np.all(d_pr <= 0.25 * (1e-4 + 1e-7 * np.abs(lo)) + 1e-12), report
    assert report["p_s"] < P_TOL, report
    assert report["w_x"] < W_TOL, report
    assert report["w_y"] < W_TOL, report
    f.close()


IOTA_BULK_CASES = [
    # (geometry, K, S, P, seed, pos_std): S >= 24 takes the FP32 bulk kernel and the selection
    (dict(J=4, Nf=10, My=4, Mz=4), 63, 64, 777, 17, 0.005),      # 64 PFs, ragged P over many blocks
    (dict(J=2, Nf=6, My=3, Mz=2), 30, 33, 401, 18, 0.02),        # S = 33 (rows 33..63 padded), Nz = 36
    (dict(J=3, Nf=10, My=4, Mz=4), 26, 27, 300, 19, 0.01),       # S in the 32-row variant
]


@pytest.mark.parametrize("case", IOTA_BULK_CASES)
def test_iota_bulk_bounds_and_selection(case):
    """Per-particle log iota sums against the FP64 oracle.  Particles evaluated in
    float-float agree to 1e-4; every other particle's FP32 value lies within its
    reported error bound, and its weight error, e^(lw_p - max lw) (e^|d_p| - 1), stays
    below e^-23 of the largest weight (the selection targets e^-24 from bounds)."""
    geom_kw, K, S, P, seed, pos = case
    g, prm, scn, eta, z, st = setup_case(geom_kw, K, S, P, seed, pos)
    z = z.astype(np.complex64).astype(np.complex128)    # the observation as the C ABI takes it
    pred = model.predict(st, prm, g.J, seed=seed, S_max=64)
    f = gpu_update_from(pred, g, prm, z, P, 64, seed)
    ll = f.diag_loglik(pred.S)["log_iota"]
    di = f.diag_iota()
    msg = messages_woodbury.update_messages(pred, prm, g, z)
    ref = msg.log_iota.sum(0)
    sel = np.zeros(P, bool)
    sel[di["selected"]] = True
    d = np.abs(ll - ref)
    report = dict(selected=int(sel.sum()), sel_err=float(d[sel].max()) if sel.any() else 0.0,
                  bulk_err=float(d[~sel].max()) if (~sel).any() else 0.0,
                  bound_min_margin=float(np.min(di["err"][~sel] - d[~sel])) if (~sel).any() else 0.0,
                  max_bound=float(np.max(di["err"][~sel])) if (~sel).any() else 0.0,
                  max_err_over_bound=float(np.max(d[~sel] / di["err"][~sel])) if (~sel).any() else 0.0)
    print(report)
    assert sel.any()
    assert np.all(d[sel] < 1e-4), report
    assert np.all(d[~sel] <= di["err"][~sel]), report
    lw = np.log(pred.w_beta) + ref
    werr = np.exp(lw - lw.max()) * np.expm1(d)
    assert np.all(werr[~sel] <= math.exp(-23.0)), report
    gw = f.diag_weights(pred.S)
    bel = beliefs.beliefs(pred, msg)
    assert rel_weight_err(gw["w_x"], bel.w_x) < W_TOL, rel_weight_err(gw["w_x"], bel.w_x)
    f.close()


def test_loglik_parity_dense():
    """Per-particle log-likelihoods against the dense (explicit covariance) definition."""
    g, prm, scn, eta, z, st = setup_case(dict(J=2, Nf=4, My=2, Mz=2), 3, 4, 96, 21, 0.02)
    pred = model.predict(st, prm, g.J, seed=21, S_max=8)
    f = gpu_update_from(pred, g, prm, z, 96, 8, 21)
    ll = f.diag_loglik(pred.S)
    msg = messages_dense.update_messages(pred, prm, g, z)
    li = msg.log_iota.sum(0)
    assert np.max(np.abs(ll["log_iota"] - li)) < 1e-3 * max(1.0, np.max(np.abs(li)) * 1e-3)
    dk = (msg.log_kappa1 - msg.log_kappa0[:, :, None]).sum(1)
    assert np.max(np.abs(ll["delta_kappa"] - dk)) < 2e-3
    # FP32 accumulation of the message table bounds this at ~1e-7 relative
    assert np.max(np.abs(ll["log_nu"] - msg.log_nu) / np.maximum(1, np.abs(msg.log_nu))) < 1e-6
    # the PR test is FP64 arithmetic on an FP32-accumulated table: its terms are of
    # size |z|^2/eta ~ 1e4 with ~1e-8 relative error, so 1e-4 absolute (+1e-7 relative);
    # the resulting p_s^(j) is held to 1e-5 absolute in test_update_parity
    lo = msg.log_omega1 - msg.log_omega0
    assert np.all(np.abs(ll["llr_omega"] - lo) < 1e-4 + 1e-7 * np.abs(lo))
    f.close()


def test_zero_mean_variant_parity():
    prm = W.Params(zero_mean=1)
    g, prm, scn, eta, z, st = setup_case(dict(J=2, Nf=10, My=4, Mz=4), 4, 5, 400, 31, 0.005, params=prm)
    st.phi[:, 4:] = 0.0
    pred = model.predict(st, prm, g.J, seed=31, S_max=8)
    f = gpu_update_from(pred, g, prm, z, 400, 8, 31)
    bel = beliefs.beliefs(pred, messages_woodbury.update_messages(pred, prm, g, z))
    gw = f.diag_weights(pred.S)
    assert rel_weight_err(gw["w_x"], bel.w_x) < W_TOL
    assert np.max(np.abs(gw["p_s"] - bel.p_s)) < P_TOL
    f.close()


def test_resampling_indices_valid_and_match():
    """GPU indices are valid for the GPU's own weights (first index whose CDF reaches
    u_i = (U + i)/P; checked with plain numpy), and equal the oracle's indices, computed
    from the oracle's weights, except where u_i lies within the weight tolerance of a
    CDF step (near-ties may resolve either way)."""
    g, prm, scn, eta, z, st = setup_case(dict(J=2, Nf=6, My=3, Mz=2), 3, 4, 1000, 41, 0.05)
    prm.T_pru = 0.0
    pred = model.predict(st, prm, g.J, seed=41, S_max=8)
    f = gpu_update_from(pred, g, prm, z, 1000, 8, 41)
    gw = f.diag_weights(pred.S)
    gi = f.diag_indices(pred.S)
    bel = beliefs.beliefs(pred, messages_woodbury.update_messages(pred, prm, g, z))
    P = 1000
    beliefs_list = [(gw["w_x"], bel.w_x, gi["x"], (0, 0))]
    beliefs_list += [(gw["w_eta"][j], bel.w_eta[j], gi["eta"][j], (2, j)) for j in range(g.J)]
    beliefs_list += [(gw["w_y"][s], bel.w_y[s], gi["y"][s], (1, s)) for s in range(pred.S)]
    for w_gpu, w_ref, idx, (kind, index) in beliefs_list:
        U = resample.resample_uniform(41, pred.n, kind, index)
        u = (U + np.arange(P)) / P
        c = np.cumsum(w_gpu) / np.sum(w_gpu)
        c[-1] = 1.0
        assert np.all(c[idx] >= u - 1e-12)
        prev = np.where(idx > 0, c[np.maximum(idx - 1, 0)], 0.0)
        assert np.all(prev < u + 1e-12)
        ref = resample.systematic_indices(w_ref, U)
        cr = np.cumsum(w_ref) / np.sum(w_ref)
        for i in np.nonzero(idx != ref)[0]:
            k = min(idx[i], ref[i])
            assert abs(cr[k] - u[i]) < W_TOL, (kind, index, i)
        assert np.mean(idx != ref) < 0.01


def _close_fp32(a, b, base, jit, rel=1e-5):
    """a equals b = resampled value + jitter up to FP32 rounding of operands of the size
    of `base`, plus rel of the jitter (FP32 bandwidth factor and products)."""
    sp = 4.0 * np.spacing(np.abs(np.asarray(base, np.float32))).astype(np.float64)
    return np.abs(a - b) <= rel * np.abs(jit) + sp + 1e-12


def _jitter_terms(X, w, active, seed, n, purpose, sub, P):
    """h_opt |L| |eps|: the size of the summands of every jitter component (FP32 rounding
    in the kernel is relative to them, not to their sum)."""
    C = resample.weighted_cov(X.astype(np.float64), w)
    C[~active, :] = 0.0
    C[:, ~active] = 0.0
    L = resample.cholesky_zeroing(C)
    eps = np.array(rng.normals(seed, np.arange(P, dtype=np.uint64), n, purpose, sub, X.shape[0]))
    return resample.h_opt(P, int(active.sum())) * (np.abs(L) @ np.abs(eps))


def _worst(a, b, base, jit, rel=1e-5):
    """The worst violation of _close_fp32: (index, a, b, allowed)."""
    sp = 4.0 * np.spacing(np.abs(np.asarray(base, np.float32))).astype(np.float64)
    tol = rel * np.abs(jit) + sp + 1e-12
    k = np.unravel_index(np.argmax(np.abs(a - b) - tol), np.shape(a))
    return k, float(np.asarray(a)[k]), float(np.asarray(b)[k]), float(tol[k])


def test_full_step_resample_and_jitter_per_particle():
    """One complete step (predict, update, resample, regularise), checked particle by
    particle (Sec. IV-D: systematic resampling, Gaussian-kernel regularisation after
    Musso et al.).  The oracle's resampling rule and jitter h_opt L eps_i (same Philox
    draws eps_i, L L^T the weighted covariance) are applied to the inputs the kernels
    used, the GPU's predicted particles and normalised weights, which the update-parity
    tests hold to the oracle's within 1e-4: every output particle must then equal its
    resampled particle plus its jitter up to FP32 rounding.  The estimates and the
    resampled clouds are also compared with the oracle's own step."""
    g, prm, scn, eta, z, st = setup_case(dict(J=2, Nf=10, My=4, Mz=4), 4, 5, 600, 51, 0.004)
    P, seed = 600, 51
    f = bp.Filter(g, prm, P=P, S_max=16, seed=seed)
    f.set_state(st)
    zd = torch.from_numpy(z.astype(np.complex64)).cuda()
    f.predict()
    pg = f.get_predicted()
    f.update(zd)
    gw = f.diag_weights(pg["S"])
    gi = f.diag_indices(pg["S"])
    new = f.get_state()
    ge = f.estimate()
    n = pg["n"]
    # the oracle's own step from the GPU-independent prediction of the same state
    op = model.predict(st, prm, g.J, seed=seed, S_max=16)
    msg = messages_woodbury.update_messages(op, prm, g, z)
    bel = beliefs.beliefs(op, msg)
    est = beliefs.estimate(op, bel, prm)
    keep = beliefs.survivors(est, prm)
    ost, *_ = resample.resample_and_regularize(op, bel, keep, prm, seed)
    assert new.S == ost.S == len(keep)
    assert np.max(np.abs(ge["x_hat"] - est.x_hat)) < 1e-4
    assert np.max(np.abs(ge["p_s"] - est.p_s)) < 1e-5
    assert np.allclose(new.w_x, 1.0 / P) and np.allclose(new.w_eta, 1.0 / P)
    assert np.allclose(new.w_y.sum(1), ost.w_y.sum(1), atol=1e-5)
    # MT: indices by the systematic rule on the GPU's weights, particles = resampled + jitter
    X = pg["x"].astype(np.float64)
    U = resample.resample_uniform(seed, n, 0, 0)
    idx = resample.systematic_indices(gw["w_x"], U)
    assert np.mean(idx == gi["x"]) > 0.999
    jit = resample._jitter(X, gw["w_x"], resample.mt_active(prm), seed, n, rng.JITTER_MT, 0, P)
    assert np.max(np.abs(jit)) > 0.0
    ref = X[:, gi["x"]] + jit
    jt = _jitter_terms(X, gw["w_x"], resample.mt_active(prm), seed, n, rng.JITTER_MT, 0, P)
    base = np.abs(X[:, gi["x"]]) + jt                        # FP32 rounding is relative to the operands
    assert np.all(_close_fp32(new.x.astype(np.float64), ref, base, jt)), _worst(new.x.astype(np.float64), ref, base, jt)
    # PFs, compacted in keep order; gamma (row 3) is reflected at 0
    for t, s in enumerate(keep):
        Y = pg["phi"][s].astype(np.float64)
        w = gw["w_y"][s]
        ii = resample.systematic_indices(w / w.sum(), resample.resample_uniform(seed, n, 1, int(s)))
        assert np.mean(ii == gi["y"][s]) > 0.999, s
        jit = resample._jitter(Y, w, resample.pf_active(prm, s), seed, n, rng.JITTER_PF, int(s), P)
        ref = Y[:, gi["y"][s]] + jit
        ref[3] = np.abs(ref[3])
        jt = _jitter_terms(Y, w, resample.pf_active(prm, s), seed, n, rng.JITTER_PF, int(s), P)
        base = np.abs(Y[:, gi["y"][s]]) + jt
        assert np.all(_close_fp32(new.phi[t].astype(np.float64), ref, base, jt)), \
            (s, _worst(new.phi[t].astype(np.float64), ref, base, jt))
    # noise variances, reflected at 0
    for j in range(g.J):
        E = pg["eta"][j].astype(np.float64)
        ii = resample.systematic_indices(gw["w_eta"][j], resample.resample_uniform(seed, n, 2, j))
        assert np.mean(ii == gi["eta"][j]) > 0.999, j
        jit = resample._jitter(E[None], gw["w_eta"][j], np.ones(1, bool), seed, n, rng.JITTER_ETA, j, P)[0]
        ref = np.abs(E[gi["eta"][j]] + jit)
        jt = _jitter_terms(E[None], gw["w_eta"][j], np.ones(1, bool), seed, n, rng.JITTER_ETA, j, P)[0]
        base = np.abs(E[gi["eta"][j]]) + jt
        assert np.all(_close_fp32(new.eta[j].astype(np.float64), ref, base, jt)), \
            (j, _worst(new.eta[j].astype(np.float64), ref, base, jt))
    # the clouds against the oracle's own step (weights within 1e-4: statistics agree)
    assert np.allclose(new.x.mean(1), ost.x.mean(1), atol=2e-3)
    f.close()


def test_multi_step_run_with_births_and_pruning():
    wl = W.workload("small_fp64")
    g, prm = wl["geom"], wl["params"]
    scn = W.make_scenario(g, prm, N=6, K=4, seed=5, clutter_mean=2.0, visibility=0.9)
    x_pos, sfv, rho, cc, cs, cr = bp.scenario_arrays(scn, range(1, 7))
    zall, eta = bp.synthesize(g, x_pos, sfv, rho, cc, cs, cr, snr_db=20.0, seed=9, step0=1)
    f = bp.Filter(g, prm, P=2000, S_max=16, seed=3)
    for n in range(6):
        f.step(zall[n])
        e = f.estimate()
        assert e["n"] == n + 1
        assert 1 <= e["S_next"] <= e["S"] <= 16
        assert np.all((e["p_s"] >= 0) & (e["p_s"] <= 1 + 1e-12))
        assert np.all(np.isfinite(e["x_hat"]))
    st = f.get_state()
    assert np.allclose(st.w_x.sum(), 1.0) and np.all(np.isfinite(st.x))
    assert f.launch_count() > 0
    f.close()


def test_synthesize_matches_oracle():
    g = W.make_geometry(J=2, Nf=10, My=4, Mz=4)
    prm = W.Params()
    scn = W.make_scenario(g, prm, N=3, K=4, seed=2, clutter_mean=3.0, visibility=0.8, snr_db=20.0)
    x_pos, sfv, rho, cc, cs, cr = bp.scenario_arrays(scn, range(1, 4))
    zg, eta_g = bp.synthesize(g, x_pos, sfv, rho, cc, cs, cr, snr_db=20.0, seed=77, step0=1)
    eta_o = synth.noise_variance(scn)
    assert eta_g == pytest.approx(eta_o, rel=1e-10)
    zg = zg.cpu().numpy()
    for t, n in enumerate(range(1, 4)):
        zo = synth.observe(scn, n, eta_o, 77)
        assert np.max(np.abs(zg[t] - zo)) < 1e-6 * np.max(np.abs(zo))


def test_invalid_arguments_fail_loudly():
    g = W.make_geometry(J=1, Nf=2, My=2, Mz=1)
    with pytest.raises(bp.BPError):
        bp.Filter(g, W.Params(), P=10, S_max=65, seed=0)
    with pytest.raises(bp.BPError):
        bp.Filter(g, W.Params(c_eta=0.5), P=10, S_max=4, seed=0)
    f = bp.Filter(g, W.Params(), P=16, S_max=4, seed=0)
    z = torch.zeros((1, g.Nz), dtype=torch.complex64, device="cuda")
    with pytest.raises(bp.BPError):
        f.update(z)           # update before predict
    f.close()
