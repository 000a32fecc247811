"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails it.  No value here comes
from the CUDA path.
"""
import math

import numpy as np
import pytest
import scipy.stats as st

from conftest import load_kat
from oracle import beliefs, brute, geometry, messages_dense, messages_woodbury, model, resample, rng, synth
from paper_2604_19723_gb300 import workload as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- random numbers
def test_philox_known_answers():
    for ctr, key, expect in load_kat():
        out = rng.philox4x32_10(*ctr, *key)
        assert [int(v) for v in out] == expect


def test_box_muller_is_standard_normal():
    idx = np.arange(200000, dtype=np.uint64)
    g = np.concatenate(rng.normals4(42, idx, 3, rng.MT_PREDICT, 0, 0))
    assert abs(g.mean()) < 5 / math.sqrt(len(g))
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0 / len(g))
    assert st.kstest(g, "norm").pvalue > 1e-3


@pytest.mark.parametrize("shape", [1.0, 3.5, 100.0])
def test_gamma_sampler_moments_and_law(shape):
    """P6: Gamma(c, eta/c) keeps the mean eta and has variance eta^2/c."""
    idx = np.arange(100000, dtype=np.uint64)
    eta = 2.5e-8
    g = rng.gamma(7, idx, 1, rng.ETA_PREDICT, 0, shape, eta / shape)
    assert abs(g.mean() / eta - 1.0) < 5 * math.sqrt(1.0 / shape / len(g))
    assert abs(g.var() / (eta * eta / shape) - 1.0) < 0.05
    assert st.kstest(g / (eta / shape), "gamma", args=(shape,)).pvalue > 1e-3


def test_birth_probability():
    """P6: Bernoulli birth p_B = mu_B/(1 + mu_B) = 1/3 at mu_B = 0.5 (Sec. III-B2, V-A)."""
    assert model.birth_probability(0.5, 1) == pytest.approx(1.0 / 3.0, abs=1e-15)
    # ratio of the Poisson pmf at 1 and 0 equals p_B/(1 - p_B)
    for muB in (0.1, 0.5, 2.0):
        pB = model.birth_probability(muB, 1)
        assert pB / (1 - pB) == pytest.approx(st.poisson.pmf(1, muB) / st.poisson.pmf(0, muB), rel=1e-12)


# ---------------------------------------------------------------- geometry (P3)
def _geom(J=2, Nf=5, My=3, Mz=2):
    return W.make_geometry(J=J, Nf=Nf, My=My, Mz=Mz)


def test_householder_orthogonal_involutive():
    r = np.random.default_rng(0)
    for _ in range(10):
        p = r.normal(size=3) * 5
        H = geometry.householder(p)
        assert np.allclose(H @ H.T, np.eye(3), atol=1e-14)
        assert np.allclose(H @ H, np.eye(3), atol=1e-14)
        assert np.linalg.det(H) == pytest.approx(-1.0, abs=1e-13)
        assert np.allclose(H @ p, -p, atol=1e-12)


def test_virtual_anchor_is_mirror_image():
    """Sec. S-I: the wall has point p_sfv/2 and normal p_sfv/|p_sfv|; the VA mirrors the PA."""
    r = np.random.default_rng(1)
    for _ in range(10):
        p_sfv = r.normal(size=3) * 6
        p_pa = r.normal(size=3) * 2
        nvec = p_sfv / np.linalg.norm(p_sfv)
        mirror = p_pa - 2.0 * np.dot(p_pa - p_sfv / 2.0, nvec) * nvec
        assert np.allclose(geometry.virtual_anchor(p_pa, p_sfv), mirror, atol=1e-12)
        # the origin mirrored across the same wall is p_sfv itself
        assert np.allclose(geometry.virtual_anchor(np.zeros(3), p_sfv), p_sfv, atol=1e-12)


def test_los_local_vector():
    g = _geom()
    p = np.array([1.0, 2.0, 0.3])
    rp = geometry.local_vector(p, None, g.p_pa[1], g.R_pa[1], los=True)
    assert np.allclose(rp, g.R_pa[1].T @ (p - g.p_pa[1]), atol=1e-14)


def test_steering_elementwise_equals_kronecker():
    """Sec. S-II: the VA-layout planar-wavefront response equals eq. (unit-modulus-array-response)."""
    g = _geom()
    r = np.random.default_rng(2)
    pts = r.uniform([-3, -0.5, -0.8], [4, 4, 0.8], size=(7, 3))
    sfv = W.room_sfvs(W.Params().p_min, W.Params().p_max)
    for j in range(g.J):
        a = geometry.steering(g, j, pts, None, los=True)
        b = geometry.steering_kronecker(g, j, pts, None, los=True)
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))
        for k in range(4):
            sf = np.broadcast_to(sfv[k], pts.shape)
            a = geometry.steering(g, j, pts, sf, los=False)
            b = geometry.steering_kronecker(g, j, pts, sf, los=False)
            assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(a))


def test_steering_norm_and_unit_modulus():
    """|psi~_k| = 1 on the torus and |psi|^2 = Nz (lambda/(4 pi |r'|))^2 (eq. array-response)."""
    g = _geom()
    p = np.array([[0.5, 1.5, 0.2]])
    sfv = np.array([[8.8, 0.0, 0.0]])
    psi = geometry.steering(g, 0, p, sfv, los=False)[0]
    d = np.linalg.norm(geometry.local_vector(p[0], sfv[0], g.p_pa[0], g.R_pa[0], los=False))
    amp = g.wavelength / (4 * np.pi * d)
    assert np.allclose(np.abs(psi), amp, rtol=1e-13)
    assert np.sum(np.abs(psi) ** 2) == pytest.approx(g.Nz * amp * amp, rel=1e-13)


def test_planar_matches_spherical_in_far_field():
    """Sec. S-II: the planar wavefront approaches the spherical one far from the array (Nf = 1)."""
    g = W.make_geometry(J=1, Nf=1, My=4, Mz=4)
    errs = []
    for dist in (10.0, 100.0, 1000.0):
        p = g.p_pa[0] + dist * g.R_pa[0] @ np.array([0.8, 0.5, 0.33]) / np.linalg.norm([0.8, 0.5, 0.33])
        a = geometry.steering(g, 0, p[None], None, los=True)[0]
        b = geometry.steering_spherical(g, 0, p, None, los=True)
        errs.append(np.max(np.abs(a / b - 1)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-3


# ---------------------------------------------------------------- complex Gaussian density
def test_log_cn_matches_real_gaussian():
    """CN(z; m, C) equals the real 2N-dim normal of [Re z, Im z] with covariance [[Re C, -Im C], [Im C, Re C]]/2."""
    r = np.random.default_rng(3)
    N = 6
    A = r.normal(size=(N, N)) + 1j * r.normal(size=(N, N))
    C = A @ A.conj().T + 0.5 * np.eye(N)
    m = r.normal(size=N) + 1j * r.normal(size=N)
    z = r.normal(size=N) + 1j * r.normal(size=N)
    lc = messages_dense.log_cn(z[None], m[None], C[None])[0]
    Cr = 0.5 * np.block([[C.real, -C.imag], [C.imag, C.real]])
    lr = st.multivariate_normal(mean=np.r_[m.real, m.imag], cov=Cr).logpdf(np.r_[z.real, z.imag])
    assert lc == pytest.approx(lr, rel=1e-12)


# ---------------------------------------------------------------- moment matching (P1)
def _tiny_pred(S, P, seed, J=1, zero_mean=False):
    g = W.make_geometry(J=J, Nf=2, My=2, Mz=1)
    prm = W.Params(zero_mean=int(zero_mean))
    r = np.random.default_rng(seed)
    x = np.zeros((6, P), np.float32)
    x[:3] = r.uniform([-1, 0, -0.2], [2, 3, 0.2], size=(P, 3)).T
    phi = np.zeros((S, 6, P), np.float32)
    for s in range(1, S):
        phi[s, :3] = (W.room_sfvs(prm.p_min, prm.p_max)[s - 1][:, None]
                      + 0.2 * r.normal(size=(3, P))).astype(np.float32)
    phi[:, 3] = r.uniform(0.2, 1.5, size=(S, P))
    if not zero_mean:
        phi[:, 4] = r.normal(size=(S, P)) * 0.7
        phi[:, 5] = r.normal(size=(S, P)) * 0.7
    eta = r.uniform(0.5e-6, 2e-6, size=(J, P)).astype(np.float32)
    pred = model.Predicted(n=1, S=S, x=x, phi=phi, eta=eta,
                           w_beta=np.full(P, 1.0 / P), w_alpha=np.full((S, P), 1.0 / P) * r.uniform(0.2, 0.8, (S, 1)),
                           w_xi=np.full((J, P), 1.0 / P), zeta=r.uniform(0.1, 0.95, (S, J)),
                           is_new=np.zeros(S, bool))
    return g, prm, pred


@pytest.mark.parametrize("S", [1, 2, 3])
def test_moment_matching_equals_exact_mixture(S):
    """P1: for one paired particle the moment-matched messages (Proposition 1 with the
    S-V representations, sqrt(pi) reading of the m-vectors) equal the exact mean and
    covariance of the 2^(2S) existence mixture of eq. (Miota-exact)..(Momega-exact)."""
    g, prm, pred = _tiny_pred(S, 1, seed=10 + S)
    prm.mvec_scaling = 1
    psi = messages_dense.all_steering(pred, g)
    tab = messages_dense.message_table(pred, prm, psi)
    ps = psi[:, 0, 0]
    gam = pred.phi[:, 3, 0].astype(float)
    mu = pred.phi[:, 4, 0].astype(float) + 1j * pred.phi[:, 5, 0].astype(float)
    Wv = pred.w_alpha.sum(1)
    zeta = pred.zeta[:, 0]
    eb = tab.eta_bar[0]
    # iota: nothing conditioned
    m_ex, C_ex = brute.mixture_moments(ps, gam, mu, Wv, zeta, eb)
    m_o, C_o = messages_dense.iota_moments(pred, tab, psi, 0)
    assert np.allclose(m_o[0], m_ex, atol=1e-12 * np.abs(m_ex).max() + 1e-300)
    assert np.allclose(C_o[0], C_ex, atol=1e-12 * np.abs(C_ex).max())
    # nu: given eta (a single particle value)
    e1 = float(pred.eta[0, 0])
    m_ex, C_ex = brute.mixture_moments(ps, gam, mu, Wv, zeta, e1)
    m_o, C_o = messages_dense.nu_moments(tab, 0, e1)
    assert np.allclose(m_o, m_ex, atol=1e-12 * np.abs(m_ex).max() + 1e-300)
    assert np.allclose(C_o[0], C_ex, atol=1e-12 * np.abs(C_ex).max())
    for s in range(S):
        # kappa, r_s = 1 given
        m_ex, C_ex = brute.mixture_moments(ps, gam, mu, Wv, zeta, eb, fixed={("r", s): 1})
        m_o, C_o, mo, A = messages_dense.kappa_moments(pred, tab, psi, s, 0)
        assert np.allclose(m_o[0], m_ex, atol=1e-12 * np.abs(m_ex).max() + 1e-300)
        assert np.allclose(C_o[0], C_ex, atol=1e-12 * np.abs(C_ex).max())
        # kappa, r_s = 0 given
        m_ex, C_ex = brute.mixture_moments(ps, gam, mu, Wv, zeta, eb, fixed={("r", s): 0})
        assert np.allclose(mo, m_ex, atol=1e-12 * np.abs(C_ex).max())
        assert np.allclose(A, C_ex, atol=1e-12 * np.abs(C_ex).max())
        # omega, r_s^(j) = 1 given
        m_ex, C_ex = brute.mixture_moments(ps, gam, mu, Wv, zeta, eb, fixed={("rj", s): 1})
        m1, C1, m0, C0 = messages_dense.omega_moments(tab, s, 0)
        assert np.allclose(m1, m_ex, atol=1e-12 * np.abs(m_ex).max() + 1e-300)
        assert np.allclose(C1, C_ex, atol=1e-12 * np.abs(C_ex).max())


def test_printed_m_vectors_differ_from_sqrt_reading_by_sqrt_pi():
    """Reading R2: the S-V m-vectors (W zeta and W outside the square root) equal the
    exact-moment ones times sqrt(pi) = sqrt(zeta W) and sqrt(W) respectively."""
    g, prm, pred = _tiny_pred(3, 5, seed=4)
    psi = messages_dense.all_steering(pred, g)
    prm.mvec_scaling = 0
    a = messages_dense.message_table(pred, prm, psi)
    prm.mvec_scaling = 1
    b = messages_dense.message_table(pred, prm, psi)
    assert np.allclose(a.m, np.sqrt(b.pi)[:, :, None] * b.m, rtol=1e-13)
    assert np.allclose(a.mw, np.sqrt(b.W)[:, None, None] * b.mw, rtol=1e-13)
    assert np.allclose(a.mu3, b.mu3) and np.allclose(a.mu4, b.mu4)


def test_paired_sums_exact_when_one_belief_is_a_point_mass():
    """Reading R1/R3: the paired sum (sum w_alpha) sum_p w_beta f(x^p, phi^p) equals the
    double integral of mu^(3) when beta is a point mass and w_alpha is uniform."""
    g, prm, pred = _tiny_pred(2, 7, seed=5)
    pred.x[:] = pred.x[:, :1]                      # beta = delta(x - x0)
    pred.w_alpha[:] = pred.w_alpha[:, :1]          # uniform alpha weights
    psi = messages_dense.all_steering(pred, g)
    tab = messages_dense.message_table(pred, prm, psi)
    for s in range(2):
        mu = pred.phi[s, 4].astype(float) + 1j * pred.phi[s, 5].astype(float)
        exact = pred.zeta[s, 0] * np.einsum("p,p,pk->k", pred.w_alpha[s], mu, psi[s, 0])
        assert np.allclose(tab.mu3[s, 0], exact, rtol=1e-12)


# ---------------------------------------------------------------- low-rank forms (P2)
@pytest.mark.parametrize("zero_mean,scaling", [(False, 0), (True, 0), (False, 1)])
def test_woodbury_equals_dense(zero_mean, scaling):
    """P2: the S-V inversion/determinant-lemma forms equal the dense definition."""
    g = W.make_geometry(J=2, Nf=4, My=2, Mz=2)
    prm = W.Params(zero_mean=int(zero_mean), mvec_scaling=scaling)
    scn = W.make_scenario(g, prm, N=2, K=3, seed=8)
    eta = synth.noise_variance(scn)
    z = synth.observe(scn, 1, eta, 3)
    st0 = W.state_near_truth(scn, P=40, S=4, n=0, seed=2, eta_true=eta, pos_std=0.05)
    pred = model.predict(st0, prm, g.J, seed=9, S_max=8)
    a = messages_dense.update_messages(pred, prm, g, z)
    b = messages_woodbury.update_messages(pred, prm, g, z)
    for k in ("log_iota", "log_nu", "log_kappa1", "log_kappa0", "log_omega1", "log_omega0"):
        x, y = getattr(a, k), getattr(b, k)
        assert np.max(np.abs(x - y) / np.maximum(1.0, np.abs(x))) < 1e-10, k


@pytest.mark.parametrize("scaling", [0, 1])
def test_streamed_table_equals_table(scaling):
    """The chunked particle sums of message_table_streamed add up to message_table."""
    g = W.make_geometry(J=2, Nf=4, My=2, Mz=2)
    prm = W.Params(mvec_scaling=scaling)
    scn = W.make_scenario(g, prm, N=2, K=3, seed=8)
    eta = synth.noise_variance(scn)
    st0 = W.state_near_truth(scn, P=101, S=4, n=0, seed=2, eta_true=eta, pos_std=0.05)
    pred = model.predict(st0, prm, g.J, seed=9, S_max=8)
    a = messages_dense.message_table(pred, prm, messages_dense.all_steering(pred, g))
    b = messages_dense.message_table_streamed(pred, prm, g, chunk=16)
    for k in ("W", "pi", "m", "mw", "mu3", "mu4", "eta_bar"):
        x, y = getattr(a, k), getattr(b, k)
        assert np.max(np.abs(x - y)) <= 1e-12 * max(np.max(np.abs(x)), 1e-300), k


# ---------------------------------------------------------------- special cases (P4)
def test_zero_mean_variant_equals_nzm_with_zero_means():
    """P4: NZM with all mu = 0 is the ZM method; the mean terms vanish (Sec. V)."""
    g, prm, pred = _tiny_pred(3, 6, seed=6, zero_mean=True)
    z = np.random.default_rng(0).normal(size=(1, g.Nz)) * 1e-3 + 0j
    a = messages_dense.update_messages(pred, W.Params(zero_mean=1), g, z)
    b = messages_dense.update_messages(pred, W.Params(zero_mean=0), g, z)
    assert np.all(a.table.mu3 == 0) and np.all(a.table.mu4 == 0)
    for k in ("log_iota", "log_nu", "log_kappa1", "log_kappa0", "log_omega1"):
        assert np.allclose(getattr(a, k), getattr(b, k), rtol=1e-13)


def test_nu_without_features_is_white_noise_likelihood():
    """P4: with every PF absent (W_s = 0) nu~ = CN(z; 0, eta I) exactly."""
    g, prm, pred = _tiny_pred(2, 5, seed=7)
    pred.w_alpha[:] = 0.0
    z = np.random.default_rng(1).normal(size=(1, g.Nz)) * 1e-3 + 1j * 0.0
    msg = messages_dense.update_messages(pred, prm, g, z)
    eta = pred.eta[0].astype(float)
    expect = -g.Nz * np.log(np.pi * eta) - np.sum(np.abs(z[0]) ** 2) / eta
    assert np.allclose(msg.log_nu[0], expect, rtol=1e-12)


def test_eta_posterior_mean_matches_quadrature():
    """P4: with no PFs the eta belief is xi(eta) CN(z; 0, eta I); starting from a single
    eta_0 the prediction is exactly Gamma(c, eta_0/c), so the particle MMSE must match
    1-D quadrature of the continuous posterior within the Monte Carlo error."""
    g = W.make_geometry(J=1, Nf=2, My=2, Mz=2)
    prm = W.Params(c_eta=100.0)
    P = 200000
    eta0 = 2e-6
    r = np.random.default_rng(11)
    z = (r.normal(size=(1, g.Nz)) + 1j * r.normal(size=(1, g.Nz))) * math.sqrt(2.4e-6 / 2)
    stt = W.StateArrays(n=0, S=1, x=np.zeros((6, P), np.float32), phi=np.zeros((1, 6, P), np.float32),
                        eta=np.full((1, P), eta0, np.float32), w_x=np.full(P, 1.0 / P),
                        w_y=np.zeros((1, P)), w_eta=np.full((1, P), 1.0 / P), p_pr=np.zeros((1, 1)))
    stt.x[0] = 1.0
    prm.Q = 0
    pred = model.predict(stt, prm, 1, seed=3, S_max=1)
    pred.w_alpha[:] = 0.0
    tab = messages_dense.message_table(pred, prm, messages_dense.all_steering(pred, g))
    ln = messages_dense.log_nu(pred, tab, z, 0)
    w = np.exp(ln - ln.max()); w /= w.sum()
    e = pred.eta[0].astype(float)
    mmse = np.sum(w * e)
    grid = np.linspace(1e-9, 8e-6, 400001)
    logpost = st.gamma.logpdf(grid, prm.c_eta, scale=float(np.float32(eta0)) / prm.c_eta) \
        - g.Nz * np.log(np.pi * grid) - np.sum(np.abs(z) ** 2) / grid
    pw = np.exp(logpost - logpost.max())
    quad = np.sum(grid * pw) / np.sum(pw)
    sd = math.sqrt(np.sum(pw * (grid - quad) ** 2) / np.sum(pw))
    ess = 1.0 / np.sum(w ** 2)
    assert abs(mmse - quad) < 5 * sd / math.sqrt(ess)


# ---------------------------------------------------------------- prediction (P5)
@pytest.mark.parametrize("dims", [3, 2])
def test_ncv_prediction_matches_kalman(dims):
    """P5: particle mean/cov after the NCV prediction converge to Phi m, Phi P Phi^T + Q."""
    prm = W.Params(T=0.1, sigma_v=0.7, motion_dims=dims, Q=0)
    P = 200000
    r = np.random.default_rng(12)
    m0 = np.array([1.0, 2.0, 0.5, 0.3, -0.2, 0.1])
    P0 = np.diag([0.01, 0.02, 0.005, 0.04, 0.03, 0.02])
    if dims == 2:
        m0[5] = 0.0; P0[2, 2] = 0.0; P0[5, 5] = 0.0
    x0 = r.multivariate_normal(m0, P0, size=P).T
    stt = W.StateArrays(n=4, S=1, x=x0.astype(np.float32), phi=np.zeros((1, 6, P), np.float32),
                        eta=np.full((1, P), 1e-6, np.float32), w_x=np.full(P, 1.0 / P),
                        w_y=np.full((1, P), 0.5 / P), w_eta=np.full((1, P), 1.0 / P), p_pr=np.full((1, 1), 0.5))
    pred = model.predict(stt, prm, 1, seed=5, S_max=1)
    F, Qa = model.ncv_matrices(prm.T, prm.sigma_v, dims)
    xs = x0.astype(np.float32).astype(float)
    m_ref = F @ xs.mean(1)
    C_ref = F @ np.cov(xs) @ F.T + Qa
    x1 = pred.x.astype(float)
    assert np.allclose(x1.mean(1), m_ref, atol=6 * np.sqrt(np.diag(C_ref) / P) + 1e-7)
    C1 = np.cov(x1)
    tol = 6 * np.sqrt((np.outer(np.diag(C_ref), np.diag(C_ref)) + C_ref ** 2) / P) + 1e-12
    assert np.all(np.abs(C1 - C_ref) <= tol)


def test_prediction_weights_and_zeta():
    """w_beta = w_x, w_xi = w_eta, w_alpha = p_S w_y, zeta(1) = p_S^PR p + p_R^PR (1 - p)."""
    prm = W.Params(Q=1)
    stt = W.state_from_prior(prm, J=2, P=64, S=3, seed=1)
    pred = model.predict(stt, prm, 2, seed=3, S_max=8)
    assert pred.S == 4
    assert np.allclose(pred.w_beta, stt.w_x) and np.allclose(pred.w_xi, stt.w_eta)
    assert np.allclose(pred.w_alpha[:3], 0.8 * stt.w_y)
    assert np.allclose(pred.zeta[:3], 0.9 * stt.p_pr + 0.1 * (1 - stt.p_pr))
    assert np.allclose(pred.w_alpha[3], (1 / 3) / 64) and np.allclose(pred.zeta[3], 0.3)
    lo, hi = np.array(prm.birth_min), np.array(prm.birth_max)
    assert np.all(pred.phi[3, :3] >= lo[:, None] - 1e-6) and np.all(pred.phi[3, :3] <= hi[:, None] + 1e-6)
    assert np.all(np.hypot(pred.phi[3, 4], pred.phi[3, 5]) <= prm.mu_max * (1 + 1e-6))


# ---------------------------------------------------------------- beliefs and invariants (P7)
def _updated(seed=0, P=50, S=4, mode="dense"):
    g = W.make_geometry(J=2, Nf=4, My=2, Mz=2)
    prm = W.Params()
    scn = W.make_scenario(g, prm, N=2, K=3, seed=seed)
    eta = synth.noise_variance(scn)
    z = synth.observe(scn, 1, eta, 5)
    st0 = W.state_near_truth(scn, P=P, S=S, n=0, seed=seed + 1, eta_true=eta, pos_std=0.1,
                             uniform_weights=False)
    pred = model.predict(st0, prm, g.J, seed=9, S_max=8)
    msg = (messages_dense if mode == "dense" else messages_woodbury).update_messages(pred, prm, g, z)
    bel = beliefs.beliefs(pred, msg)
    return g, prm, pred, msg, bel


def test_belief_normalisation_invariants():
    g, prm, pred, msg, bel = _updated()
    assert bel.w_x.sum() == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(bel.w_eta.sum(1), 1.0, atol=1e-12)
    assert np.allclose(bel.w_y.sum(1), bel.p_s, atol=1e-15)
    assert np.all((bel.p_s >= 0) & (bel.p_s <= 1 + 1e-12))
    # Sec. S-IV identity: 1 = sum w~_y / C + (1 - W) prod_j kappa~(., 0) / C
    for s in range(pred.S):
        lhs = np.exp(beliefs.logsumexp(bel.log_wy[s]) - bel.log_Cy[s]) + np.exp(bel.log_null[s] - bel.log_Cy[s])
        assert lhs == pytest.approx(1.0, abs=1e-12)


def _real_cn_logpdf(z, m, C):
    """log CN(z; m, C) as the real 2N-dim normal of [Re z, Im z] (scipy), independent of the oracle."""
    Cr = 0.5 * np.block([[C.real, -C.imag], [C.imag, C.real]])
    return st.multivariate_normal(mean=np.r_[m.real, m.imag], cov=Cr).logpdf(np.r_[z.real, z.imag])


@pytest.mark.parametrize("W_s,J", [(0.5, 1), (0.2, 2), (0.85, 2)])
def test_existence_posterior_is_the_bernoulli_posterior_for_a_point_mass(W_s, J):
    """Sec. S-IV null term of C_y,s: one PF (the LoS), zeta = 1 on every PA, and every
    belief a point mass (MT, PF and noise particles all equal).  Moment matching is then
    exact, so p_s must be the posterior existence probability of a Bernoulli component
    with prior W_s:  W prod_j CN(z_j; mu psi_j, eta I + gamma psi_j psi_j^H) /
    (W prod_j CN(...) + (1 - W) prod_j CN(z_j; 0, eta I)).  Both densities come from the
    enumeration in brute.mixture_moments with r_s fixed and from scipy's real normal."""
    P = 5
    g = W.make_geometry(J=J, Nf=3, My=2, Mz=1)
    prm = W.Params(Q=0)
    r = np.random.default_rng(17 + J)
    x = np.zeros((6, P), np.float32)
    x[:3] = np.array([0.7, 1.9, 0.1], np.float32)[:, None]
    phi = np.zeros((1, 6, P), np.float32)
    phi[0, 3] = 0.3
    phi[0, 4] = 0.25
    phi[0, 5] = -0.125
    eta = np.full((J, P), 0.5, np.float32)
    pred = model.Predicted(n=1, S=1, x=x, phi=phi, eta=eta, w_beta=np.full(P, 1.0 / P),
                           w_alpha=np.full((1, P), W_s / P), w_xi=np.full((J, P), 1.0 / P),
                           zeta=np.ones((1, J)), is_new=np.zeros(1, bool))
    psi = messages_dense.all_steering(pred, g)          # (S, J, P, Nz)
    Nz = psi.shape[-1]
    z = (r.normal(size=(J, Nz)) + 1j * r.normal(size=(J, Nz))) * 0.6
    msg = messages_dense.update_messages(pred, prm, g, z)
    bel = beliefs.beliefs(pred, msg)
    gam = np.array([0.3]); mu = np.array([0.25 - 0.125j])
    l1 = l0 = 0.0
    for j in range(J):
        ps = psi[:, j, 0]
        m1, C1 = brute.mixture_moments(ps, gam, mu, np.array([W_s]), np.ones(1), 0.5, fixed={("r", 0): 1})
        m0, C0 = brute.mixture_moments(ps, gam, mu, np.array([W_s]), np.ones(1), 0.5, fixed={("r", 0): 0})
        l1 += _real_cn_logpdf(z[j], m1, C1)
        l0 += _real_cn_logpdf(z[j], m0, C0)
    a = math.log(W_s) + l1
    b = math.log1p(-W_s) + l0
    p_exact = 1.0 / (1.0 + math.exp(b - a))
    assert 1e-3 < p_exact < 1 - 1e-3                     # the case is not saturated
    assert bel.p_s[0] == pytest.approx(p_exact, abs=1e-10)
    assert np.allclose(bel.w_y[0], p_exact / P, rtol=1e-9)


@pytest.mark.parametrize("dims", [3, 2])
def test_legacy_pf_random_walk_moments(dims):
    """Sec. V-A transitions of a legacy PF: p_sfv <- p_sfv + N(0, sigma_sfv^2 I) and
    mu <- CN(mu, sigma_mu^2), circular with total variance sigma_mu^2 (reading R10).
    The per-particle increments must have zero mean, covariance sigma_sfv^2 I (the z
    component held in planar motion), E|d mu|^2 = sigma_mu^2, E[d mu^2] = 0; the LoS
    slot keeps its (unused) SFV.  Tolerances are 6 Monte Carlo standard errors."""
    P = 200000
    prm = W.Params(Q=0, sigma_sfv=0.05, sigma_mu=0.2, motion_dims=dims)
    r = np.random.default_rng(21)
    phi = np.zeros((2, 6, P), np.float32)
    phi[:, :3] = r.normal([[1.0], [2.0], [0.5]], 0.3, size=(2, 3, P)).astype(np.float32)
    phi[:, 3] = r.uniform(0.5, 1.0, size=(2, P)).astype(np.float32)
    phi[:, 4] = r.normal(0.3, 0.1, size=(2, P)).astype(np.float32)
    phi[:, 5] = r.normal(-0.2, 0.1, size=(2, P)).astype(np.float32)
    stt = W.StateArrays(n=3, S=2, x=np.zeros((6, P), np.float32), phi=phi,
                        eta=np.full((1, P), 1e-6, np.float32), w_x=np.full(P, 1.0 / P),
                        w_y=np.full((2, P), 0.5 / P), w_eta=np.full((1, P), 1.0 / P),
                        p_pr=np.full((2, 1), 0.5))
    pred = model.predict(stt, prm, 1, seed=6, S_max=2)
    d = pred.phi[1].astype(float) - phi[1].astype(float)
    sd = prm.sigma_sfv
    k = 3 if dims == 3 else 2
    assert np.all(np.abs(d[:k].mean(1)) < 6 * sd / math.sqrt(P))
    C = np.cov(d[:k])
    assert np.all(np.abs(C - sd * sd * np.eye(k)) < 6 * sd * sd * math.sqrt(2.0 / P))
    if dims == 2:
        assert np.all(d[2] == 0.0)
    dmu = d[4] + 1j * d[5]
    s2 = prm.sigma_mu ** 2
    assert abs(dmu.mean()) < 6 * prm.sigma_mu / math.sqrt(P)
    assert abs(np.mean(np.abs(dmu) ** 2) - s2) < 6 * s2 / math.sqrt(P)
    assert abs(np.mean(dmu * dmu)) < 6 * s2 / math.sqrt(P)
    assert np.all(pred.phi[0, :3] == phi[0, :3])        # LoS: no SFV random walk


def test_pr_existence_logistic_equals_ratio():
    """Sec. S-VI: sigma(log-odds + log-LR) equals eq. (PR-normalization)."""
    r = np.random.default_rng(3)
    zeta = r.uniform(0.01, 0.99, 50)
    l1 = r.normal(size=50) * 3
    l0 = r.normal(size=50) * 3
    ratio = zeta * np.exp(l1) / (zeta * np.exp(l1) + (1 - zeta) * np.exp(l0))
    assert np.allclose(beliefs.pr_existence(zeta, l1, l0), ratio, rtol=1e-13)
    assert beliefs.pr_existence(np.array(1.0), np.array(-1e4), np.array(0.0)) == 1.0


def test_estimates_are_weighted_means():
    g, prm, pred, msg, bel = _updated()
    est = beliefs.estimate(pred, bel, prm)
    x = pred.x.astype(float)
    assert np.allclose(est.x_hat, (x * bel.w_x).sum(1))
    assert np.allclose(est.p_pr_any, 1 - np.prod(1 - bel.p_pr, axis=1))
    keep = beliefs.survivors(est, prm)
    assert keep[0] == 0
    for s in range(1, pred.S):
        assert (s in keep) == (est.p_s[s] >= prm.T_pru and est.p_pr_any[s] >= prm.T_pru)


# ---------------------------------------------------------------- resampling (P7)
def test_systematic_resampling_counts():
    r = np.random.default_rng(4)
    for P in (1, 7, 1000):
        w = r.gamma(0.3, size=P); w /= w.sum()
        for U in (0.0, 0.37, 0.999):
            idx = resample.systematic_indices(w, U)
            cnt = np.bincount(idx, minlength=P)
            assert cnt.sum() == P
            assert np.all(np.abs(cnt - P * w) < 1.0 + 1e-9)
            assert np.all(np.diff(idx) >= 0)


def test_regularisation_jitter_covariance():
    """Jitter covariance = h_opt^2 x weighted covariance (Musso et al., Gaussian kernel)."""
    P = 100000
    r = np.random.default_rng(5)
    C = np.array([[0.04, 0.01], [0.01, 0.09]])
    X = r.multivariate_normal([0, 0], C, size=P).T
    w = np.full(P, 1.0 / P)
    jit = resample._jitter(X, w, np.ones(2, bool), 3, 1, rng.JITTER_MT, 0, P)
    h = resample.h_opt(P, 2)
    assert np.allclose(np.cov(jit), h * h * resample.weighted_cov(X, w), rtol=0.03, atol=1e-5)


def test_h_opt_minimises_the_gaussian_kernel_amise():
    """h_opt (Musso et al., as cited in Sec. IV-D, the regularisation paragraph) is the
    bandwidth that minimises the asymptotic mean integrated squared error of a Gaussian
    kernel estimate of a Gaussian density in whitened coordinates:
    AMISE(h) = R(K)/(P h^d) + h^4/4 int (Laplacian f)^2.  Both integrals are taken here by
    quadrature on a grid and AMISE is minimised numerically, independent of the formula."""
    from scipy import optimize
    for d in (1, 2, 3):
        g = np.linspace(-7.0, 7.0, 121)
        dx = g[1] - g[0]
        r2 = sum(x * x for x in np.meshgrid(*([g] * d), indexing="ij"))
        f = np.exp(-r2 / 2) / (2 * np.pi) ** (d / 2)
        lap2 = np.sum(((r2 - d) * f) ** 2) * dx ** d      # int (Laplacian f)^2
        RK = np.sum(f ** 2) * dx ** d                       # int K^2, K the standard normal
        for P in (100, 3000, 100000):
            h = optimize.minimize_scalar(lambda t: RK / (P * t ** d) + t ** 4 / 4 * lap2, bounds=(1e-4, 5.0),
                                         method="bounded", options={"xatol": 1e-12}).x
            assert resample.h_opt(P, d) == pytest.approx(h, rel=1e-6), (d, P)


def test_regularisation_covariance_is_the_weighted_moment():
    """The kernel's covariance is the second central moment of the belief, i.e. of the
    weighted particle set (reading R8): two clouds of coincident particles at a and b with
    total weights w and 1 - w have covariance w (1 - w) (a - b)(a - b)^T whatever the
    particle counts, a rank-one matrix, so the zeroing Cholesky leaves one column and the
    jitter moves particles along a - b only, with variance h_opt^2 w (1 - w) |a - b|^2."""
    P, w = 200000, 0.3
    a, b = np.array([1.0, -2.0, 0.5]), np.array([1.4, -1.0, 0.5])
    n_a = P // 4                                   # 1/4 of the particles carry weight w
    X = np.concatenate([np.repeat(a[:, None], n_a, 1), np.repeat(b[:, None], P - n_a, 1)], axis=1)
    wt = np.concatenate([np.full(n_a, w / n_a), np.full(P - n_a, (1 - w) / (P - n_a))])
    D = a - b
    C = resample.weighted_cov(X, wt)
    assert np.allclose(C, w * (1 - w) * np.outer(D, D), rtol=1e-9, atol=1e-14)
    # the unweighted moment of the same set differs: (1/4)(3/4) instead of w (1 - w)
    assert not np.allclose(np.cov(X, bias=True), C, rtol=1e-3)
    jit = resample._jitter(X, wt, np.ones(3, bool), 5, 1, rng.JITTER_PF, 2, P)
    h = resample.h_opt(P, 3)
    along = D / np.linalg.norm(D)
    proj = along @ jit
    assert np.var(proj) == pytest.approx(h * h * w * (1 - w) * (D @ D), rel=0.02)
    # off a - b only what FP64 rounding leaves in the rank-one factor (a second pivot of
    # ~1e-17 keeps a column of ~sqrt(1e-17))
    assert np.max(np.abs(jit - np.outer(along, proj))) < 1e-6 * np.max(np.abs(jit))


def test_zeroing_cholesky():
    C = np.diag([4.0, 0.0, 9.0])
    C[0, 2] = C[2, 0] = 1.0
    L = resample.cholesky_zeroing(C)
    assert np.allclose(L @ L.T, C)
    assert np.all(L[:, 1] == 0)


# ---------------------------------------------------------------- synthetic data
def test_synthetic_noise_and_snr():
    g = W.make_geometry(J=2, Nf=10, My=4, Mz=4)
    prm = W.Params()
    scn = W.make_scenario(g, prm, N=3, K=4, seed=1, snr_db=20.0)
    eta = synth.noise_variance(scn)
    sig = synth.clean_signal(scn, 1)
    assert np.sum(np.abs(sig) ** 2) / (g.Nz * g.J) / eta == pytest.approx(100.0, rel=1e-12)
    res = np.concatenate([synth.observe(scn, n, eta, 2) - synth.clean_signal(scn, n) for n in (1, 2, 3)]).ravel()
    assert np.mean(np.abs(res) ** 2) / eta == pytest.approx(1.0, abs=5 * math.sqrt(1.0 / res.size))


# ---------------------------------------------------------------- time-0 beliefs with S0 PFs
def test_init_state_birth_pfs_follow_the_birth_density():
    """Slots 1 .. S0-1 are draws of f_B (Sec. III-B2) over the whole birth box: each
    coordinate uniform on [2 p_min, 2 p_max] (mean and variance of the uniform law),
    gamma uniform on [0, gamma_max], mu uniform on the disc of radius mu_max
    (E|mu|^2 = mu_max^2 / 2, circular phase); weights p_B / P, PR existence p_B^PR;
    S0 = 1 is the plain time-0 belief."""
    prm = W.Params()
    P, J = 40000, 3
    st0 = model.init_state(prm, J, P, 5)
    st = model.init_state(prm, J, P, 5, S0=4)
    assert st.S == 4 and st0.S == 1
    assert np.array_equal(st.x, st0.x) and np.array_equal(st.eta, st0.eta) and np.array_equal(st.phi[0], st0.phi[0])
    lo, hi = np.asarray(prm.birth_min), np.asarray(prm.birth_max)
    for s in range(1, 4):
        ph = st.phi[s].astype(np.float64)
        for k in range(3):
            width = hi[k] - lo[k]
            assert lo[k] <= ph[k].min() and ph[k].max() <= hi[k]
            assert abs(ph[k].mean() - 0.5 * (lo[k] + hi[k])) < 5 * width / math.sqrt(12 * P)
            assert ph[k].var() == pytest.approx(width ** 2 / 12, rel=0.03)
        assert 0 <= ph[3].min() and ph[3].max() <= prm.gamma_max
        assert abs(ph[3].mean() - 0.5 * prm.gamma_max) < 5 * prm.gamma_max / math.sqrt(12 * P)
        m2 = ph[4] ** 2 + ph[5] ** 2
        assert m2.max() <= prm.mu_max ** 2 * (1 + 1e-6)
        assert m2.mean() == pytest.approx(0.5 * prm.mu_max ** 2, rel=0.03)
        assert abs(np.mean(ph[4] + 1j * ph[5])) < 5 * prm.mu_max / math.sqrt(2 * P)
    pB = model.birth_probability(prm.mu_B, max(prm.Q, 1))
    assert np.allclose(st.w_y, pB / P) and np.allclose(st.p_pr, prm.pB_pr)
    # independent slots: different draws
    assert not np.allclose(st.phi[1], st.phi[2])


def test_batched_scenario_shapes():
    """The batched workload's shapes: S in 1..64, P in 256..16384, Nz in 5..300 with one
    antenna (Nf = Nz) below 16 samples and a 2 x 2 URA (Nf = ceil(Nz / 4)) above."""
    sc = W.batched_scenarios(2000, seed=3)
    S = np.array([d["S"] for d in sc])
    P = np.array([d["P"] for d in sc])
    assert S.min() == 1 and S.max() == 64 and P.min() >= 256 and P.max() <= 16384
    for d in sc:
        g = d["geom"]
        assert g.J == 4
        if g.My == 1:
            assert g.Mz == 1 and 5 <= g.Nf < 16 and g.Nz == g.Nf
        else:
            assert g.My == g.Mz == 2 and 16 <= g.Nz <= 300 + 3 and g.Nf == -(-g.Nz // 4)
    assert len({d["seed"] for d in sc}) == len(sc)


# ---------------------------------------------------------------- birth proposal (Sec. IV-D)
def _proposal_case(seed=3, K=3, P=4000):
    from oracle import birth_proposal as bpro
    g = W.make_geometry(J=3, Nf=8, My=3, Mz=2)
    prm = W.Params(Q=2, birth_proposal=1, N_g=512)
    scn = W.make_scenario(g, prm, N=3, K=K, seed=seed, snr_db=30.0)
    eta = synth.noise_variance(scn)
    z = synth.observe(scn, 1, eta, seed + 9)
    st = W.state_near_truth(scn, P=P, S=K + 1, n=0, seed=seed + 1, eta_true=eta, pos_std=0.005, sfv_std=0.005)
    pred = model.predict(st, prm, g.J, seed=seed, S_max=K + 1 + prm.Q)
    return bpro, g, prm, scn, z, st, pred


def test_birth_proposal_residual_is_the_orthogonal_projection():
    """z~ = (I - Psi Psi^+) z: orthogonal to every LoS / legacy steering column, and
    projecting it again changes nothing."""
    bpro, g, prm, scn, z, st, pred = _proposal_case()
    x_hat = bpro.mt_mean(pred)
    pos = bpro.legacy_means(pred, st.S)
    zr = bpro.residual(g, z, x_hat, pos)
    for j in range(g.J):
        Psi = np.stack([geometry.steering(g, j, x_hat[None, :3], pos[s][None, :], los=(s == 0))[0]
                        for s in range(st.S)], axis=1)
        assert np.max(np.abs(Psi.conj().T @ zr[j])) < 1e-10 * np.linalg.norm(Psi) * np.linalg.norm(z[j])
    zr2 = bpro.residual(g, zr, x_hat, pos)
    assert np.allclose(zr2, zr, rtol=0, atol=1e-12 * np.max(np.abs(z)))
    assert np.all(np.linalg.norm(zr, axis=1) < np.linalg.norm(z, axis=1))


def test_bartlett_spectrum_peaks_at_the_unexplained_surface():
    """One surface that no legacy PF explains: with the LoS projected out, the coherent
    Bartlett spectrum over its partition peaks within a few cm of its SFV."""
    from oracle import birth_proposal as bpro
    g = W.make_geometry(J=4, Nf=10, My=4, Mz=4)
    prm = W.Params(Q=1)
    x = np.array([1.0, 2.0, 0.2])
    sfv = np.array([[9.0, 3.0, 0.5]])
    z = np.stack([geometry.steering(g, j, x[None], x[None], los=True)[0] * 1.0 +
                  geometry.steering(g, j, x[None], sfv, los=False)[0] * 0.5 * np.exp(0.7j) for j in range(g.J)])
    zr = bpro.residual(g, z, np.r_[x, 0, 0, 0], np.zeros((1, 3)))
    r = np.random.default_rng(1)
    lo, hi = np.asarray(prm.birth_min), np.asarray(prm.birth_max)
    cand = np.concatenate([lo + (hi - lo) * r.random((20000, 3)), sfv + 0.02 * r.standard_normal((200, 3))])
    c = bpro.bartlett(g, zr, np.r_[x, 0, 0, 0], cand)
    i_star, mu, C = bpro.moments(cand, c)
    assert np.linalg.norm(mu - sfv[0]) < 0.05
    # the residual carries only the surface: its spectrum at the true SFV is |0.5 psi^H psi / Nz|^2 summed coherently
    ref = abs(sum(0.5 * np.exp(0.7j) * np.vdot(geometry.steering(g, j, x[None], sfv, los=False)[0],
                                                 geometry.steering(g, j, x[None], sfv, los=False)[0]) / g.Nz
                  for j in range(g.J))) ** 2
    c_true = bpro.bartlett(g, zr, np.r_[x, 0, 0, 0], sfv)[0]
    assert c_true == pytest.approx(ref, rel=1e-3)   # the LoS projection removes ~nothing of the surface here


def test_birth_proposal_weights_are_importance_weights():
    """w_alpha sums to p_B, is zero outside the PF's partition, and reweights the
    proposal draws to the uniform birth density: the weighted mean of any function of
    the position matches its mean over the partition (checked on the position itself
    and its square, within the Monte Carlo error of the weights)."""
    bpro, g, prm, scn, z, st, pred = _proposal_case(P=20000)
    pred2, props = bpro.apply(pred, prm, g, z, st.S, prm.N_g, seed=3)
    pB = model.birth_probability(prm.mu_B, prm.Q)
    for pr in props:
        s = pr.slot
        w = pred2.w_alpha[s]
        assert w.sum() == pytest.approx(pB, rel=1e-12)
        lo, hi = bpro.partition_bounds(prm, prm.Q, pr.q)
        pos = pred2.phi[s, :3].astype(np.float64)
        outside = np.any((pos < lo[:, None] - 1e-5) | (pos > hi[:, None] + 1e-5), axis=0)
        assert np.all(w[outside] == 0)
        # proposal draws: mean mu, covariance L L^T
        assert np.allclose(pr.L @ pr.L.T, pr.C, atol=1e-12)
        wn = w / w.sum()
        ess = 1.0 / np.sum(wn ** 2)
        for k in range(3):
            if pr.L[k, k] == 0:
                continue
            se = (hi[k] - lo[k]) / math.sqrt(12 * max(ess, 1.0))
            m = np.sum(wn * pos[k])
            assert abs(m - 0.5 * (lo[k] + hi[k])) < 6 * se + 0.02 * (hi[k] - lo[k])


# ---------------------------------------------------------------- PCRLB (Sec. VI, S-VII)
def _pcrlb_case(J=2):
    g = W.make_geometry(J=J, Nf=4, My=2, Mz=2)
    x = np.array([1.0, 2.0, 0.3, 0.1, 0.2, 0.0])
    sfvs = np.array([[9.0, 3.0, 0.5], [-5.0, 6.0, 1.0]])
    r = np.random.default_rng(4)
    mod = 0.3 + r.random((J, 3))
    ph = r.uniform(-np.pi, np.pi, 3)          # coherent: one nuisance phase per component
    phj = r.uniform(-np.pi, np.pi, (J, 3))    # noncoherent: one per component and PA
    return g, x, sfvs, mod, ph, phj


def _mean_model(g, p, sfvs, mod, phases, coherent):
    """Observation mean of every PA from global parameters: components k with modulus
    mod[j, k], phase (nuisance + carrier -2 pi |r'| / lambda) and the unit-modulus response
    at the local delay and angles (the PCRLB model of Sec. S-VII)."""
    from oracle import pcrlb
    lam = g.c / g.fc
    out = []
    for j in range(g.J):
        mu = np.zeros(g.Nz, complex)
        for k in range(len(sfvs) + 1):
            rp, _ = pcrlb.local_vector(g, j, p, None if k == 0 else sfvs[k - 1], k == 0)
            d, th, az = pcrlb.spherical(rp)
            a = pcrlb.response(g, d / g.c, th, az)[0]
            phi = (phases[k] if coherent else phases[j, k]) - 2 * np.pi * d / lam
            mu += mod[j, k] * np.exp(1j * phi) * a
        out.append(mu)
    return out


def _rho_t(g, p, sfvs, mod, phases, coherent):
    from oracle import pcrlb
    lam = g.c / g.fc
    rho = np.zeros((g.J, len(sfvs) + 1), complex)
    for j in range(g.J):
        for k in range(len(sfvs) + 1):
            rp, _ = pcrlb.local_vector(g, j, p, None if k == 0 else sfvs[k - 1], k == 0)
            d = np.linalg.norm(rp)
            rho[j, k] = mod[j, k] * np.exp(1j * ((phases[k] if coherent else phases[j, k]) - 2 * np.pi * d / lam))
    return rho


@pytest.mark.parametrize("coherent", [False, True])
def test_pcrlb_snapshot_fim_equals_finite_difference_fisher(coherent):
    """J_C assembled from Table S-I and the Jacobians of Sec. S-VII-B equals the Fisher
    information of the complex Gaussian observation model computed from central finite
    differences of its mean w.r.t. every global parameter: sum_j (2/eta) Re(G_j^H G_j)
    plus J Nz / eta^2 for eta (Slepian-Bangs).  A wrong derivative, sign, index or
    Jacobian block anywhere in the assembly fails it."""
    from oracle import pcrlb
    g, x, sfvs, mod, ph, phj = _pcrlb_case()
    phases = ph if coherent else phj
    eta = 2e-3
    K = len(sfvs)
    dd = pcrlb.dims(K, g.J, coherent)
    Jfim = pcrlb.snapshot_fim(g, x, sfvs, _rho_t(g, x[:3], sfvs, mod, phases, coherent), eta, coherent)

    def unpack(v):
        p = v[0:3]
        s = v[6:6 + 3 * K].reshape(K, 3)
        phs = v[dd["o_ph"]:dd["o_a"]]
        phs = phs if coherent else phs.reshape(g.J, K + 1)
        m = v[dd["o_a"]:dd["o_eta"]].reshape(g.J, K + 1)
        return p, s, m, phs

    v0 = np.zeros(dd["dim"])
    v0[0:6] = x
    v0[6:6 + 3 * K] = sfvs.ravel()
    v0[dd["o_ph"]:dd["o_a"]] = phases.ravel()
    v0[dd["o_a"]:dd["o_eta"]] = mod.ravel()
    v0[dd["o_eta"]] = eta
    G = [np.zeros((g.Nz, dd["dim"]), complex) for _ in range(g.J)]
    for i in range(dd["dim"] - 1):
        h = 1e-6 * max(1.0, abs(v0[i]))
        vp, vm = v0.copy(), v0.copy()
        vp[i] += h
        vm[i] -= h
        mp = _mean_model(g, *unpack(vp), coherent)
        mm = _mean_model(g, *unpack(vm), coherent)
        for j in range(g.J):
            G[j][:, i] = (mp[j] - mm[j]) / (2 * h)
    Jnum = sum(2.0 / eta * np.real(Gj.conj().T @ Gj) for Gj in G)
    Jnum[dd["o_eta"], dd["o_eta"]] = g.J * g.Nz / eta ** 2
    scale = np.sqrt(np.outer(np.diag(Jnum), np.diag(Jnum))) + 1e-300
    assert np.max(np.abs(Jfim - Jnum) / scale) < 1e-5


def test_pcrlb_recursion_closed_forms():
    """With no measurement information the posterior covariance follows the prediction
    P_n = F P_{n-1} F^T + Q; with a static state (F = I, Q = 0) and a constant snapshot FIM
    the information adds up: J_n = n J_B + J_{1|0}."""
    from oracle import pcrlb
    r = np.random.default_rng(2)
    d = 5
    A = r.standard_normal((d, d))
    P0 = A @ A.T + d * np.eye(d)
    F = np.eye(d) + 0.1 * r.standard_normal((d, d))
    B = r.standard_normal((d, d))
    Q = B @ B.T * 0.01 + 1e-3 * np.eye(d)
    Js = pcrlb.recursion([np.zeros((d, d))] * 4, F, Q, np.linalg.inv(P0))
    P = P0
    for n in range(4):
        assert np.allclose(np.linalg.inv(Js[n]), P, rtol=1e-9, atol=1e-12)
        P = F @ P @ F.T + Q
    JB = A @ A.T
    Js = pcrlb.recursion([JB] * 5, np.eye(d), np.zeros((d, d)), np.linalg.inv(P0))
    for n in range(5):
        assert np.allclose(Js[n], (n + 1) * JB + np.linalg.inv(P0), rtol=1e-9)


def test_pcrlb_coherent_bound_is_tighter():
    """The coherent model has K~ nuisance phases instead of K~ J: its position bound is never
    larger; with a single PA the two models are the same."""
    from oracle import pcrlb
    for J in (1, 3):
        g, x, sfvs, mod, ph, phj = _pcrlb_case(J)
        eta = 2e-3
        prm = W.Params(motion_dims=3)
        out = {}
        for coherent in (False, True):
            phases = ph if coherent else np.broadcast_to(ph, (J, 3)).copy()
            Jc = pcrlb.snapshot_fim(g, x, sfvs, _rho_t(g, x[:3], sfvs, mod, phases, coherent), eta, coherent)
            dd = pcrlb.dims(len(sfvs), J, coherent)
            F, Q = pcrlb.transition(prm, len(sfvs), J, coherent, 10.0, 10.0, 10.0)
            J10 = np.linalg.inv(Q + 1e-2 * np.eye(dd["dim"]))
            post = pcrlb.recursion([Jc] * 3, F, Q, J10)
            out[coherent] = pcrlb.bounds(post[-1], len(sfvs))
        assert out[True][0] <= out[False][0] * (1 + 1e-9)
        if J == 1:
            assert out[True][0] == pytest.approx(out[False][0], rel=1e-9)
