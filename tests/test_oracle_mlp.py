"""Pins of the proposal-network oracle (oracle/mlp.py) against what the mathematics
fixes: central finite differences of the loss, the composed linear map when every ReLU
passes, the Gaussian log-density of a library routine, Adam's first step, and the BF16
rounding rule."""
import numpy as np
import pytest

from oracle import mlp
from paper_2604_19723_gb300 import workload as W


def _case(B=37, seed=3):
    rng = np.random.default_rng(seed)
    theta = W.mlp_init(seed, out_scale=0.5).astype(np.float64)
    theta[mlp.NPARAM - 16:] = rng.normal(0, 0.1, 16)           # non-zero output biases
    X = rng.normal(size=(B, mlp.IN))
    T = rng.normal(size=(B, mlp.TD))
    return theta, X, T


def test_backward_equals_central_differences():
    theta, X, T = _case()
    g = mlp.backward(theta, X, T)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 60, replace=False), np.arange(mlp.NPARAM - 16, mlp.NPARAM)])
    h = 1e-6
    for j in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (mlp.mean_loss(tp, X, T) - mlp.mean_loss(tm, X, T)) / (2 * h)
        assert abs(fd - g[j]) < 1e-6 * max(1.0, abs(fd)), (j, fd, g[j])


def test_forward_is_the_composed_affine_map_when_every_relu_passes():
    rng = np.random.default_rng(1)
    p = {"W1": rng.uniform(0, 1, (64, 16)), "b1": rng.uniform(0, 1, 64), "W2": rng.uniform(0, 1, (64, 64)),
         "b2": rng.uniform(0, 1, 64), "W3": rng.normal(size=(16, 64)), "b3": rng.normal(size=16)}
    theta = mlp.pack(p)
    X = rng.uniform(0, 1, (5, 16))
    y = mlp.forward(theta, X)["y"]
    A = p["W3"] @ p["W2"] @ p["W1"]
    c = p["W3"] @ (p["W2"] @ p["b1"] + p["b2"]) + p["b3"]
    assert np.allclose(y, X @ A.T + c, rtol=1e-12, atol=1e-9)


def test_loss_is_the_gaussian_negative_log_likelihood():
    from scipy.stats import norm
    theta, X, T = _case(B=9)
    y = mlp.forward(theta, X)["y"]
    ref = -np.sum(norm.logpdf(T, loc=y[:, :3], scale=np.exp(y[:, 3:6])), axis=1) - 1.5 * np.log(2 * np.pi)
    assert np.allclose(mlp.loss_terms(y, T), ref, rtol=1e-12, atol=1e-12)


def test_adam_first_step_moves_by_the_learning_rate_against_the_sign():
    g = np.array([3.0, -0.5, 1e-3, -2e-2])
    th, m, v = mlp.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), t=1, lr=0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_keeps_eight_significant_bits_nearest_even():
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0                      # halfway: to even
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6         # halfway: to even (up)
    assert mlp.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7             # representable
    x = np.random.default_rng(2).normal(size=1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= 2 ** -8 * np.abs(x) * (1 + 1e-9))   # half an ulp of 8 bits


# ---------------------------------------------------------------- learned MT proposal
def _pred_case(P=4000, seed=21, motion_dims=3):
    from oracle import model, synth
    g = W.make_geometry(J=4, Nf=6, My=2, Mz=2)
    prm = W.Params(motion_dims=motion_dims, Q=0)
    scn = W.make_scenario(g, prm, N=3, K=3, seed=seed)
    eta = synth.noise_variance(scn)
    z = synth.observe(scn, 1, eta, seed + 1)
    st = W.state_near_truth(scn, P=P, S=2, n=0, seed=seed + 2, eta_true=eta)
    pred = model.predict(st, prm, g.J, seed=seed, S_max=4)
    return g, prm, z, pred


def _const_net(mu, ls):
    """A network whose output is the constant (mu, log s) whatever the input."""
    theta = np.zeros(mlp.NPARAM)
    p = mlp.unpack(theta)
    p["b3"][:3] = mu
    p["b3"][3:6] = ls
    return mlp.pack(p)


@pytest.mark.parametrize("motion_dims", [3, 2])
def test_learned_proposal_with_a_null_network_is_the_transition(motion_dims):
    from oracle import learned_proposal as LP
    g, prm, z, pred = _pred_case(P=500, motion_dims=motion_dims)
    new, r = LP.apply(pred, prm, g, z, np.zeros(mlp.NPARAM), seed=21)
    assert np.all(r.logr == 0.0)
    assert np.allclose(new.w_beta, pred.w_beta / pred.w_beta.sum(), rtol=1e-15)
    fx, _ = LP.prev_means(pred, prm, 21)
    from oracle import rng
    gg = np.stack(rng.normals(21, np.arange(500, dtype=np.uint64), pred.n, rng.LEARNED_PROP, 0, 3), axis=0)
    dims = motion_dims
    ref = fx.copy()
    ref[:dims] += 0.5 * prm.T ** 2 * prm.sigma_v * gg[:dims]
    ref[3:3 + dims] += prm.T * prm.sigma_v * gg[:dims]
    assert np.allclose(new.x, ref.astype(np.float32), rtol=0, atol=1e-6)


def test_learned_proposal_weights_restore_the_transition():
    """A shifted, narrowed Gaussian proposal: E_q[r] = 1, and the self-normalised weights
    give the transition's moments of u (mean 0, variance 1) again."""
    from oracle import learned_proposal as LP
    g, prm, z, pred = _pred_case(P=200000)
    theta = _const_net(np.array([0.7, -0.4, 0.2]), np.log(np.array([0.8, 0.9, 1.1])))
    new, r = LP.apply(pred, prm, g, z, theta, seed=21)
    assert abs(np.mean(np.exp(r.logr)) - 1.0) < 0.02
    fx, _ = LP.prev_means(pred, prm, 21)
    u = (new.x[:3].astype(np.float64) - fx[:3]) / (0.5 * prm.T ** 2 * prm.sigma_v)
    w = new.w_beta / new.w_beta.sum()
    assert np.all(np.abs(u @ w) < 0.02)
    assert np.all(np.abs((u * u) @ w - 1.0) < 0.03)


def test_learned_proposal_summary_of_a_pure_los_observation():
    """z_j = e^{i phi} psi_j(xbar): every PA's correlation has the common phase, so the
    relative correlations are 1 and |rho_0| = 1."""
    from oracle import geometry, learned_proposal as LP
    g = W.make_geometry(J=4, Nf=6, My=2, Mz=2)
    prm = W.Params()
    xbar = np.array([1.0, 2.0, 0.3, 0, 0, 0])
    z = np.stack([np.exp(0.7j) * geometry.steering(g, j, xbar[None, :3], xbar[None, :3], los=True)[0]
                  for j in range(g.J)])
    f = LP.summary(prm, xbar, LP.correlations(g, z, xbar))
    assert np.allclose(f[3:9], [1, 0, 1, 0, 1, 0], atol=1e-12)
    assert f[9] == pytest.approx(1.0, abs=1e-12)
    lo, hi = np.asarray(prm.p_min), np.asarray(prm.p_max)
    assert np.allclose(f[:3], (xbar[:3] - 0.5 * (lo + hi)) / (0.5 * (hi - lo)))
