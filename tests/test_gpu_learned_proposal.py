"""The learned MT proposal on the GPU against the FP64 oracle, through the C ABI: the
summary of z at the predicted mean, the network inputs and outputs, the importance
ratios and the update that follows; the exact case of a null network; and the training
data simulated from the model."""
import numpy as np
import pytest

from oracle import beliefs, learned_proposal as LP, messages_woodbury, mlp, model, synth
from paper_2604_19723_gb300 import workload as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import bp  # noqa: E402


def setup(P, seed, motion_dims=3, K=4):
    g = W.make_geometry(J=4, Nf=10, My=4, Mz=4)
    prm = W.Params(motion_dims=motion_dims, Q=0)
    scn = W.make_scenario(g, prm, N=3, K=K, seed=seed, snr_db=20.0)
    eta = synth.noise_variance(scn)
    # the observation as the C ABI takes it (complex64), for both sides
    z = synth.observe(scn, 1, eta, seed + 100).astype(np.complex64).astype(np.complex128)
    st = W.state_near_truth(scn, P=P, S=K + 1, n=0, seed=seed + 1, eta_true=eta, pos_std=0.005, sfv_std=0.005)
    pred = model.predict(st, prm, g.J, seed=seed, S_max=8)
    return g, prm, z, pred


def gpu_update(g, prm, z, pred, P, seed, theta):
    f = bp.Filter(g, prm, P=P, S_max=8, seed=seed)
    net = bp.Mlp(theta)
    f.set_mt_proposal(net)
    f.set_predicted(pred.n, pred.S, pred.x, pred.phi, pred.eta, pred.w_beta, pred.w_alpha, pred.w_xi, pred.zeta)
    f.update(torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda())
    torch.cuda.synchronize()
    return f, net


def check_summary(d, r):
    assert np.allclose(d["xbar"], r.xbar, rtol=0, atol=1e-12)
    scale = np.max(np.abs(r.cor), axis=0)
    assert np.all(np.abs(d["cor"] - r.cor) <= 1e-9 * scale[None, :]), np.max(np.abs(d["cor"] - r.cor))
    assert np.max(np.abs(d["X"] - r.X)) < 1e-5 * max(1.0, np.max(np.abs(r.X)))


@pytest.mark.parametrize("motion_dims", [3, 2])
def test_null_network_is_the_transition_exactly(motion_dims):
    """Zero weights: the network outputs (0, 0), the proposal is the transition itself
    (other draws), every importance ratio is exactly 1, and the update that follows
    equals the oracle's update of its own redrawn prediction."""
    P, seed = 600, 61
    g, prm, z, pred = setup(P, seed, motion_dims)
    z32 = z.astype(np.complex64).astype(np.complex128)
    theta = np.zeros(mlp.NPARAM, np.float32)
    f, net = gpu_update(g, prm, z, pred, P, seed, theta)
    d = f.diag_lproposal()
    new, r = LP.apply(pred, prm, g, z32, theta, seed)
    check_summary(d, r)
    assert np.all(d["Y"] == 0.0) and np.all(d["logr"] == 0.0)
    bel = beliefs.beliefs(new, messages_woodbury.update_messages(new, prm, g, z32))
    gw = f.diag_weights(pred.S)
    # the redrawn particles agree to FP32 rounding (FP32 vs FP64 Box-Muller of the draws)
    assert float(np.max(np.abs(gw["w_x"] - bel.w_x)) / np.max(bel.w_x)) < 1e-3
    assert np.max(np.abs(gw["p_s"] - bel.p_s)) < 1e-4
    f.close(); net.close()


def test_random_network_matches_oracle():
    P, seed = 700, 62
    g, prm, z, pred = setup(P, seed)
    z32 = z.astype(np.complex64).astype(np.complex128)
    theta = W.mlp_init(63, out_scale=0.3)
    f, net = gpu_update(g, prm, z, pred, P, seed, theta)
    d = f.diag_lproposal()
    new, r = LP.apply(pred, prm, g, z32, theta, seed)
    check_summary(d, r)
    # BF16 inference: accumulation order can flip a stored activation by one BF16 unit
    # (2^-8 relative), ~1e-3 of the output scale through the last layer
    ysc = max(1.0, np.max(np.abs(r.Y[:, :6])))
    dy = np.abs(d["Y"][:, :6] - r.Y[:, :6])
    assert dy.max() < 2e-2 * ysc and dy.mean() < 1e-3 * ysc, (dy.max(), dy.mean())
    # log r moves by |u| |d mu| + |g| s |d log s| + |d log s|: a few times the output error
    dl = np.abs(d["logr"] - r.logr)
    assert dl.max() < 0.2 and np.median(dl) < 1e-2, (dl.max(), np.median(dl))
    # the update that follows: the MT posterior mean within 1e-4 m of the oracle's
    bel = beliefs.beliefs(new, messages_woodbury.update_messages(new, prm, g, z32))
    est = beliefs.estimate(new, bel, prm)
    assert np.max(np.abs(f.estimate()["x_hat"][:3] - est.x_hat[:3])) < 1e-4
    f.close(); net.close()


def test_training_samples_follow_the_model():
    """Targets of the training samples are the least-squares NCV noise that carries each
    particle to its true successor: for a particle at the true previous state they are
    the true noise, N(0, 1); the summary features lie in their ranges."""
    g = W.make_geometry(J=4, Nf=10, My=4, Mz=4)
    prm = W.Params()
    sfv = W.room_sfvs(prm.p_min, prm.p_max)
    X, T = bp.lp_dataset(g, prm, sfv, np.array([1.0, 0.5, 0.5, 0.5, 0.5]), 4e-8, 20000, seed=3,
                         err_pos=0.0, err_vel=0.0, spread_pos=0.0, spread_vel=0.0)
    X, T = X.cpu().numpy(), T.cpu().numpy()
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(T))
    assert np.allclose(X[:, :6], 0.0, atol=1e-4)                 # the particle is the mean
    assert abs(T.mean()) < 0.03 and abs(T.std() - 1.0) < 0.03     # the true N(0, I) noise
    # ROI coordinates of the predicted mean, one step (T v_max) past the ROI at most
    hw = np.maximum(0.5 * (np.asarray(prm.p_max) - np.asarray(prm.p_min)), 0.5)
    assert np.all(np.abs(X[:, 6:9]) <= 1.0 + prm.T * np.asarray(prm.v_max) / hw + 1e-6)
    assert np.all((X[:, 15] >= 0) & (X[:, 15] <= 1.0 + 1e-6))    # |rho_0|
    assert np.all(np.abs(X[:, 9:15]) <= 1.0 + 1e-6)              # relative correlations
    # the LoS dominates at 20 dB: the correlation at the predicted (= true) mean is high
    assert np.median(X[:, 15]) > 0.5


def test_trained_network_gains_over_the_transition():
    """Trained on the model's own simulations (GPU data, GPU training), the learned
    proposal tracks with a fraction of the transition proposal's error at 2000 particles
    (same observations, same starts; measured 5 mm against 40 mm RMSE)."""
    from paper_2604_19723_gb300 import learned
    res = learned.compare("paper_exp1_proposal", runs=3, steps=40, P=2000, seed=500,
                          train=learned.train_proposal("paper_exp1_proposal", n_samples=1 << 16, steps=1500))
    assert res["loss"][-1][1] < res["loss"][0][1] - 0.5
    lr, tr = res["learned"], res["transition"]
    assert lr["failed_steps"] == 0
    assert lr["rmse"] < 0.5 * tr["rmse"], (lr, tr)
    assert lr["mean_ess"] > tr["mean_ess"], (lr, tr)


def test_training_samples_coherent_and_noncoherent_phases():
    """At the true state the LoS correlations of coherent data share the amplitude's
    phase, so their ratios to PA 0 are near-real and positive; with phases drawn per PA
    the ratios spread over the circle."""
    g = W.make_geometry(J=4, Nf=10, My=4, Mz=4)
    prm = W.Params()
    sfv = W.room_sfvs(prm.p_min, prm.p_max)
    kw = dict(err_pos=0.0, err_vel=0.0, spread_pos=0.0, spread_vel=0.0)
    Xc, _ = bp.lp_dataset(g, prm, sfv, np.array([1.0, 0.5, 0.5, 0.5, 0.5]), 4e-8, 5000, seed=5, coherent=True, **kw)
    Xn, _ = bp.lp_dataset(g, prm, sfv, np.array([1.0, 0.5, 0.5, 0.5, 0.5]), 4e-8, 5000, seed=5, coherent=False, **kw)
    Xc, Xn = Xc.cpu().numpy(), Xn.cpu().numpy()
    re_c, re_n = Xc[:, [9, 11, 13]], Xn[:, [9, 11, 13]]
    assert np.median(re_c) > 0.3
    assert abs(np.mean(re_n)) < 0.05 and abs(np.mean(Xn[:, [10, 12, 14]])) < 0.05


def test_attach_refused_on_batch_handles_and_detach_restores_the_transition():
    """Handles of a batch share workspaces and take no network (BP_ERR_STATE); on a
    single filter, detaching (None) brings back the transition proposal exactly."""
    P, seed = 300, 64
    g, prm, z, pred = setup(P, seed)
    net = bp.Mlp(W.mlp_init(65, out_scale=0.3))
    b = bp.Batch([(g, prm, P, 8, 5, seed)], n_streams=1)
    with pytest.raises(bp.BPError):
        b.member(0).set_mt_proposal(net)
    b.close()
    zt = torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda()
    out = []
    for attach in (False, True):
        f = bp.Filter(g, prm, P=P, S_max=8, seed=seed)
        if attach:
            f.set_mt_proposal(net)
            f.set_mt_proposal(None)
        f.set_predicted(pred.n, pred.S, pred.x, pred.phi, pred.eta, pred.w_beta, pred.w_alpha, pred.w_xi, pred.zeta)
        f.update(zt)
        out.append(f.diag_weights(pred.S)["w_x"])
        f.close()
    assert np.allclose(out[0], out[1], rtol=1e-9, atol=0)
    net.close()
