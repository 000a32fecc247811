"""Failure detection without a GPU fault: a bounded device wait on an mbarrier phase that
nothing completes gives up, the kernel ends normally and reports BP_ERR_TIMEOUT, and the
context stays usable (a filter step afterwards matches the oracle).  Host-side failures
(invalid arguments, numerical underflow) come back as status codes."""
import numpy as np
import pytest

from oracle import beliefs, messages_woodbury, model, synth
from paper_2604_19723_gb300 import workload as W

pytestmark = [pytest.mark.gpu]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import bp  # noqa: E402


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    assert bp.selftest_wait(4096) == 5          # BP_ERR_TIMEOUT
    assert bp.selftest_wait(0) == 1             # BP_ERR_INVALID_ARG: no launch
    # the context is intact: one update matches the oracle
    g = W.make_geometry(J=2, Nf=4, My=2, Mz=2)
    prm = W.Params()
    scn = W.make_scenario(g, prm, N=2, K=3, seed=71)
    eta = synth.noise_variance(scn)
    z = synth.observe(scn, 1, eta, 72)
    st = W.state_near_truth(scn, P=256, S=3, n=0, seed=73, eta_true=eta)
    pred = model.predict(st, prm, g.J, seed=74, S_max=8)
    f = bp.Filter(g, prm, P=256, S_max=8, seed=74)
    f.set_predicted(pred.n, pred.S, pred.x, pred.phi, pred.eta, pred.w_beta, pred.w_alpha, pred.w_xi, pred.zeta)
    f.update(torch.from_numpy(z.astype(np.complex64)).cuda())
    bel = beliefs.beliefs(pred, messages_woodbury.update_messages(pred, prm, g, z))
    gw = f.diag_weights(pred.S)
    assert np.max(np.abs(gw["p_s"] - bel.p_s)) < 1e-5
    f.close()


def test_invalid_arguments_are_status_codes():
    g = W.make_geometry(J=2, Nf=4, My=2, Mz=2)
    with pytest.raises(bp.BPError) as e:
        bp.Filter(g, W.Params(), P=0, S_max=8, seed=1)
    assert e.value.status == 1
    with pytest.raises(bp.BPError) as e:
        bp.Filter(g, W.Params(motion_dims=5), P=16, S_max=8, seed=1)
    assert e.value.status == 1


def test_checkpoint_and_resume_continue_the_same_run(tmp_path):
    """A filter restored from a checkpoint after step 2 gives the estimates of the
    uninterrupted run at steps 3 and 4 (same Philox streams, keyed by seed and step)."""
    g = W.make_geometry(J=2, Nf=4, My=2, Mz=2)
    prm = W.Params(Q=1)
    scn = W.make_scenario(g, prm, N=5, K=3, seed=81)
    eta = synth.noise_variance(scn)
    zs = [torch.from_numpy(synth.observe(scn, n, eta, 82 + n).astype(np.complex64)).cuda() for n in range(1, 5)]
    st = W.state_near_truth(scn, P=512, S=3, n=0, seed=83, eta_true=eta)
    f = bp.Filter(g, prm, P=512, S_max=8, seed=84)
    f.set_state(st)
    for n in range(2):
        f.step(zs[n])
    path = str(tmp_path / "ckpt.npz")
    f.save(path)
    ref = []
    for n in range(2, 4):
        f.step(zs[n])
        ref.append(f.estimate())
    f.close()
    g2 = W.make_geometry(J=3, Nf=4, My=2, Mz=2)
    with pytest.raises(ValueError, match="another geometry"):
        bp.Filter.load(path, g2, prm)
    r = bp.Filter.load(path, g, prm)
    bad = r.get_state()
    bad.eta = bad.eta[:1]
    with pytest.raises(ValueError, match="eta has shape"):
        r.set_state(bad)
    for n in range(2, 4):
        r.step(zs[n])
        e = r.estimate()
        assert e["n"] == ref[n - 2]["n"] and e["S"] == ref[n - 2]["S"]
        assert np.allclose(e["x_hat"], ref[n - 2]["x_hat"], rtol=0, atol=1e-9)
        assert np.allclose(e["p_s"], ref[n - 2]["p_s"], rtol=0, atol=1e-9)
    r.close()


def test_non_finite_observation_is_reported():
    g = W.make_geometry(J=2, Nf=4, My=2, Mz=2)
    prm = W.Params()
    scn = W.make_scenario(g, prm, N=2, K=3, seed=91)
    eta = synth.noise_variance(scn)
    z = synth.observe(scn, 1, eta, 92).astype(np.complex64)
    z[1, 3] = np.nan
    st = W.state_near_truth(scn, P=256, S=3, n=0, seed=93, eta_true=eta)
    f = bp.Filter(g, prm, P=256, S_max=8, seed=94)
    f.set_state(st)
    f.step(torch.from_numpy(z).cuda())
    with pytest.raises(bp.BPError) as e:
        f.estimate()
    assert e.value.status == 4 and "NaN or Inf" in str(e.value)
    f.close()
