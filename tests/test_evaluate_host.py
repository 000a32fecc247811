"""Host logic of the Monte Carlo evaluation (Sec. VII): Hungarian association of SFV
estimates, RMSE over runs with unassociated entries, and the bound's F, Q, amplitudes and
prior information against the oracle's definitions.  No GPU needed."""
import numpy as np
import pytest

from oracle import pcrlb
from paper_2604_19723_gb300 import evaluate as E
from paper_2604_19723_gb300 import workload as W

pytest.importorskip("scipy")


def test_association_recovers_a_permutation():
    rng = np.random.default_rng(0)
    truth = rng.normal(size=(4, 3)) * 5
    perm = [2, 0, 3, 1]
    est = truth[perm] + 0.01 * rng.normal(size=(4, 3))
    err = E.associate(est, truth)
    ref = np.linalg.norm(est[np.argsort(perm)] - truth, axis=1)
    assert np.allclose(err, ref)


def test_association_with_missed_detections_and_false_alarms():
    truth = np.array([[0.0, 0, 0], [10.0, 0, 0], [0, 10.0, 0]])
    est = np.array([[10.1, 0, 0], [50.0, 50.0, 0]])          # one hit, one false alarm
    err = E.associate(est, truth)
    # the optimal assignment pairs the hit with surface 1 and the false alarm with one of
    # the others; the third surface stays unassociated
    assert err[1] == pytest.approx(0.1)
    assert np.sum(np.isnan(err)) == 1
    assert np.all(np.isnan(E.associate(np.zeros((0, 3)), truth)))


def test_rmse_ignores_unassociated_entries():
    e = np.array([[3.0, np.nan], [4.0, 2.0], [np.nan, np.nan]])
    r = E.rmse(e.T, axis=1)
    assert r[0] == pytest.approx(np.sqrt((9 + 16) / 2))
    assert r[1] == pytest.approx(2.0)
    assert np.isnan(E.rmse(np.array([[np.nan, np.nan]]), axis=1)[0])


@pytest.mark.parametrize("coherent", [False, True])
def test_transition_matches_oracle(coherent):
    prm = W.Params(T=0.1, sigma_v=0.5, sigma_sfv=1e-4)
    F, Q = E.transition(prm, 3, 4, coherent)
    s = E.NUISANCE_SIGMA
    Fo, Qo = pcrlb.transition(prm, 3, 4, coherent, s, s, s)
    assert np.allclose(F, Fo, rtol=0, atol=0)
    assert np.allclose(Q, Qo, rtol=1e-14, atol=0)


def test_bound_amplitudes_absorb_path_loss_and_carrier_phase():
    g = W.make_geometry(J=3, Nf=4, My=2, Mz=2)
    prm = W.Params()
    scn = W.make_scenario(g, prm, N=2, K=3, seed=5)
    rho_t = E.bound_amplitudes(scn, 1)
    lam = g.c / g.fc
    for j in range(g.J):
        for k in range(4):
            rp, _ = pcrlb.local_vector(g, j, scn.x_true[1, :3], None if k == 0 else scn.sfv_true[k - 1], k == 0)
            d = np.linalg.norm(rp)
            ref = scn.rho_abs[k] * np.exp(1j * scn.rho_phase[1, j, k]) * lam / (4 * np.pi * d) * np.exp(-2j * np.pi * d / lam)
            assert rho_t[j, k] == pytest.approx(ref, rel=1e-12)


def test_prior_information_matches_the_start():
    prm = W.Params()
    K, J = 4, 4
    for init in ("prior", "truth", "truth_map"):
        Jp = E.prior_information(prm, K, J, True, init)
        d = np.diag(Jp)
        assert Jp.shape == (pcrlb.dims(K, J, True)["dim"],) * 2
        if init == "prior":
            assert d[0] == pytest.approx(12.0 / 8.0 ** 2)
        else:
            assert d[0] == pytest.approx(1.0 / 0.02 ** 2)
        sfv_var = 1.0 / d[6]
        assert sfv_var == pytest.approx(0.02 ** 2 if init == "truth_map" else 16.0 ** 2 / 12.0)
