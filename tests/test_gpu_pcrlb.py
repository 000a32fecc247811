"""Posterior CRLBs (Sec. VI, Supplementary Sec. S-VII) on the GPU against the FP64 oracle,
through the C ABI: the Bayesian snapshot FIM (mean over state realisations) for the
coherent and the noncoherent parameterisation, and the information recursion with the
position and mapping error bounds."""
import numpy as np
import pytest

from oracle import pcrlb
from paper_2604_19723_gb300 import workload as W

pytestmark = [pytest.mark.gpu]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import bp  # noqa: E402


def realisations(g, K, M, seed):
    r = np.random.default_rng(seed)
    x = np.zeros((M, 6))
    x[:, :3] = np.array([1.0, 2.0, 0.3]) + 0.2 * r.standard_normal((M, 3))
    x[:, 3:] = 0.3 * r.standard_normal((M, 3))
    base = np.array([[9.0, 3.0, 0.5], [-5.0, 6.0, 1.0], [2.0, -4.0, -1.0], [4.0, 9.5, 0.2]])[:K]
    sfv = base[None] + 0.05 * r.standard_normal((M, K, 3))
    rho = (0.3 + r.random((M, g.J, K + 1))) * np.exp(1j * r.uniform(-np.pi, np.pi, (M, g.J, K + 1)))
    return x, sfv, rho


@pytest.mark.parametrize("coherent", [False, True])
@pytest.mark.parametrize("shape", [dict(J=2, Nf=4, My=2, Mz=2), dict(J=4, Nf=10, My=4, Mz=4)])
def test_snapshot_fim_matches_oracle(coherent, shape):
    g = W.make_geometry(**shape)
    K, M, eta = 3, 6, 2e-3
    x, sfv, rho = realisations(g, K, M, 7)
    gpu = bp.pcrlb_fim(g, x, sfv, rho, eta, coherent)
    ref = np.mean([pcrlb.snapshot_fim(g, x[m], sfv[m], rho[m], eta, coherent) for m in range(M)], axis=0)
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref))) + 1e-300
    assert np.max(np.abs(gpu - ref) / scale) < 1e-9


def test_recursion_matches_oracle():
    g = W.make_geometry(J=3, Nf=6, My=2, Mz=2)
    K, eta, coherent = 2, 2e-3, True
    prm = W.Params(motion_dims=3)
    dd = pcrlb.dims(K, g.J, coherent)
    Js = []
    for n in range(4):
        x, sfv, rho = realisations(g, K, 5, 20 + n)
        Js.append(np.mean([pcrlb.snapshot_fim(g, x[m], sfv[m], rho[m], eta, coherent) for m in range(5)], axis=0))
    F, Q = pcrlb.transition(prm, K, g.J, coherent, 10.0, 10.0, 10.0)
    J10 = np.linalg.inv(Q + 1e-2 * np.eye(dd["dim"]))
    post = pcrlb.recursion(Js, F, Q, J10)
    peb, meb = bp.pcrlb_recursion(F, Q, J10, np.stack(Js), K)
    for n in range(4):
        p_ref, m_ref = pcrlb.bounds(post[n], K)
        assert peb[n] == pytest.approx(p_ref, rel=1e-8)
        assert np.allclose(meb[n], m_ref, rtol=1e-8)
    # the SFVs barely move (sigma_sfv = 0.1 mm): their information accumulates step by step
    assert np.all(np.diff(meb, axis=0) < 0)
