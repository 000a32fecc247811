"""The allocation-free resampler (bp_resample_noalloc) against the resampling
bp_update performs, through the C ABI.

Callers that cannot allocate device memory (graph-captured code, real-time
loops, hosts with their own allocator) use this entry point; its scratch is a
static device array shared by all calls.  Two calls in a row must reproduce the
indices of the existing path for the same weights and draws (index work: exact,
except where u_i lies within rounding of a step of the cumulative weights).
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import model, synth
from paper_2604_19723_gb300 import workload as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import bp  # noqa: E402


def _check(idx_new, idx_ref, w, U):
    P = len(w)
    c = np.cumsum(w) / np.sum(w)
    u = (U + np.arange(P)) / P
    for i in np.nonzero(idx_new != idx_ref)[0]:
        k = min(idx_new[i], idx_ref[i])
        assert abs(c[k] - u[i]) < 1e-12, i
    assert np.mean(idx_new != idx_ref) < 1e-3


def test_noalloc_resampler_matches_update_path():
    g = W.make_geometry(J=2, Nf=6, My=3, Mz=2)
    prm = W.Params(T_pru=0.0)
    scn = W.make_scenario(g, prm, N=2, K=3, seed=61)
    eta = synth.noise_variance(scn)
    z = synth.observe(scn, 1, eta, 62)
    P, seed = 3000, 63
    st = W.state_near_truth(scn, P=P, S=4, n=0, seed=64, eta_true=eta, pos_std=0.02, sfv_std=0.02)
    pred = model.predict(st, prm, g.J, seed=seed, S_max=8)
    f = bp.Filter(g, prm, P=P, S_max=8, seed=seed)
    f.set_predicted(pred.n, pred.S, pred.x, pred.phi, pred.eta, pred.w_beta, pred.w_alpha, pred.w_xi, pred.zeta)
    f.update(torch.from_numpy(z.astype(np.complex64)).cuda())
    gw = f.diag_weights(pred.S)
    gi = f.diag_indices(pred.S)
    cases = [(gw["w_x"], gi["x"], 0, 0), (gw["w_eta"][1], gi["eta"][1], 2, 1)]
    for w_host, idx_ref, kind, index in cases:       # two calls in a row
        w = torch.from_numpy(np.ascontiguousarray(w_host)).cuda()
        idx = bp.resample_noalloc(w, seed, pred.n, kind, index)
        torch.cuda.synchronize()
        U = ((int(_philox_u0(seed, (kind << 16) | index, pred.n)) + 0.5) * 2.0 ** -32)
        _check(idx.cpu().numpy(), idx_ref, w_host, U)
    f.close()


def test_noalloc_smaller_call_after_larger_on_a_side_stream():
    """The static scratch keeps the previous call's contents: a P = 3000 call after a
    P = 5000 call must not see the larger call's cumulative weights.  Both run on a
    non-default stream; the indices equal the plain systematic rule on the host."""
    r = np.random.default_rng(65)
    s = torch.cuda.Stream()
    for P in (5000, 3000):
        w_host = r.gamma(0.4, size=P)
        w = torch.from_numpy(w_host).cuda()
        with torch.cuda.stream(s):
            idx = bp.resample_noalloc(w, 66, 3, 1, 2, stream=s)
        s.synchronize()
        U = ((int(_philox_u0(66, (1 << 16) | 2, 3)) + 0.5) * 2.0 ** -32)
        c = np.cumsum(w_host) / np.sum(w_host)
        c[-1] = 1.0
        ref = np.searchsorted(c, (U + np.arange(P)) / P, side="left")
        _check(idx.cpu().numpy(), ref, w_host, U)


def test_noalloc_rejects_capacity():
    w = torch.ones(bp.NOALLOC_MAX_P + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(bp.BPError) as e:
        bp.resample_noalloc(w, 1, 1, 0, 0)
    assert e.value.status == 3


def _philox_u0(seed, item, n):
    """First word of the Philox block the library draws U from (test-side recomputation
    from the published Philox4x32-10 definition, via the oracle's generator)."""
    from oracle import rng
    return rng.draw(seed, np.array([item], np.uint64), n, rng.RESAMPLE, 0, 0)[0][0]
