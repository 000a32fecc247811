"""Batches of independent scenarios (bp_batch_*, through the C ABI): ragged shapes
(S, P, Nz and the antenna layout differ per scenario) stepped together on
concurrent streams, replayed from CUDA graphs or launched directly.

  - the time-0 beliefs with S0 PFs equal the oracle's (Sec. V-A, Sec. III-B2);
  - one step of every scenario from an identical exported state matches the FP64
    oracle within the tolerances of the single-filter parity tests;
  - a batch step gives the results of single filters run one after another (with
    shared workspaces, graph replay, and with PF counts that change).
"""
import numpy as np
import pytest

from oracle import beliefs, messages_woodbury, model, synth
from paper_2604_19723_gb300 import workload as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import bp  # noqa: E402

W_TOL = 1e-4
P_TOL = 1e-5
M_TOL = 1e-4

CASES = [
    # (geometry, S PFs, P, seed)
    (dict(J=4, Nf=7, My=1, Mz=1), 2, 256, 31),      # one antenna, Nz = 7
    (dict(J=4, Nf=3, My=2, Mz=2), 3, 300, 32),      # 2 x 2 URA, Nz = 12
    (dict(J=4, Nf=20, My=2, Mz=2), 20, 333, 33),    # FP32 MT path with repairs
    (dict(J=4, Nf=75, My=2, Mz=2), 40, 256, 34),    # Nz = 300, float-float MT path
    (dict(J=4, Nf=10, My=4, Mz=4), 64, 257, 35),    # tensor-core PF path, ragged P
]


def rel_weight_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(b), 1e-300))


def params_for(seed, dynamic=False):
    if dynamic:
        return W.Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4, Q=1, T_pru=1e-3)
    return W.Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4, Q=0, T_pru=0.0)


def make_inputs(cases, dynamic=False):
    """Per scenario: geometry, parameters, a state near the truth and two steps of
    observations (oracle signal model)."""
    out = []
    for geom_kw, S, P, seed in cases:
        g = W.make_geometry(**geom_kw)
        prm = params_for(seed, dynamic)
        scn = W.make_scenario(g, prm, N=3, K=S - 1, seed=seed, snr_db=20.0)
        eta = synth.noise_variance(scn)
        # the observations as the C ABI takes them (complex64), for both sides
        zs = [synth.observe(scn, n, eta, seed + 100 + n).astype(np.complex64).astype(np.complex128) for n in (1, 2)]
        st = W.state_near_truth(scn, P=P, S=S, n=0, seed=seed + 1, eta_true=eta, pos_std=0.005, sfv_std=0.005)
        out.append(dict(g=g, prm=prm, S=S, P=P, seed=seed, st=st, zs=zs))
    return out


def concat_z(batch, inputs, step):
    z = torch.zeros(batch.z_floats(), dtype=torch.float32, device="cuda")
    for i, d in enumerate(inputs):
        o = batch.z_offset(i)
        zi = np.ascontiguousarray(d["zs"][step].astype(np.complex64)).view(np.float32).reshape(-1)
        z[o:o + zi.size] = torch.from_numpy(zi).cuda()
    return z


def gpu_prediction(d, pred_o):
    """The particles a single filter with the scenario's key predicts from d["st"], as an
    oracle Predicted; checked against the oracle's own prediction pred_o."""
    g = d["g"]
    f = bp.Filter(g, d["prm"], P=d["P"], S_max=d["S"], seed=d["seed"])
    f.set_state(d["st"])
    f.predict()
    gp = f.get_predicted()
    f.close()
    assert gp["S"] == pred_o.S and gp["n"] == pred_o.n
    scale = np.maximum(np.abs(pred_o.x.astype(float)), 1.0)
    assert np.max(np.abs(gp["x"] - pred_o.x) / scale) < 1e-6
    assert np.max(np.abs(gp["eta"] - pred_o.eta) / pred_o.eta) < 1e-6
    for k in range(6):
        sc = np.maximum(np.abs(pred_o.phi[:, k].astype(float)), 1e-3 if k >= 3 else 1.0)
        assert np.max(np.abs(gp["phi"][:, k] - pred_o.phi[:, k]) / sc) < 2e-6, k
    assert np.allclose(gp["w_alpha"], pred_o.w_alpha, rtol=1e-14, atol=0)
    assert np.allclose(gp["zeta"], pred_o.zeta, rtol=1e-14, atol=0)
    return model.Predicted(n=pred_o.n, S=pred_o.S, x=gp["x"].copy(), phi=gp["phi"].copy(), eta=gp["eta"].copy(),
                           w_beta=gp["w_beta"].copy(), w_alpha=gp["w_alpha"].copy(), w_xi=gp["w_xi"].copy(),
                           zeta=gp["zeta"].copy(), is_new=pred_o.is_new)


def make_batch(inputs, S_max=None, **kw):
    sc = [(d["g"], d["prm"], d["P"], S_max or d["S"], d["S"], d["seed"]) for d in inputs]
    return bp.Batch(sc, **kw)


def test_time0_beliefs_match_oracle():
    inputs = make_inputs(CASES)
    b = make_batch(inputs, n_streams=3)
    for i, d in enumerate(inputs):
        gs = b.member(i).get_state()
        os_ = model.init_state(d["prm"], d["g"].J, d["P"], d["seed"], S0=d["S"])
        assert gs.S == os_.S == d["S"]
        for key in ("x", "eta", "phi"):
            a, r = getattr(gs, key), getattr(os_, key)
            assert np.max(np.abs(a - r) / np.maximum(np.abs(r), 1e-3)) < 2e-6, (i, key)
        assert np.array_equal(gs.w_x, os_.w_x) and np.array_equal(gs.w_y, os_.w_y)
        assert np.array_equal(gs.p_pr, os_.p_pr)
    b.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_step_matches_oracle(use_graph):
    inputs = make_inputs(CASES)
    # per-scenario workspaces keep the diagnostics of every scenario readable
    b = make_batch(inputs, n_streams=2, shared_workspace=False, use_graph=use_graph)
    for i, d in enumerate(inputs):
        b.member(i).set_state(d["st"])
    b.step(concat_z(b, inputs, 0))
    b.sync()
    for i, d in enumerate(inputs):
        g, prm, st = d["g"], d["prm"], d["st"]
        # the update is compared on the particles the GPU predicted (a single filter with
        # the same key predicts the same particles as the batch); those are checked against
        # the oracle's FP64 prediction at the predict-parity tolerances, as in the
        # single-filter tests, which compare the two stages apart
        pred_o = model.predict(st, prm, g.J, seed=d["seed"], S_max=d["S"])
        pred = gpu_prediction(d, pred_o)
        msg = messages_woodbury.update_messages(pred, prm, g, d["zs"][0])
        bel = beliefs.beliefs(pred, msg)
        est = beliefs.estimate(pred, bel, prm)
        m = b.member(i)
        gw = m.diag_weights(pred.S)
        assert np.max(np.abs(gw["p_pr"] - bel.p_pr)) < P_TOL, i
        assert np.max(np.abs(gw["p_s"] - bel.p_s)) < P_TOL, i
        assert rel_weight_err(gw["w_x"], bel.w_x) < W_TOL, (i, rel_weight_err(gw["w_x"], bel.w_x))
        for j in range(g.J):
            assert rel_weight_err(gw["w_eta"][j], bel.w_eta[j]) < W_TOL, (i, j)
        for s in range(pred.S):
            assert rel_weight_err(gw["w_y"][s], bel.w_y[s]) < W_TOL, (i, s)
        ge = m.estimate()
        assert ge["n"] == 1
        assert np.max(np.abs(ge["x_hat"] - est.x_hat)) < M_TOL, i
        assert np.max(np.abs(ge["eta_hat"] - est.eta_hat) / est.eta_hat) < M_TOL, i
        for s in range(pred.S):
            if est.p_s[s] > 1e-3:
                assert np.max(np.abs(ge["phi_hat"][s, :3] - est.phi_hat[s, :3])) < M_TOL, (i, s)
    b.close()


def run_single(inputs, steps):
    ests = []
    for d in inputs:
        f = bp.Filter(d["g"], d["prm"], P=d["P"], S_max=d["S"], seed=d["seed"])
        f.set_state(d["st"])
        e = []
        for n in range(steps):
            f.step(torch.from_numpy(np.ascontiguousarray(d["zs"][n].astype(np.complex64))).cuda())
            e.append(f.estimate())
        f.close()
        ests.append(e)
    return ests


def close_est(a, b, tol):
    assert a["n"] == b["n"] and a["S"] == b["S"] and a["S_next"] == b["S_next"]
    assert np.allclose(a["x_hat"], b["x_hat"], rtol=tol, atol=tol)
    assert np.allclose(a["p_s"], b["p_s"], rtol=tol, atol=tol)
    assert np.allclose(a["eta_hat"], b["eta_hat"], rtol=tol, atol=0)
    assert np.allclose(a["phi_hat"], b["phi_hat"], rtol=tol, atol=tol)


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_single_filters(use_graph):
    """Two steps with shared workspaces (five scenarios on two streams) against single
    filters.  The kernels and inputs are the same; the only difference allowed is the
    order of FP64 shared-memory atomics in the basis stage (last bits)."""
    inputs = make_inputs(CASES)
    b = make_batch(inputs, n_streams=2, shared_workspace=True, use_graph=use_graph)
    assert len({b.stream_of(i) for i in range(len(inputs))}) == 2
    for i, d in enumerate(inputs):
        b.member(i).set_state(d["st"])
    z = [concat_z(b, inputs, n) for n in (0, 1)]
    got = [[None, None] for _ in inputs]
    for n in range(2):
        b.step(z[n])
        for i in range(len(inputs)):
            got[i][n] = b.member(i).estimate()
    with pytest.raises(bp.BPError):
        b.member(0).diag_weights(inputs[0]["S"])   # workspace shared with other scenarios
    ref = run_single(inputs, 2)
    for i in range(len(inputs)):
        close_est(got[i][0], ref[i][0], 1e-9)
        close_est(got[i][1], ref[i][1], 1e-6)
    b.close()


def test_batch_with_changing_pf_counts():
    """Births (Q = 1) and pruning: the batch launches directly and reads every
    scenario's new PF count back once per batch step."""
    cases = [(dict(J=4, Nf=5, My=2, Mz=2), 3, 256, 41), (dict(J=4, Nf=9, My=1, Mz=1), 2, 300, 42)]
    inputs = make_inputs(cases, dynamic=True)
    b = make_batch(inputs, S_max=8, n_streams=2)
    for i, d in enumerate(inputs):
        b.member(i).set_state(d["st"])
    got = []
    for n in range(2):
        b.step(concat_z(b, inputs, n))
        got.append([b.member(i).estimate() for i in range(len(inputs))])
    ref = []
    for d in inputs:
        f = bp.Filter(d["g"], d["prm"], P=d["P"], S_max=8, seed=d["seed"])
        f.set_state(d["st"])
        e = []
        for n in range(2):
            f.step(torch.from_numpy(np.ascontiguousarray(d["zs"][n].astype(np.complex64))).cuda())
            e.append(f.estimate())
        f.close()
        ref.append(e)
    for n in range(2):
        for i in range(len(inputs)):
            close_est(got[n][i], ref[i][n], 1e-6)
    assert got[0][0]["S"] == inputs[0]["S"] + 1   # one birth in the first step
    b.close()


def test_batch_rejects_bad_arguments():
    g = W.make_geometry(J=4, Nf=4, My=1, Mz=1)
    prm = params_for(0)
    with pytest.raises(bp.BPError):
        bp.Batch([(g, prm, 256, 4, 5, 1)])          # S0 > S_max
    with pytest.raises(bp.BPError):
        bp.Batch([(g, prm, 256, 4, 2, 1)], n_streams=500)


def test_autotuner_picks_the_fastest_measured_configuration():
    """The tuner times every candidate on the batch and returns the fastest; a batch
    built with its choice gives the same estimates as the default configuration."""
    from paper_2604_19723_gb300 import autotune
    inputs = make_inputs(CASES)
    sc = [(d["g"], d["prm"], d["P"], d["S"], d["S"], d["seed"]) for d in inputs]
    b0 = make_batch(inputs, n_streams=2)
    z = torch.stack([concat_z(b0, inputs, 0), concat_z(b0, inputs, 1)])
    b0.close()
    cands = ((1, False), (2, True), (5, True))
    res = autotune.tune_batch(sc, z, candidates=cands, steps=2, warmup=1)
    assert len(res["ms"]) == 3 and all(v > 0 for v in res["ms"].values())
    best_ms = res["ms"][f"{res['best'][0]} streams, graph {res['best'][1]}"]
    assert best_ms == min(res["ms"].values())
    outs = []
    for n_streams, graph in (res["best"], (2, True)):
        b = make_batch(inputs, n_streams=n_streams, use_graph=graph)
        for i, d in enumerate(inputs):
            b.member(i).set_state(d["st"])
        b.step(z[0])
        b.sync()
        outs.append([b.member(i).estimate()["x_hat"] for i in range(len(inputs))])
        b.close()
    for a, c in zip(*outs):
        assert np.max(np.abs(a - c)) < 1e-6
