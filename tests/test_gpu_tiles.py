"""Kernel tile shapes (bp_set_tiles) and their autotuner, through the C ABI.

  * the tile fields are validated on the host;
  * every candidate the tuner measures (PF-likelihood column buckets S~ = 16, 24, 32, 48,
    64, one or two blocks per SM, a quarter frequency chunk, tensor-core kernel on or
    off, at 64 columns and, for arrays of 32 or more elements, at 32; message-table
    particle chunks) gives the FP64 oracle's update within the
    parity tolerances (Supplementary Sec. S-V: the PF message kappa~ in the
    eigen-whitened basis does not depend on how its columns are tiled);
  * the tuner keeps the measured minimum and leaves it on the filter;
  * a batch tuned per shape class steps to the results of the untuned batch.
"""
import numpy as np
import pytest

from oracle import beliefs, messages_woodbury, model, synth
from paper_2604_19723_gb300 import workload as W

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import autotune as A  # noqa: E402
from paper_2604_19723_gb300 import bp  # noqa: E402

W_TOL = 1e-4
P_TOL = 1e-5

CASES = [
    # (geometry, S, S_max, P, seed)
    (dict(J=4, Nf=6, My=2, Mz=2), 12, 16, 300, 61),      # bucket 16 only
    (dict(J=4, Nf=20, My=2, Mz=2), 20, 20, 333, 62),     # buckets 24, 32; two blocks per SM
    (dict(J=4, Nf=10, My=4, Mz=4), 40, 64, 257, 63),     # bucket 48, 64 on the tensor cores or not
    (dict(J=4, Nf=75, My=2, Mz=2), 40, 40, 256, 64),     # buckets 48, 64 (CUDA-core), frequency chunks
    (dict(J=4, Nf=6, My=4, Mz=8), 40, 64, 300, 65),      # 4 x 8 array: tensor-core rounds of half a frequency
    (dict(J=4, Nf=3, My=8, Mz=8), 28, 32, 300, 66),      # 8 x 8 array: the 32-column tensor-core kernel or not
]


def rel_weight_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(b), 1e-300))


def setup(geom_kw, S, S_max, P, seed):
    g = W.make_geometry(**geom_kw)
    prm = W.Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4, Q=0, T_pru=0.0)
    scn = W.make_scenario(g, prm, N=3, K=S - 1, seed=seed, snr_db=20.0)
    eta = synth.noise_variance(scn)
    # the observation as the C ABI takes it (complex64), for both sides
    z = synth.observe(scn, 1, eta, seed + 100).astype(np.complex64).astype(np.complex128)
    st = W.state_near_truth(scn, P=P, S=S, n=0, seed=seed + 1, eta_true=eta, pos_std=0.005, sfv_std=0.005)
    pred = model.predict(st, prm, g.J, seed=seed, S_max=S_max)
    return g, prm, z, st, pred, scn, eta


def gpu_update(g, prm, pred, z, P, S_max, seed, tiles):
    f = bp.Filter(g, prm, P=P, S_max=S_max, seed=seed)
    f.set_tiles(**tiles)
    assert all(f.get_tiles()[k] == v for k, v in tiles.items())
    f.set_predicted(pred.n, pred.S, pred.x, pred.phi, pred.eta, pred.w_beta, pred.w_alpha, pred.w_xi, pred.zeta)
    f.update(torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda())
    torch.cuda.synchronize()
    return f


def test_tile_fields_are_validated():
    g = W.make_geometry(J=2, Nf=4, My=2, Mz=2)
    f = bp.Filter(g, W.Params(), P=64, S_max=8, seed=1)
    assert f.get_tiles() == {k: 0 for k in bp.TILE_FIELDS}
    for bad in (dict(kappa_sc=20), dict(kappa_blocks=3), dict(kappa_tc=2), dict(table_chunk=48),
                dict(kappa_fch=-1), dict(table_split=-2)):
        with pytest.raises(bp.BPError):
            f.set_tiles(**bad)
        assert f.get_tiles() == {k: 0 for k in bp.TILE_FIELDS}   # nothing changed
    f.set_tiles(kappa_sc=16, kappa_blocks=1, kappa_fch=2, kappa_tc=-1, table_chunk=32, table_split=3)
    assert f.get_tiles() == dict(kappa_sc=16, kappa_blocks=1, kappa_fch=2, kappa_tc=-1, table_chunk=32, table_split=3)
    with pytest.raises(ValueError):
        f.set_tiles(kappa_columns=8)
    f.close()


@pytest.mark.parametrize("case", CASES)
def test_every_tile_candidate_matches_the_oracle(case):
    geom_kw, S, S_max, P, seed = case
    g, prm, z, st, pred, _, _ = setup(geom_kw, S, S_max, P, seed)
    msg = messages_woodbury.update_messages(pred, prm, g, z)
    bel = beliefs.beliefs(pred, msg)
    dk = (msg.log_kappa1 - msg.log_kappa0[:, :, None]).sum(1)
    cands = A.kappa_candidates(S, S_max, g) + [dict(kappa_sc=0, table_chunk=c) for c in (16, 32, 64)] + \
        [dict(table_split=2)]
    for c in cands:
        f = gpu_update(g, prm, pred, z, P, S_max, seed, c)
        gw = f.diag_weights(pred.S)
        ll = f.diag_loglik(pred.S)
        f.close()
        rep = dict(p_s=float(np.max(np.abs(gw["p_s"] - bel.p_s))),
                   w_x=rel_weight_err(gw["w_x"], bel.w_x),
                   w_y=max(rel_weight_err(gw["w_y"][s], bel.w_y[s]) for s in range(pred.S)),
                   dkappa=float(np.max(np.abs(ll["delta_kappa"] - dk) / np.maximum(1.0, 1e-6 * np.abs(dk)))))
        print(c, rep)
        assert rep["p_s"] < P_TOL and rep["w_x"] < W_TOL and rep["w_y"] < W_TOL, (c, rep)


def test_tuner_keeps_the_measured_minimum():
    geom_kw, S, S_max, P, seed = CASES[1]
    g, prm, z, st, pred, scn, eta = setup(geom_kw, S, S_max, 4096, seed)
    f = bp.Filter(g, prm, P=4096, S_max=S_max, seed=seed)
    f.set_state(st)
    zc = torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda()
    res = A.tune_tiles(f, zc, reps=2)
    k_best = min(res["kappa_ms"], key=res["kappa_ms"].get)
    t_best = min(res["table_ms"], key=res["table_ms"].get)
    want = {**A._parse(k_best), **A._parse(t_best)}
    assert all(res["best"][k] == v for k, v in want.items())
    assert f.get_tiles() == res["best"]
    assert len(res["kappa_ms"]) == len(A.kappa_candidates(S, S_max, g))
    f.close()


def test_batch_tuned_per_shape_class_steps_like_the_untuned_batch():
    cases = [(dict(J=4, Nf=20, My=2, Mz=2), 20, 400, 71), (dict(J=4, Nf=22, My=2, Mz=2), 22, 300, 72),
             (dict(J=4, Nf=10, My=4, Mz=4), 40, 257, 73)]
    inputs = []
    for geom_kw, S, P, seed in cases:
        g = W.make_geometry(**geom_kw)
        prm = W.Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4, Q=0, T_pru=0.0)
        scn = W.make_scenario(g, prm, N=3, K=S - 1, seed=seed, snr_db=20.0)
        eta = synth.noise_variance(scn)
        z = synth.observe(scn, 1, eta, seed + 100)
        stt = W.state_near_truth(scn, P=P, S=S, n=0, seed=seed + 1, eta_true=eta, pos_std=0.005, sfv_std=0.005)
        inputs.append(dict(g=g, prm=prm, S=S, P=P, seed=seed, st=stt, z=z))
    sc = [(d["g"], d["prm"], d["P"], d["S"], d["S"], d["seed"]) for d in inputs]
    out = []
    for tuned in (False, True):
        b = bp.Batch(sc, n_streams=2, shared_workspace=False, use_graph=True)
        for i, d in enumerate(inputs):
            b.member(i).set_state(d["st"])
        zt = torch.zeros(b.z_floats(), dtype=torch.float32, device="cuda")
        for i, d in enumerate(inputs):
            zi = np.ascontiguousarray(d["z"].astype(np.complex64)).view(np.float32).reshape(-1)
            zt[b.z_offset(i):b.z_offset(i) + zi.size] = torch.from_numpy(zi).cuda()
        if tuned:
            res = A.tune_batch_tiles(b, sc, zt, reps=1)
            # the two 2 x 2-URA scenarios with S~ = 24 share a class; the 4 x 4-URA one has its own
            assert len(res) == 2 and sorted(v["scenarios"] for v in res.values()) == [1, 2]
            for i, d in enumerate(inputs):            # the tuner stepped single filters, not the batch
                b.member(i).set_state(d["st"])
        b.step(zt)
        b.sync()
        out.append([b.member(i).diag_weights(d["S"]) for i, d in enumerate(inputs)])
        b.close()
    for a, t in zip(out[0], out[1]):
        assert rel_weight_err(t["w_x"], a["w_x"]) < W_TOL
        for s in range(a["w_y"].shape[0]):
            assert rel_weight_err(t["w_y"][s], a["w_y"][s]) < W_TOL
        assert np.max(np.abs(t["p_s"] - a["p_s"])) < P_TOL
