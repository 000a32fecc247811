"""Host logic of the kernel tile tuner (no GPU): the candidate tile sets it measures and
the shape classes a batch is tuned by."""
from paper_2604_19723_gb300 import autotune as A
from paper_2604_19723_gb300 import workload as W


def test_kappa_candidates_hold_S_within_the_basis_stride():
    for geom_kw in (dict(J=4, Nf=10, My=4, Mz=4), dict(J=4, Nf=75, My=2, Mz=2), dict(J=4, Nf=7, My=1, Mz=1)):
        g = W.make_geometry(**geom_kw)
        for S_max in (1, 5, 8, 9, 16, 20, 24, 30, 32, 40, 48, 64):
            for S in range(1, S_max + 1):
                cands = A.kappa_candidates(S, S_max, g)
                assert cands, (S, S_max)
                top = A.basis_stride(S_max)
                for c in cands:
                    assert S <= c["kappa_sc"] <= top and c["kappa_sc"] in A.BUCKETS
                    # two blocks per SM only where the kernel is compiled for it (buckets <= 32)
                    assert c["kappa_blocks"] in (0, 1, 2)
                    assert c["kappa_blocks"] != 2 or c["kappa_sc"] in (24, 32)
                    # the tensor-core kernel only for its shapes and the 64-column bucket
                    if c["kappa_tc"] == 1:
                        assert c["kappa_sc"] == 64 and A.tensor_core_shape(g, S_max)
                # the smallest bucket that holds S is always among them
                smallest = next(b for b in A.BUCKETS if b >= S)
                assert any(c["kappa_sc"] == smallest for c in cands)


def test_tensor_core_shape_matches_the_kernel_rules():
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=4, Mz=4), 64)
    assert not A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=4, Mz=4), 32)     # stride 32
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=75, My=2, Mz=2), 64)         # frequencies grouped
    assert not A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=8, Mz=8), 64)     # 2 My Mz = 128
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=16, My=2, Mz=2), 64)


def test_shape_classes_group_equal_shapes():
    g1 = W.make_geometry(J=4, Nf=20, My=2, Mz=2)
    g2 = W.make_geometry(J=4, Nf=22, My=2, Mz=2)
    g3 = W.make_geometry(J=4, Nf=40, My=2, Mz=2)
    assert A.shape_class(g1, 1000, 20, 20) == A.shape_class(g2, 5000, 22, 24)   # bucket 24, Nf range 2
    assert A.shape_class(g1, 1000, 20, 20) != A.shape_class(g3, 1000, 20, 20)   # Nf range differs
    assert A.shape_class(g1, 1000, 20, 20) != A.shape_class(g1, 1000, 30, 32)   # bucket differs


def test_keys_round_trip():
    d = dict(kappa_sc=24, kappa_blocks=2, kappa_fch=5, kappa_tc=-1)
    assert A._parse(A._key(d)) == d
