"""Host logic of the kernel tile tuner (no GPU): the candidate tile sets it measures and
the shape classes a batch is tuned by."""
from paper_2604_19723_gb300 import autotune as A
from paper_2604_19723_gb300 import workload as W


def test_kappa_candidates_hold_S_within_the_basis_stride():
    for geom_kw in (dict(J=4, Nf=10, My=4, Mz=4), dict(J=4, Nf=75, My=2, Mz=2), dict(J=4, Nf=7, My=1, Mz=1),
                    dict(J=4, Nf=16, My=8, Mz=8)):
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
                    # the tensor-core kernel only for its shapes, at the basis stride's width
                    if c["kappa_tc"] == 1:
                        assert c["kappa_sc"] == top and A.tensor_core_shape(g, S_max)
                # the smallest bucket that holds S is always among them
                smallest = next(b for b in A.BUCKETS if b >= S)
                assert any(c["kappa_sc"] == smallest for c in cands)


def test_tensor_core_shape_matches_the_kernel_rules():
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=4, Mz=4), 64)
    assert not A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=4, Mz=4), 32)     # stride 32
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=75, My=2, Mz=2), 64)         # frequencies grouped
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=16, My=2, Mz=2), 64)
    # arrays of 32 or more elements (a multiple of 16): rounds within a frequency, 64 or 32 columns
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=16, My=8, Mz=8), 32)         # the stress shape
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=8, Mz=8), 64)
    assert A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=4, Mz=8), 32)
    assert not A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=8, Mz=8), 16)     # stride 16
    assert not A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=4, Mz=4), 32)     # small array, stride 32
    assert not A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=8, Mz=1), 64)     # Mz odd
    assert not A.tensor_core_shape(W.make_geometry(J=4, Nf=10, My=5, Mz=8), 64)     # 40 elements
    assert not A.tensor_core_shape(W.make_geometry(J=4, Nf=800, My=8, Mz=8), 64)    # r0 over the shared memory


def test_tensor_core_shared_memory_matches_the_kernel_figures():
    # the 4 x 4 URA at Nf = 10 with 64 columns: 87 584 B (two blocks per SM); the 8 x 8 URA at
    # Nf = 16 with 32 and 64 columns: 111 152 and 111 664 B, within the 115 712 B that two
    # blocks per SM allow (228 KB per SM, 1 KB reserved per block)
    assert A.tensor_core_smem(W.make_geometry(J=4, Nf=10, My=4, Mz=4), 64) == 87584
    assert A.tensor_core_smem(W.make_geometry(J=4, Nf=16, My=8, Mz=8), 32) == 111152
    assert A.tensor_core_smem(W.make_geometry(J=4, Nf=16, My=8, Mz=8), 64) == 111664
    for w in (32, 64):
        assert A.tensor_core_smem(W.make_geometry(J=4, Nf=16, My=8, Mz=8), w) <= 233472 // 2 - 1024


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
