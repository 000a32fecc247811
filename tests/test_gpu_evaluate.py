"""Monte Carlo evaluation of the variants (Sec. VII) end to end on the GPU: observations
synthesised by bp_synthesize, the filter stepped through the C ABI, the bounds from
bp_pcrlb_fim and bp_pcrlb_recursion.  A small run (2 runs x 30 steps, the tracking
phase: map in place at time 0, births on)."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
pytest.importorskip("scipy")

from paper_2604_19723_gb300 import evaluate as E  # noqa: E402


def test_variants_track_and_bounds_order():
    res = E.evaluate("paper_exp1_proposal", ("nzm", "zm", "nzm_nc"), runs=2, steps=30, P=8000, seed=300,
                     init="truth_map")
    v = res["variants"]
    for name, d in v.items():
        assert all(f < 0 for f in d["failed"]), name
        assert len(d["rmse_pos"]) == 30 and np.all(np.isfinite(d["rmse_pos"]))
        assert np.all(np.isfinite(d["peb"])) and np.all(np.asarray(d["peb"]) > 0)
        # the map is in place at time 0: the MT stays within a few centimetres
        assert d["median_pos"][-1] < 0.1, (name, d["median_pos"][-1])
    # the coherent bound uses the same data with fewer nuisance phases: never above the
    # noncoherent one (same truth: seeds equal across variants)
    peb_c, peb_nc = np.asarray(v["nzm"]["peb"]), np.asarray(v["nzm_nc"]["peb"])
    assert np.all(peb_c <= peb_nc * (1 + 1e-9))
    # information accumulates: the position bound after 30 steps is below the start's
    assert peb_c[-1] < peb_c[0]
