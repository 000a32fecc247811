"""The checked build (-DBP_CHECKED: data-dependent indices range-checked on the device,
a failed check raises a flag that bp_estimate reports) runs a full step, resampling and
compaction included, with no check firing and the results of the normal build.  Built
on demand; runs in a subprocess because the library is chosen at load time."""
import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
from oracle import beliefs, messages_woodbury, model, synth
from paper_2604_19723_gb300 import bp, workload as W
assert bp.LIB_PATH.endswith("libbp_checked.so"), bp.LIB_PATH
g = W.make_geometry(J=2, Nf=6, My=2, Mz=2)
prm = W.Params(Q=1, T_pru=0.2)
scn = W.make_scenario(g, prm, N=4, K=3, seed=101)
eta = synth.noise_variance(scn)
st = W.state_near_truth(scn, P=700, S=4, n=0, seed=102, eta_true=eta)
f = bp.Filter(g, prm, P=700, S_max=8, seed=103)
f.set_state(st)
for n in range(1, 4):
    z = synth.observe(scn, n, eta, 104 + n).astype(np.complex64)
    f.step(torch.from_numpy(z).cuda())
    e = f.estimate()          # raises BPError (BP_ERR_STATE) if an index check fired
print("checked ok", e["S"], e["x_hat"][:3])
"""


def test_checked_build_runs_steps_without_a_failed_check():
    sys.path.insert(0, ROOT)
    from paper_2604_19723_gb300 import build as b
    b.build(checked=True)
    env = dict(os.environ, BP_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, cwd=ROOT, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked ok" in r.stdout
