"""The proposal network on the tensor cores (BF16 operands, FP32 accumulation) against
the FP64 oracle with BF16 rounding at the same places, through the C ABI: forward
outputs, gradients of the mean Gaussian negative log-likelihood, one Adam step, and a
training run that must learn a known conditional Gaussian."""
import numpy as np
import pytest

from oracle import mlp
from paper_2604_19723_gb300 import workload as W

pytestmark = [pytest.mark.gpu]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_19723_gb300 import bp  # noqa: E402

GROUPS = [(name, slice(o, o + int(np.prod(s)))) for (name, s), o in
          zip(mlp.SHAPES, np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])[:-1])]


def data(B, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, 16)).astype(np.float32)
    T = rng.normal(size=(B, 3)).astype(np.float32)
    return X, T


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# accumulation order (FP32 on the tensor cores, FP64 in the oracle) can flip the BF16
# rounding of a stored activation or gradient by one unit (2^-8 relative); through the
# next layer that moves an output by ~1e-3 of its scale, so the bounds are 2e-2 of the
# scale for single elements and 1e-3 on average
@pytest.mark.parametrize("B", [128, 1000, 1])
def test_forward_matches_oracle(B):
    theta = W.mlp_init(5, out_scale=1.0)
    X, _ = data(B, 6)
    net = bp.Mlp(theta)
    y = net.forward(cuda(X)).cpu().numpy().astype(np.float64)
    ref = mlp.forward(theta.astype(np.float64), X.astype(np.float64), bf=True)["y"]
    scale = max(1.0, np.max(np.abs(ref)))
    err = np.abs(y - ref)
    assert err.max() < 2e-2 * scale, err.max()
    assert err.mean() < 1e-3 * scale, err.mean()
    net.close()


@pytest.mark.parametrize("B", [256, 777])
def test_gradients_match_oracle(B):
    theta = W.mlp_init(7, out_scale=0.5)
    X, T = data(B, 8)
    net = bp.Mlp(theta)
    g, lsum = net.grads(cuda(X), cuda(T))
    th = theta.astype(np.float64)
    ref = mlp.backward(th, X.astype(np.float64), T.astype(np.float64), bf=True)
    y = mlp.forward(th, X.astype(np.float64), bf=True)["y"]
    assert lsum == pytest.approx(np.sum(mlp.loss_terms(y, T.astype(np.float64))), rel=1e-3)
    for name, sl in GROUPS:
        scale = np.max(np.abs(ref[sl]))
        assert np.max(np.abs(g[sl] - ref[sl])) < 2e-2 * scale, (name, np.max(np.abs(g[sl] - ref[sl])), scale)
    assert np.all(net.params() == theta)          # gradients only: parameters unchanged
    net.close()


def test_adam_step_matches_oracle():
    theta = W.mlp_init(9, out_scale=0.5)
    X, T = data(512, 10)
    lr = 1e-3
    net = bp.Mlp(theta)
    net.train_step(cuda(X), cuda(T), lr)
    net.sync()
    p1 = net.params().astype(np.float64)
    th = theta.astype(np.float64)
    g = mlp.backward(th, X.astype(np.float64), T.astype(np.float64), bf=True)
    ref, _, _ = mlp.adam(th, g, np.zeros_like(th), np.zeros_like(th), 1, lr)
    # the first step moves each parameter by lr against the sign of its gradient: exact
    # up to FP32 where the gradient is clearly non-zero, a sign either way where the
    # gradient is within the BF16 error of zero
    for name, sl in GROUPS:
        big = np.abs(g[sl]) > 0.05 * np.max(np.abs(g[sl]))
        d = np.abs(p1[sl] - ref[sl])
        assert np.all(d[big] < 1e-3 * lr + 1e-7), name
        assert np.all(d <= 2 * lr + 1e-7), name
    net.close()


def test_training_learns_a_conditional_gaussian():
    """t = A x[:3] + 0.1 n: the trained network's mean loss (oracle, FP64) falls by more
    than 3 nats per row and its predicted log standard deviation approaches log 0.1."""
    rng = np.random.default_rng(11)
    A = rng.normal(size=(3, 3))
    B = 4096
    theta0 = W.mlp_init(12)
    net = bp.Mlp(theta0)
    for step in range(400):
        X = rng.normal(size=(B, 16)).astype(np.float32)
        T = (X[:, :3] @ A.T + 0.1 * rng.normal(size=(B, 3))).astype(np.float32)
        net.train_step(cuda(X), cuda(T), 3e-3)
    net.sync()
    th = net.params().astype(np.float64)
    Xv = rng.normal(size=(2000, 16))
    Tv = Xv[:, :3] @ A.T + 0.1 * rng.normal(size=(2000, 3))
    l0 = mlp.mean_loss(theta0.astype(np.float64), Xv, Tv)
    l1 = mlp.mean_loss(th, Xv, Tv)
    assert l1 < l0 - 3.0, (l0, l1)
    ls = mlp.forward(th, Xv)["y"][:, 3:6]
    assert abs(np.median(ls) - np.log(0.1)) < 0.7, np.median(ls)
    net.close()
