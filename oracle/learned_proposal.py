"""Oracle of the learned MT proposal (an extension; the paper's MT proposal is the
state-transition PDF).

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the CPU legs of
bench.py; the product path never calls it.

For the prediction at step n with observation z:
  1. xbar = sum_p w_beta^p x_n^p / sum_p w_beta^p (predicted MT mean).
  2. Per PA j, c_j = psi_j(xbar)^H z_j with the LoS steering vector by its plain
     per-element definition (geometry.steering), |z_j|^2, |psi_j|^2; rho_j =
     c_j / sqrt(|z_j|^2 |psi_j|^2).
  3. Shared summary s = [(xbar_pos - ROI centre) / max(ROI half width, 0.5) (3),
     Re, Im of rho_j conj(rho_0) / |rho_0| for j = 1..3 (6, zero for absent PAs),
     |rho_0|].
  4. F x_{n-1}^p = x_n^p - Gamma sigma_v g_prior^p with the prediction's own normals
     (purpose MT_PREDICT); inputs X_p = [(F x_{n-1}^p - xbar)_pos / 0.01,
     (F x_{n-1}^p - xbar)_vel / 0.1, s], held in FP32 like the GPU's input rows.
  5. (mu, log s) = network(X_p) (oracle.mlp with BF16 rounding), log s clamped to [-4, 1];
     g ~ N(0, I) (purpose LEARNED_PROP); u = mu + s g;
     x_n^p = F x_{n-1}^p + Gamma sigma_v u; log r_p = -|u|^2/2 + |g|^2/2 + sum log s.
  6. w_beta^p <- w_beta^p exp(log r_p), normalised to one.
Planar motion (motion_dims = 2) leaves z and v_z alone and drops them from log r.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import geometry, mlp, rng

POS_UNIT, VEL_UNIT, LS_MIN, LS_MAX = 0.01, 0.1, -4.0, 1.0


def predicted_mean(pred) -> np.ndarray:
    w = np.asarray(pred.w_beta, np.float64)
    return pred.x.astype(np.float64) @ w / np.sum(w)


def correlations(geom, z: np.ndarray, xbar: np.ndarray) -> np.ndarray:
    """(J, 4): Re, Im of psi_j(xbar)^H z_j, |z_j|^2, |psi_j|^2."""
    out = np.zeros((geom.J, 4))
    for j in range(geom.J):
        psi = geometry.steering(geom, j, xbar[None, :3], xbar[None, :3], los=True)[0]
        c = np.vdot(psi, z[j])
        out[j] = [c.real, c.imag, np.sum(np.abs(z[j]) ** 2), np.sum(np.abs(psi) ** 2)]
    return out


def summary(params, xbar: np.ndarray, cor: np.ndarray) -> np.ndarray:
    lo, hi = np.asarray(params.p_min, float), np.asarray(params.p_max, float)
    f = np.zeros(10)
    f[:3] = (xbar[:3] - 0.5 * (lo + hi)) / np.maximum(0.5 * (hi - lo), 0.5)
    rho = np.zeros(4, complex)
    for j in range(min(cor.shape[0], 4)):
        nn = cor[j, 2] * cor[j, 3]
        if nn > 0:
            rho[j] = (cor[j, 0] + 1j * cor[j, 1]) / np.sqrt(nn)
    r0 = abs(rho[0])
    for j in range(1, 4):
        t = rho[j] * np.conj(rho[0]) / max(r0, 1e-12)
        f[3 + 2 * (j - 1)] = t.real
        f[4 + 2 * (j - 1)] = t.imag
    f[9] = r0
    return f


def prev_means(pred, params, seed: int):
    """F x_{n-1}^p (6, P) and the prediction's standard normals (3, P)."""
    P = pred.x.shape[1]
    g = np.stack(rng.normals(seed, np.arange(P, dtype=np.uint64), pred.n, rng.MT_PREDICT, 0, 3), axis=0)
    if params.motion_dims == 2:
        g[2] = 0.0
    T, sv = params.T, params.sigma_v
    fx = pred.x.astype(np.float64).copy()
    fx[:3] -= 0.5 * T * T * sv * g
    fx[3:] -= T * sv * g
    return fx, g


@dataclasses.dataclass
class Result:
    xbar: np.ndarray
    cor: np.ndarray
    X: np.ndarray        # (P, 16) inputs (FP32 values)
    Y: np.ndarray        # (P, 16) network outputs
    logr: np.ndarray     # (P,)


def apply(pred, params, geom, z: np.ndarray, theta: np.ndarray, seed: int):
    """The prediction with every MT particle redrawn from the learned proposal and the
    prediction weights multiplied by the transition / proposal ratio."""
    xbar = predicted_mean(pred)
    cor = correlations(geom, z, xbar)
    s = summary(params, xbar, cor)
    fx, _ = prev_means(pred, params, seed)
    P = pred.x.shape[1]
    X = np.zeros((P, 16))
    X[:, :3] = ((fx[:3] - xbar[:3, None]) / POS_UNIT).T
    X[:, 3:6] = ((fx[3:] - xbar[3:, None]) / VEL_UNIT).T
    X[:, 6:] = s[None, :]
    X = X.astype(np.float32).astype(np.float64)
    Y = mlp.forward(np.asarray(theta, np.float64), X, bf=True)["y"]
    g = np.stack(rng.normals(seed, np.arange(P, dtype=np.uint64), pred.n, rng.LEARNED_PROP, 0, 3), axis=0)
    T, sv = params.T, params.sigma_v
    dims = 3 if params.motion_dims == 3 else 2
    x = pred.x.astype(np.float64).copy()
    logr = np.zeros(P)
    for k in range(dims):
        mu = Y[:, k]
        ls = np.clip(Y[:, 3 + k], LS_MIN, LS_MAX)
        u = mu + np.exp(ls) * g[k]
        logr += -0.5 * u * u + 0.5 * g[k] * g[k] + ls
        x[k] = fx[k] + 0.5 * T * T * sv * u
        x[3 + k] = fx[3 + k] + T * sv * u
    w = np.asarray(pred.w_beta, np.float64) * np.exp(logr)
    w /= np.sum(w)
    new = dataclasses.replace(pred, x=x.astype(np.float32), w_beta=w)
    return new, Result(xbar=xbar, cor=cor, X=X, Y=Y, logr=logr)
