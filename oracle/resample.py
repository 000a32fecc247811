"""Systematic resampling and regularisation (oracle, FP64; test infrastructure only).

Systematic resampling follows Arulampalam et al. (2002), Algorithm 2, as cited
in Sec. IV-D: one uniform U per belief, u_i = (U + i)/P for i = 0..P-1, and
particle i takes the first index k whose cumulative weight c_k >= u_i
(c is accumulated in FP64 and its last entry set to 1).

Regularisation (Sec. IV-D, citing Musso et al. 2001, p. 253): every resampled
particle is moved by h_opt L eps with L L^T the weighted covariance of the
belief before resampling, eps ~ N(0, I) and the Gaussian-kernel optimum
h_opt = (4/(P (d + 2)))^(1/(d + 4)) for d active dimensions (reading R8).
Dimensions that do not move (LoS p_sfv, mu in the ZM variant, z and v_z in
planar motion) have zero covariance and receive no jitter.  gamma and eta are
reflected at 0.  Pins: P7 (|N_i - P w_i| < 1) and the covariance of the jitter.
"""
from __future__ import annotations

import numpy as np

from . import rng


def systematic_indices(w: np.ndarray, U: float) -> np.ndarray:
    P = len(w)
    c = np.cumsum(np.asarray(w, np.float64))
    c = c / c[-1] if c[-1] > 0 else np.linspace(1.0 / P, 1.0, P)
    c[-1] = 1.0
    u = (U + np.arange(P, dtype=np.float64)) / P
    return np.searchsorted(c, u, side="left")


def resample_uniform(seed: int, n: int, kind: int, index: int) -> float:
    """U for belief (kind, index): kind 0 = MT, 1 = PF slot, 2 = eta_j."""
    x = rng.draw(seed, np.array([(kind << 16) | index], np.uint64), n, rng.RESAMPLE, 0, 0)
    return float(rng.u32d(x[0])[0])


def weighted_cov(X: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_p w_p (X_p - m)(X_p - m)^T with normalised w; X (d, P)."""
    w = w / w.sum()
    m = X @ w
    D = X - m[:, None]
    return (D * w) @ D.T


def cholesky_zeroing(C: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor; a pivot <= 0 yields a zero column (no jitter there)."""
    d = C.shape[0]
    L = np.zeros_like(C)
    for k in range(d):
        piv = C[k, k] - np.dot(L[k, :k], L[k, :k])
        if piv <= 0.0:
            continue
        L[k, k] = np.sqrt(piv)
        for i in range(k + 1, d):
            L[i, k] = (C[i, k] - np.dot(L[i, :k], L[k, :k])) / L[k, k]
    return L


def h_opt(P: int, d: int) -> float:
    return (4.0 / (P * (d + 2.0))) ** (1.0 / (d + 4.0))


def mt_active(params) -> np.ndarray:
    a = np.ones(6, bool)
    if params.motion_dims == 2:
        a[2] = a[5] = False
    return a


def pf_active(params, s: int) -> np.ndarray:
    a = np.ones(6, bool)
    if s == 0:
        a[:3] = False
    elif params.motion_dims == 2:
        a[2] = False
    if params.zero_mean:
        a[4:] = False
    return a


def _jitter(X, w, active, seed, n, purpose, sub, P):
    d = int(active.sum())
    C = weighted_cov(X.astype(np.float64), w)
    C[~active, :] = 0.0
    C[:, ~active] = 0.0
    L = cholesky_zeroing(C)
    eps = np.array(rng.normals(seed, np.arange(P, dtype=np.uint64), n, purpose, sub, X.shape[0]))
    return h_opt(P, d) * (L @ eps)


def resample_and_regularize(pred, bel, keep, params, seed: int):
    """Resample every belief independently and jitter (Sec. IV-D).  `keep` lists
    the PF slots that survive pruning, in order; they are compacted to 0..len-1.
    Returns the new state (FP32 particles) and the index arrays used."""
    from paper_2604_19723_gb300.workload import StateArrays
    n = pred.n
    P = pred.x.shape[1]
    J = pred.eta.shape[0]
    X = pred.x.astype(np.float64)
    idx_x = systematic_indices(bel.w_x, resample_uniform(seed, n, 0, 0))
    xn = X[:, idx_x]
    if params.regularize:
        xn = xn + _jitter(X, bel.w_x, mt_active(params), seed, n, rng.JITTER_MT, 0, P)
    S2 = len(keep)
    phin = np.zeros((S2, 6, P))
    idx_y = []
    for t, s in enumerate(keep):
        ws = bel.w_y[s]
        ps = ws.sum()
        Y = pred.phi[s].astype(np.float64)
        ii = systematic_indices(ws / ps if ps > 0 else np.full(P, 1.0 / P), resample_uniform(seed, n, 1, int(s)))
        idx_y.append(ii)
        phin[t] = Y[:, ii]
        if params.regularize and ps > 0:
            phin[t] = phin[t] + _jitter(Y, ws, pf_active(params, s), seed, n, rng.JITTER_PF, int(s), P)
        phin[t, 3] = np.abs(phin[t, 3])
    etan = np.zeros((J, P))
    idx_e = []
    for j in range(J):
        E = pred.eta[j].astype(np.float64)
        ii = systematic_indices(bel.w_eta[j], resample_uniform(seed, n, 2, j))
        idx_e.append(ii)
        etan[j] = E[ii]
        if params.regularize:
            etan[j] = etan[j] + _jitter(E[None], bel.w_eta[j], np.ones(1, bool), seed, n, rng.JITTER_ETA, j, P)[0]
        etan[j] = np.abs(etan[j])
    p_s = bel.p_s[keep]
    st = StateArrays(n=n, S=S2, x=xn.astype(np.float32), phi=phin.astype(np.float32),
                     eta=etan.astype(np.float32), w_x=np.full(P, 1.0 / P),
                     w_y=p_s[:, None] * np.full((S2, P), 1.0 / P), w_eta=np.full((J, P), 1.0 / P),
                     p_pr=bel.p_pr[keep].copy())
    return st, idx_x, idx_y, idx_e
