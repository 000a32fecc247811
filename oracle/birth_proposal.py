"""Oracle of the birth proposal PDF (Sec. IV-D, "An Efficient Birth Proposal PDF").

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the CPU legs of
bench.py; the product path never calls it.

For each new PF (partition q of the birth box) the spatial part of the birth density is
replaced by a Gaussian proposal N(mu_q, C_q) built from the observation residual that the
LoS and the legacy PFs do not explain:

  1. x_hat = sum_p w_beta^p x^p (predicted MT MMSE estimate) and, per legacy PF s, the
     MMSE estimate of its position.  Reading: the PF estimates are taken as the means of
     the legacy PFs' prediction messages (the random walk of the PF state has zero mean,
     so these equal the MMSE estimates of step n-1 in expectation; the update receives
     the predicted particles only).
  2. Psi_j = [psi_j(x_hat, phi_0) ... psi_j(x_hat, phi_{S_L-1})] (LoS in column 0) and the
     residual z~_j = (I - Psi_j Psi_j^+) z_j (projector onto the orthogonal complement of
     the column space; minimum-norm least squares).
  3. N_g candidate positions p_i ~ U(P_q) (Philox, purpose BIRTH_CAND, item i, sub q).
  4. Coherent Bartlett spectrum c_i = | sum_j (1/Nz) z~_j^H psi_j(x_hat, p_i) |^2, weights
     w_i = c_i / sum c.
  5. mu_q = p_{i*}, i* = argmax_i c_i (the first maximum); C_q = sum_i w_i (p_i - mu_q)
     (p_i - mu_q)^T.
  6. Particles of the new PF: p^(p) = mu_q + L_q g^(p) with L_q the zeroing Cholesky factor
     of C_q and g^(p) standard normals (purpose BIRTH_PROP, sub = PF slot); gamma and mu
     from their birth priors exactly as in the plain birth (same draws).
  7. Weights w_alpha^(p) proportional to 1_{P_q}(p^(p)) / N(p^(p); mu_q, C_q) on the
     dimensions with a positive pivot; since p^(p) - mu_q = L_q g^(p), the Mahalanobis
     distance is |g^(p)|^2 over those dimensions, so the unnormalised weight is
     1_{P_q}(p^(p)) exp(|g_A^(p)|^2 / 2) (the Gaussian's constant cancels in the
     normalisation).  The weights are scaled to sum to p_B, the PF's birth existence.

Every steering vector here is formed per antenna element by the plain definition
(geometry.steering); numbers are FP64.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import geometry, model, resample, rng


@dataclasses.dataclass
class Proposal:
    """The proposal of one new PF (partition q)."""
    q: int
    slot: int
    costs: np.ndarray      # (N_g,) Bartlett spectrum at the candidates
    cand: np.ndarray       # (N_g, 3) candidate positions
    i_star: int
    mu: np.ndarray         # (3,)
    C: np.ndarray          # (3, 3)
    L: np.ndarray          # (3, 3) zeroing Cholesky factor


def partition_bounds(params, Q: int, q: int):
    """Bounds of partition q of the birth box U(2 p_min, 2 p_max): slabs along x."""
    lo = np.asarray(params.birth_min, float).copy()
    hi = np.asarray(params.birth_max, float).copy()
    width = (hi[0] - lo[0]) / Q
    lo[0] = params.birth_min[0] + q * width
    hi[0] = lo[0] + width
    return lo, hi


def mt_mean(pred) -> np.ndarray:
    """x_hat = sum_p w_beta^p x^p of the predicted MT particles."""
    w = pred.w_beta / np.sum(pred.w_beta)
    return pred.x.astype(np.float64) @ w


def legacy_means(pred, S_legacy: int) -> np.ndarray:
    """Position estimate of each legacy PF from its prediction message."""
    out = np.zeros((S_legacy, 3))
    for s in range(S_legacy):
        w = pred.w_alpha[s]
        if not np.sum(w) > 0:
            w = np.ones_like(w)   # a PF without existence mass: plain particle mean
        out[s] = pred.phi[s, :3].astype(np.float64) @ w / np.sum(w)
    return out


def residual(geom, z: np.ndarray, x_hat: np.ndarray, pf_pos: np.ndarray) -> np.ndarray:
    """z~_j = z_j - Psi_j Psi_j^+ z_j for every PA (z: (J, Nz) complex)."""
    out = np.empty_like(z, dtype=np.complex128)
    for j in range(geom.J):
        cols = [geometry.steering(geom, j, x_hat[None, :3], pf_pos[s][None, :], los=(s == 0))[0]
                for s in range(pf_pos.shape[0])]
        Psi = np.stack(cols, axis=1)
        c, *_ = np.linalg.lstsq(Psi, z[j].astype(np.complex128), rcond=None)
        out[j] = z[j] - Psi @ c
    return out


def candidates(params, Q: int, q: int, N_g: int, n: int, seed: int) -> np.ndarray:
    lo, hi = partition_bounds(params, Q, q)
    u = np.stack(rng.uniforms24(seed, np.arange(N_g, dtype=np.uint64), n, rng.BIRTH_CAND, q, 3), axis=1)
    return lo[None, :] + (hi - lo)[None, :] * u


def bartlett(geom, z_res: np.ndarray, x_hat: np.ndarray, cand: np.ndarray) -> np.ndarray:
    """c_i = | sum_j (1/Nz) z~_j^H psi_j(x_hat, p_i) |^2."""
    acc = np.zeros(cand.shape[0], np.complex128)
    xb = np.broadcast_to(x_hat[:3], cand.shape)
    for j in range(geom.J):
        psi = geometry.steering(geom, j, xb, cand, los=False)      # (N_g, Nz)
        acc += psi @ np.conj(z_res[j]) / geom.Nz
    return np.abs(acc) ** 2


def moments(cand: np.ndarray, costs: np.ndarray):
    """(i*, mu, C): first maximum and the weighted second moment about it."""
    i_star = int(np.argmax(costs))
    mu = cand[i_star].copy()
    w = costs / np.sum(costs)
    d = cand - mu[None, :]
    C = (d * w[:, None]).T @ d
    return i_star, mu, C


def propose(pred, params, geom, z: np.ndarray, S_legacy: int, N_g: int, seed: int):
    """The proposal of every new PF of a prediction (slots S_legacy .. pred.S - 1)."""
    x_hat = mt_mean(pred)
    pf_pos = legacy_means(pred, S_legacy)
    z_res = residual(geom, z, x_hat, pf_pos)
    out = []
    for s in range(S_legacy, pred.S):
        q = s - S_legacy
        cand = candidates(params, params.Q, q, N_g, pred.n, seed)
        c = bartlett(geom, z_res, x_hat, cand)
        if not (np.sum(c) > 0 and np.isfinite(np.sum(c))):
            # a residual with no power left: the PF keeps its draws from the birth density
            out.append(Proposal(q=q, slot=s, costs=c, cand=cand, i_star=-1, mu=None, C=None, L=None))
            continue
        i_star, mu, C = moments(cand, c)
        out.append(Proposal(q=q, slot=s, costs=c, cand=cand, i_star=i_star, mu=mu, C=C,
                            L=resample.cholesky_zeroing(C)))
    return out


def apply(pred, params, geom, z: np.ndarray, S_legacy: int, N_g: int, seed: int):
    """The prediction with every new PF's particles and weights drawn from its proposal."""
    props = propose(pred, params, geom, z, S_legacy, N_g, seed)
    P = pred.x.shape[1]
    idx = np.arange(P, dtype=np.uint64)
    phi = pred.phi.astype(np.float64).copy()
    w_alpha = pred.w_alpha.copy()
    pB = model.birth_probability(params.mu_B, params.Q)
    for pr in props:
        if pr.mu is None:
            continue
        s = pr.slot
        g = np.stack(rng.normals(seed, idx, pred.n, rng.BIRTH_PROP, s, 3), axis=0)   # (3, P)
        pos = pr.mu[:, None] + pr.L @ g
        lo, hi = partition_bounds(params, params.Q, pr.q)
        inside = np.all((pos >= lo[:, None]) & (pos <= hi[:, None]), axis=0)
        active = np.diag(pr.L) > 0
        m2 = np.sum(g[active] ** 2, axis=0)
        wt = np.where(inside, np.exp(0.5 * m2), 0.0)
        tot = np.sum(wt)
        if not tot > 0:
            continue            # no draw inside the partition: the PF keeps its birth-density draws
        w_alpha[s] = pB * wt / tot
        phi[s, :3] = pos
    return dataclasses.replace(pred, phi=phi.astype(np.float32), w_alpha=w_alpha), props
