"""Update messages through the low-rank identities of Supplementary Sec. S-V
(oracle, FP64; test infrastructure only).

The same messages as ``messages_dense`` evaluated the way S-V writes them:
  * A^-1 by the matrix inversion lemma,  a^H A^-1 b = a^H b/eta - (M^H a)^H (I + M^H M/eta)^-1 (M^H b)/eta^2
    (S-V eq. Maha-expression), det A = eta^Nz det(I + M^H M/eta) (determinant lemma)
  * kappa~ and omega~: rank-one update of A_s by q psi psi^H (resp. m^w m^w^H):
    log CN = q|psi^H A^-1 e|^2/(1 + q psi^H A^-1 psi) - e^H A^-1 e - log(1 + q psi^H A^-1 psi)
             - log det A - Nz log pi      (S-V, PF and PR state update messages)
  * iota~ and nu~:  e^H A^-1 e = |e|^2/eta - |(I + M^H M/eta)^{-1/2} M^H e|^2/eta^2,
    log CN = -e^H A^-1 e - Nz log(pi eta) - log det(I + M^H M/eta)   (S-V, MT and noise messages)
The "-1/2" power is taken through the Cholesky factor L L^H = I + M^H M/eta.
The terms S-V drops because they cancel in a normalisation (det A^kappa,
pi^Nz) are kept here so that every value equals its dense counterpart (pin P2).
"""
from __future__ import annotations

import numpy as np

from .messages_dense import Messages, all_steering, message_table, mean_others


def _inner(a, b):
    """a^H b along the last axis."""
    return np.sum(a.conj() * b, axis=-1)


class WoodburyA:
    """A = eta I + M M^H with M = [cols] (Nz x K); evaluates a^H A^-1 b and log det A."""

    def __init__(self, eta: float, cols: np.ndarray):
        self.eta = eta
        self.M = cols.T                                  # (Nz, K)
        K = self.M.shape[1]
        self.Nz = self.M.shape[0]
        G = self.M.conj().T @ self.M
        self.Kinv = np.linalg.inv(np.eye(K) + G / eta) if K else np.zeros((0, 0))
        sign, ld = np.linalg.slogdet(np.eye(K) + G / eta) if K else (1.0, 0.0)
        self.logdet = self.Nz * np.log(eta) + float(np.real(ld))

    def form(self, a, b):
        """a^H A^-1 b for batches a (..., Nz), b (..., Nz)."""
        t = _inner(a, b) / self.eta
        if self.M.shape[1] == 0:
            return t
        Ma = a @ self.M.conj()                            # (..., K) = M^H a
        Mb = b @ self.M.conj()
        return t - np.einsum("...k,kl,...l->...", Ma.conj(), self.Kinv, Mb) / self.eta ** 2


def _rank1_logcn(Ainv: WoodburyA, e, v, q):
    """log CN(z; ., A + q v v^H) with e = z - mean: matrix inversion + determinant lemma."""
    Nz = e.shape[-1]
    vAe = Ainv.form(v, e)
    vAv = np.real(Ainv.form(v, v))
    eAe = np.real(Ainv.form(e, e))
    den = 1.0 + q * vAv
    return q * np.abs(vAe) ** 2 / den - eAe - np.log(den) - Ainv.logdet - Nz * np.log(np.pi)


def _lowrank_logcn(eta, Mcols, e):
    """log CN(z; ., eta I + M M^H) through the Cholesky factor of I + M^H M/eta.
    Mcols (..., K, Nz), e (..., Nz), eta scalar or (...)."""
    Nz = e.shape[-1]
    K = Mcols.shape[-2]
    eta = np.asarray(eta, np.float64)
    M = np.swapaxes(Mcols, -1, -2)                                   # (..., Nz, K)
    G = np.swapaxes(M.conj(), -1, -2) @ M
    Gm = np.eye(K) + G / eta[..., None, None]
    L = np.linalg.cholesky(Gm)
    Me = np.einsum("...kc,...k->...c", M.conj(), e)                   # M^H e
    y = np.linalg.solve(L, Me[..., None])[..., 0]
    quad = np.sum(np.abs(e) ** 2, axis=-1) / eta - np.sum(np.abs(y) ** 2, axis=-1) / eta ** 2
    logdet = 2.0 * np.sum(np.log(np.real(np.diagonal(L, axis1=-2, axis2=-1))), axis=-1)
    return -quad - Nz * np.log(np.pi * eta) - logdet


def update_messages(pred, params, geom, z, psi=None) -> Messages:
    if psi is None:
        psi = all_steering(pred, geom)
    return messages_from_table(pred, message_table(pred, params, psi), geom, z, psi)


def messages_from_table(pred, tab, geom, z, psi=None) -> Messages:
    """Every update message of the particles in `pred` from a given message table (for
    a subset of the particles the table was summed over)."""
    if psi is None:
        psi = all_steering(pred, geom)
    S, J, P = pred.S, geom.J, pred.x.shape[1]
    gam = pred.phi[:, 3].astype(np.float64)
    mu = pred.phi[:, 4].astype(np.float64) + 1j * pred.phi[:, 5].astype(np.float64)
    li = np.empty((J, P)); ln = np.empty((J, P))
    k1 = np.empty((S, J, P)); k0 = np.empty((S, J))
    o1 = np.empty((S, J)); o0 = np.empty((S, J))
    for j in range(J):
        # MT message: particle-dependent columns sqrt(pi (gamma + |mu|^2 pddot)) psi_s
        pi = tab.pi[:, j]
        d = np.sqrt(pi[:, None] * (gam + np.abs(mu) ** 2 * (1.0 - pi)[:, None]))   # (S, P)
        cols = np.transpose(d[:, :, None] * psi[:, j], (1, 0, 2))                    # (P, S, Nz)
        mean = np.einsum("s,sp,spk->pk", pi, mu, psi[:, j])
        li[j] = _lowrank_logcn(tab.eta_bar[j], cols, z[j][None] - mean)
        # noise message: columns m_s, particle-dependent eta
        e = z[j] - tab.mu3[:, j].sum(axis=0)
        ln[j] = _lowrank_logcn(pred.eta[j].astype(np.float64), np.broadcast_to(tab.m[:, j], (P, S, geom.Nz)),
                               np.broadcast_to(e, (P, geom.Nz)))
        for s in range(S):
            A = WoodburyA(tab.eta_bar[j], np.delete(tab.m[:, j], s, axis=0))
            mo = mean_others(tab, s, j)
            zeta = pred.zeta[s, j]
            q = (gam[s] + np.abs(mu[s]) ** 2 * (1.0 - zeta)) * zeta
            e1 = z[j][None] - mo[None] - zeta * mu[s][:, None] * psi[s, j]
            k1[s, j] = _rank1_logcn(A, e1, psi[s, j], q)
            e0 = z[j] - mo
            k0[s, j] = -np.real(A.form(e0, e0)) - A.logdet - geom.Nz * np.log(np.pi)
            o1[s, j] = _rank1_logcn(A, e0 - tab.mu4[s, j], tab.mw[s, j], 1.0)
            o0[s, j] = k0[s, j]
    return Messages(table=tab, log_iota=li, log_nu=ln, log_kappa1=k1, log_kappa0=k0,
                    log_omega1=o1, log_omega0=o0)
