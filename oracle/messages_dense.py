"""Update messages by their plain definition (oracle, FP64; test infrastructure only).

Every approximate message is a complex Gaussian CN(z; mean, C) (Sec. IV-C,
Proposition 1).  Here mean and C are formed explicitly in C^Nz and C^{Nz x Nz}
from the particle representations of Supplementary Sec. S-V, and
    log CN(z; mu, C) = -Nz log(pi) - log det C - (z - mu)^H C^{-1} (z - mu)
is evaluated with a dense Cholesky factorisation.  No low-rank identity is
used; ``messages_woodbury`` is the separate S-V rendering pinned against this.

Message table (Sec. S-V; Proposition 1 terms mu^(3), mu^(4)), with
W_s = sum_p w_alpha,s^p, pi_s^(j) = zeta_s^(j)(1) W_s,
pdot_s^(j) = 1 - zeta_s^(j)(1), pdot_s = 1 - W_s, pddot_s^(j) = 1 - pi_s^(j):
    m_s^(j)      = c_m  sum_p w_beta^p sqrt(gamma_s^p + |mu_s^p|^2 pddot_s^(j)) psi_s^(j,p)
    m_s^w(j)     = c_w  sum_p w_beta^p sqrt(gamma_s^p + |mu_s^p|^2 pdot_s) psi_s^(j,p)
    mu3_s^(j)    = zeta W_s sum_p w_beta^p mu_s^p psi_s^(j,p),   mu4_s^(j) = mu3_s^(j)/zeta
with c_m = W_s zeta, c_w = W_s as printed in S-V (reading R2, mvec_scaling = 0)
or c_m = sqrt(W_s zeta), c_w = sqrt(W_s) (mvec_scaling = 1).
Particle pairing (reading R1, parity unpinned as a modelling choice): the
MT particle p and PF particle p share one index, psi_s^(j,p) = psi^(j)(x^p, phi_s^p).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import geometry


@dataclasses.dataclass
class Table:
    W: np.ndarray        # (S,)     sum_p w_alpha
    pi: np.ndarray       # (S, J)
    m: np.ndarray        # (S, J, Nz)
    mw: np.ndarray       # (S, J, Nz)
    mu3: np.ndarray      # (S, J, Nz)
    mu4: np.ndarray      # (S, J, Nz)
    eta_bar: np.ndarray  # (J,)     sum_p w_xi eta


def all_steering(pred, geom) -> np.ndarray:
    """psi_s^(j,p) for every (s, j, p): (S, J, P, Nz) complex128."""
    S, P = pred.S, pred.x.shape[1]
    pos = pred.x[:3].astype(np.float64).T                       # (P, 3)
    out = np.empty((S, geom.J, P, geom.Nz), np.complex128)
    for s in range(S):
        sfv = pred.phi[s, :3].astype(np.float64).T
        for j in range(geom.J):
            out[s, j] = geometry.steering(geom, j, pos, sfv, los=(s == 0))
    return out


def message_table(pred, params, psi) -> Table:
    S, J = pred.S, pred.zeta.shape[1]
    W = pred.w_alpha.sum(axis=1)
    zeta = pred.zeta
    pi = zeta * W[:, None]
    gam = pred.phi[:, 3].astype(np.float64)
    mu = pred.phi[:, 4].astype(np.float64) + 1j * pred.phi[:, 5].astype(np.float64)
    wb = pred.w_beta
    Nz = psi.shape[-1]
    m = np.zeros((S, J, Nz), complex)
    mw = np.zeros((S, J, Nz), complex)
    mu3 = np.zeros((S, J, Nz), complex)
    mu4 = np.zeros((S, J, Nz), complex)
    for s in range(S):
        for j in range(J):
            pdd = 1.0 - pi[s, j]
            pd_s = 1.0 - W[s]
            if params.mvec_scaling == 0:
                cm, cw = W[s] * zeta[s, j], W[s]
            else:
                cm, cw = np.sqrt(W[s] * zeta[s, j]), np.sqrt(W[s])
            a = wb * np.sqrt(gam[s] + np.abs(mu[s]) ** 2 * pdd)
            b = wb * np.sqrt(gam[s] + np.abs(mu[s]) ** 2 * pd_s)
            c = wb * mu[s]
            m[s, j] = cm * (a @ psi[s, j])
            mw[s, j] = cw * (b @ psi[s, j])
            mu4[s, j] = W[s] * (c @ psi[s, j])
            mu3[s, j] = zeta[s, j] * mu4[s, j]
    eta_bar = np.sum(pred.w_xi * pred.eta.astype(np.float64), axis=1)
    return Table(W=W, pi=pi, m=m, mw=mw, mu3=mu3, mu4=mu4, eta_bar=eta_bar)


def table_sums(x, phi, w_beta, pi, W, geom):
    """The particle sums of `message_table` over one set of particles (S-V):
    sum_p w_beta^p sqrt(gamma_s^p + |mu_s^p|^2 pddot_s^(j)) psi_s^(j,p),
    sum_p w_beta^p sqrt(gamma_s^p + |mu_s^p|^2 pdot_s) psi_s^(j,p) and
    sum_p w_beta^p mu_s^p psi_s^(j,p), each (S, J, Nz).  pi and W are those of the
    whole particle set.  Sums over disjoint particle sets add up to the full sums."""
    S, J = phi.shape[0], pi.shape[1]
    pos = x[:3].astype(np.float64).T
    gam = phi[:, 3].astype(np.float64)
    mu = phi[:, 4].astype(np.float64) + 1j * phi[:, 5].astype(np.float64)
    sa = np.zeros((S, J, geom.Nz), complex)
    sb = np.zeros((S, J, geom.Nz), complex)
    sc = np.zeros((S, J, geom.Nz), complex)
    for s in range(S):
        sfv = phi[s, :3].astype(np.float64).T
        for j in range(J):
            ps = geometry.steering(geom, j, pos, sfv, los=(s == 0))
            sa[s, j] = (w_beta * np.sqrt(gam[s] + np.abs(mu[s]) ** 2 * (1.0 - pi[s, j]))) @ ps
            sb[s, j] = (w_beta * np.sqrt(gam[s] + np.abs(mu[s]) ** 2 * (1.0 - W[s]))) @ ps
            sc[s, j] = (w_beta * mu[s]) @ ps
    return sa, sb, sc


def _table_sums_task(args):
    return table_sums(*args)


def message_table_streamed(pred, params, geom, chunk: int = 4096, pool=None) -> Table:
    """`message_table` for particle sets too large to hold every steering vector at
    once: the same sums, taken over particle chunks (optionally in a process pool)
    and added, then scaled as in `message_table`."""
    S, J = pred.S, pred.zeta.shape[1]
    P = pred.x.shape[1]
    W = pred.w_alpha.sum(axis=1)
    zeta = pred.zeta
    pi = zeta * W[:, None]
    tasks = [(pred.x[:, sl], pred.phi[:, :, sl], pred.w_beta[sl], pi, W, geom) for sl in _chunks(P, chunk)]
    parts = (pool.map(_table_sums_task, tasks) if pool is not None else [_table_sums_task(t) for t in tasks])
    sa = sum(p[0] for p in parts)
    sb = sum(p[1] for p in parts)
    sc = sum(p[2] for p in parts)
    if params.mvec_scaling == 0:
        cm, cw = W[:, None] * zeta, np.broadcast_to(W[:, None], (S, J))
    else:
        cm, cw = np.sqrt(W[:, None] * zeta), np.broadcast_to(np.sqrt(W)[:, None], (S, J))
    m = cm[:, :, None] * sa
    mw = cw[:, :, None] * sb
    mu4 = W[:, None, None] * sc
    mu3 = zeta[:, :, None] * mu4
    eta_bar = np.sum(pred.w_xi * pred.eta.astype(np.float64), axis=1)
    return Table(W=W, pi=pi, m=m, mw=mw, mu3=mu3, mu4=mu4, eta_bar=eta_bar)


def log_cn(z: np.ndarray, mean: np.ndarray, C: np.ndarray) -> np.ndarray:
    """log CN(z; mean, C) for batches: mean (..., Nz), C (..., Nz, Nz)."""
    Nz = z.shape[-1]
    L = np.linalg.cholesky(C)
    e = (z - mean)[..., None]
    y = np.linalg.solve(L, e)[..., 0]
    quad = np.sum(np.abs(y) ** 2, axis=-1)
    logdet = 2.0 * np.sum(np.log(np.real(np.diagonal(L, axis1=-2, axis2=-1))), axis=-1)
    return -Nz * np.log(np.pi) - logdet - quad


def _chunks(P, size):
    for a in range(0, P, size):
        yield slice(a, min(P, a + size))


def iota_moments(pred, tab: Table, psi, j: int, sl=slice(None)):
    """Mean and covariance of iota~(x^p; z^(j)) for the particles in `sl` (S-V, MT message):
    mu^iota = sum_s pi_s mu_s^p psi_s, C^iota = eta_bar I + sum_s pi_s (gamma_s^p + |mu_s^p|^2 pddot_s) psi_s psi_s^H."""
    Nz = psi.shape[-1]
    gam = pred.phi[:, 3, sl].astype(np.float64)
    mu = pred.phi[:, 4, sl].astype(np.float64) + 1j * pred.phi[:, 5, sl].astype(np.float64)
    pi = tab.pi[:, j]
    Ps = psi[:, j, sl]                                                 # (S, p, Nz)
    mean = np.einsum("s,sp,spk->pk", pi, mu, Ps)
    d2 = pi[:, None] * (gam + np.abs(mu) ** 2 * (1.0 - pi)[:, None])  # (S, p)
    C = tab.eta_bar[j] * np.eye(Nz)[None] + np.einsum("sp,spk,spl->pkl", d2, Ps, Ps.conj())
    return mean, C


def log_iota(pred, tab: Table, psi, z, j: int, chunk: int = 64) -> np.ndarray:
    """log iota~(x^p; z^(j)) = log CN(z; mu^iota(x^p), C^iota(x^p))."""
    P = pred.x.shape[1]
    out = np.empty(P)
    for sl in _chunks(P, chunk):
        mean, C = iota_moments(pred, tab, psi, j, sl)
        out[sl] = log_cn(z[j][None], mean, C)
    return out


def nu_moments(tab: Table, j: int, eta):
    """Mean and covariance of nu~(eta; z^(j)) (S-V): sum_s mu3_s and eta I + sum_s m_s m_s^H."""
    Nz = tab.m.shape[-1]
    mean = tab.mu3[:, j].sum(axis=0)
    MM = np.einsum("sk,sl->kl", tab.m[:, j], tab.m[:, j].conj())
    eta = np.atleast_1d(np.asarray(eta, np.float64))
    return mean, eta[:, None, None] * np.eye(Nz)[None] + MM[None]


def log_nu(pred, tab: Table, z, j: int, chunk: int = 256) -> np.ndarray:
    """log nu~(eta^(j,p); z^(j)) = log CN(z; mu^nu, C^nu(eta^(j,p)))."""
    P = pred.x.shape[1]
    eta = pred.eta[j].astype(np.float64)
    out = np.empty(P)
    for sl in _chunks(P, chunk):
        mean, C = nu_moments(tab, j, eta[sl])
        out[sl] = log_cn(z[j][None], mean[None], C)
    return out


def A_kappa(tab: Table, s: int, j: int) -> np.ndarray:
    """A_s^kappa(j) = eta_bar I + M_{-s} M_{-s}^H with M_{-s} = [m_s']_{s' != s} (S-V)."""
    Nz = tab.m.shape[-1]
    others = [t for t in range(tab.m.shape[0]) if t != s]
    M = tab.m[others, j]                                               # (S-1, Nz)
    return tab.eta_bar[j] * np.eye(Nz) + M.T @ M.conj()


def mean_others(tab: Table, s: int, j: int) -> np.ndarray:
    """sum_{s' != s} mu3_s'^(j)."""
    return tab.mu3[:, j].sum(axis=0) - tab.mu3[s, j]


def kappa_moments(pred, tab: Table, psi, s: int, j: int, sl=slice(None)):
    """Mean and covariance of kappa~(phi_s^p, r = 1; z^(j)) (S-V, PF message):
    mean zeta mu^p psi_s + sum_{s'!=s} mu3_s', cov q psi psi^H + A_s,
    q = (gamma^p + |mu^p|^2 pdot^(j)) zeta.  Under r = 0: sum_{s'!=s} mu3_s' and A_s."""
    zeta = pred.zeta[s, j]
    A = A_kappa(tab, s, j)
    mo = mean_others(tab, s, j)
    gam = pred.phi[s, 3, sl].astype(np.float64)
    mu = pred.phi[s, 4, sl].astype(np.float64) + 1j * pred.phi[s, 5, sl].astype(np.float64)
    q = (gam + np.abs(mu) ** 2 * (1.0 - zeta)) * zeta
    Ps = psi[s, j, sl]
    mean = mo[None] + zeta * mu[:, None] * Ps
    C = A[None] + q[:, None, None] * Ps[:, :, None] * Ps[:, None, :].conj()
    return mean, C, mo, A


def log_kappa(pred, tab: Table, psi, z, s: int, j: int, chunk: int = 64):
    """log kappa~(phi_s^p, 1; z^(j)) per particle and log kappa~(., 0; z^(j))."""
    P = pred.x.shape[1]
    out = np.empty(P)
    for sl in _chunks(P, chunk):
        mean, C, mo, A = kappa_moments(pred, tab, psi, s, j, sl)
        out[sl] = log_cn(z[j][None], mean, C)
    mo = mean_others(tab, s, j)
    l0 = log_cn(z[j][None], mo[None], A_kappa(tab, s, j)[None])[0]
    return out, l0


def omega_moments(tab: Table, s: int, j: int):
    """Mean and covariance of omega~(r = 1; z^(j)) (S-V, PR message):
    mean mu4_s + sum_{s'!=s} mu3_s', cov m^w m^w^H + A_s (r = 0: sum_{s'!=s} mu3_s', A_s)."""
    A = A_kappa(tab, s, j)
    mo = mean_others(tab, s, j)
    mw = tab.mw[s, j]
    return mo + tab.mu4[s, j], A + np.outer(mw, mw.conj()), mo, A


def log_omega(tab: Table, z, s: int, j: int):
    """log omega~(1; z^(j)) and log omega~(0; z^(j))."""
    m1, C1, m0, C0 = omega_moments(tab, s, j)
    l1 = log_cn(z[j][None], m1[None], C1[None])[0]
    l0 = log_cn(z[j][None], m0[None], C0[None])[0]
    return l1, l0


@dataclasses.dataclass
class Messages:
    table: Table
    log_iota: np.ndarray      # (J, P)
    log_nu: np.ndarray        # (J, P)
    log_kappa1: np.ndarray    # (S, J, P)
    log_kappa0: np.ndarray    # (S, J)
    log_omega1: np.ndarray    # (S, J)
    log_omega0: np.ndarray    # (S, J)


def update_messages(pred, params, geom, z) -> Messages:
    """Phase (iii) of the schedule: every update message, computed once (Sec. IV)."""
    psi = all_steering(pred, geom)
    tab = message_table(pred, params, psi)
    S, J, P = pred.S, geom.J, pred.x.shape[1]
    li = np.stack([log_iota(pred, tab, psi, z, j) for j in range(J)])
    ln = np.stack([log_nu(pred, tab, z, j) for j in range(J)])
    k1 = np.empty((S, J, P)); k0 = np.empty((S, J))
    o1 = np.empty((S, J)); o0 = np.empty((S, J))
    for s in range(S):
        for j in range(J):
            k1[s, j], k0[s, j] = log_kappa(pred, tab, psi, z, s, j)
            o1[s, j], o0[s, j] = log_omega(tab, z, s, j)
    return Messages(table=tab, log_iota=li, log_nu=ln, log_kappa1=k1, log_kappa0=k0,
                    log_omega1=o1, log_omega0=o0)
