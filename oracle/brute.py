"""Exact complex-Gaussian mixture moments by enumeration (oracle; test infrastructure only).

For one paired particle (P = 1) the exact messages of eq. (Miota-exact) ..
(Momega-exact) are finite mixtures over the 2^(2 S~) existence configurations
(r_s, r_s^(j)).  Given the configuration, z ~ CN(sum_s b_s rho-mean, eta I +
sum_s b_s gamma_s psi_s psi_s^H) with b_s = r_s r_s^(j) (eq. likelihood-Type-II),
and the prediction messages give the configuration probabilities:
P(r_s = 1) = W_s (= sum_p w_alpha,s), P(r_s^(j) = 1) = zeta_s^(j)(1).
This module enumerates the mixture and returns its exact first two moments
(mean and covariance), which Proposition 1 matches; used by pin P1.
"""
from __future__ import annotations

import itertools

import numpy as np


def mixture_moments(psi, gamma, mu, W, zeta, eta_mean, fixed=None):
    """Exact mean and covariance of z under the existence mixture.

    psi (S, Nz) steering vectors of the paired particle; gamma, mu, W, zeta (S,);
    eta_mean = E[eta] under the noise message.  `fixed` = dict {("r", s): v} or
    {("rj", s): v} conditions the named existence variable on value v (the
    variable the message is sent to)."""
    S, Nz = psi.shape
    fixed = fixed or {}
    mean = np.zeros(Nz, complex)
    second = np.zeros((Nz, Nz), complex)
    total = 0.0
    for bits in itertools.product([0, 1], repeat=2 * S):
        r = bits[:S]
        rj = bits[S:]
        prob = 1.0
        ok = True
        for s in range(S):
            if ("r", s) in fixed:
                if r[s] != fixed[("r", s)]:
                    ok = False
                    break
            else:
                prob *= W[s] if r[s] else (1.0 - W[s])
            if ("rj", s) in fixed:
                if rj[s] != fixed[("rj", s)]:
                    ok = False
                    break
            else:
                prob *= zeta[s] if rj[s] else (1.0 - zeta[s])
        if not ok or prob == 0.0:
            continue
        b = np.array([r[s] * rj[s] for s in range(S)], float)
        m = (b * mu) @ psi
        C = eta_mean * np.eye(Nz) + np.einsum("s,sk,sl->kl", b * gamma, psi, psi.conj())
        mean += prob * m
        second += prob * (C + np.outer(m, m.conj()))
        total += prob
    mean /= total
    second /= total
    return mean, second - np.outer(mean, mean.conj())
