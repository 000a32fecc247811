"""Synthetic observations from the generative signal model (oracle, FP64).

Test infrastructure only.  z_n^(j) = sum_k rho_k,n^(j) psi^(j)(p_n, p_sfv,k) + n_n^(j)
(eq. observation-generative), invisible paths have rho = 0 (Sec. II-B); the
noise is CN(0, eta I) with eta fixed so that SNR = P^ch_1/eta, where
P^ch_n = (1/(Nz J)) sum_j |sum_k rho_k,n^(j) psi_k,n^(j)|^2 (Sec. V-A, "System
Parameters").  Spurious one-step components ("clutter") are not in the paper;
they are added, when a scenario asks for them, as extra terms of the same form
and are not counted in P^ch.

Noise draws: Philox block (c0 = element index k, c1 = n, purpose SYNTH_NOISE,
sub = j, c3 = 0); x0, x1 -> FP64 Box-Muller pair -> sqrt(eta/2) (g0 + i g1).
"""
from __future__ import annotations

import numpy as np

from . import geometry, rng


def clean_signal(scn, n: int) -> np.ndarray:
    """sum_k rho psi for step n (true components only): (J, Nz) complex."""
    g = scn.geom
    out = np.zeros((g.J, g.Nz), complex)
    p = scn.x_true[n, :3]
    K = scn.sfv_true.shape[0]
    for j in range(g.J):
        for k in range(K + 1):
            if not scn.visible[n, j, k]:
                continue
            rho = scn.rho_abs[k] * np.exp(1j * scn.rho_phase[n, j, k])
            sfv = scn.sfv_true[k - 1] if k > 0 else np.zeros(3)
            out[j] += rho * geometry.steering(g, j, p[None], sfv[None], los=(k == 0))[0]
    return out


def noise_variance(scn) -> float:
    """eta = P^ch_1 / 10^(SNR/10) with the sum-channel power at n = 1."""
    sig = clean_signal(scn, 1)
    pch = np.sum(np.abs(sig) ** 2) / (scn.geom.Nz * scn.geom.J)
    return float(pch / 10.0 ** (scn.snr_db / 10.0))


def observe(scn, n: int, eta: float, seed: int) -> np.ndarray:
    """z_n: (J, Nz) complex128 (signal + clutter + noise)."""
    g = scn.geom
    z = clean_signal(scn, n)
    p = scn.x_true[n, :3]
    for c in range(scn.clutter_sfv[n].shape[0]):
        for j in range(g.J):
            z[j] += scn.clutter_rho[n][c, j] * geometry.steering(g, j, p[None], scn.clutter_sfv[n][c][None], los=False)[0]
    k = np.arange(g.Nz, dtype=np.uint64)
    for j in range(g.J):
        x = rng.draw(seed, k, n, rng.SYNTH_NOISE, j, 0)
        g0, g1 = rng.box_muller(rng.u32d(x[0]), rng.u32d(x[1]))
        z[j] += np.sqrt(eta / 2.0) * (g0 + 1j * g1)
    return z
