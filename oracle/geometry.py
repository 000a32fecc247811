"""Geometric model and array response (oracle, FP64; test infrastructure only).

Follows Sec. II-A (eq. rangep, house, posPA-SB), Sec. II-B (eq.
array-response, unit-modulus-array-response) and Supplementary Sec. S-I/S-II
(template layout eq. Ptemplate, VA layout eq. VA-layout-SB, planar-wavefront
response).  The steering vector is evaluated element by element from the
virtual-anchor array layout in global coordinates, not through the Kronecker
factorisation; tests pin the two against each other (Sec. S-II shows they
are equal).

Pins: Householder orthogonal and involutive; VA = mirror image of the PA
across the plane through p_sfv/2 with normal p_sfv/|p_sfv| (Sec. S-I);
element-wise response == Kronecker response; LoS local vector = R^T (p - p_pa).
"""
from __future__ import annotations

import numpy as np


def householder(p_sfv: np.ndarray) -> np.ndarray:
    """H = I - 2 p p^T / |p|^2 (eq. house).  p_sfv: (..., 3) -> (..., 3, 3)."""
    p = np.asarray(p_sfv, np.float64)
    nn = np.sum(p * p, axis=-1)[..., None, None]
    return np.eye(3) - 2.0 * p[..., :, None] * p[..., None, :] / nn


def virtual_anchor(p_pa: np.ndarray, p_sfv: np.ndarray) -> np.ndarray:
    """p_va = p_pa - (2 p_pa^T p_sfv / |p_sfv|^2 - 1) p_sfv (eq. posPA-SB)."""
    p = np.asarray(p_sfv, np.float64)
    a = np.asarray(p_pa, np.float64)
    nn = np.sum(p * p, axis=-1)
    coef = 2.0 * np.sum(a * p, axis=-1) / nn - 1.0
    return a - coef[..., None] * p


def template_layout(p_y: np.ndarray, p_z: np.ndarray) -> np.ndarray:
    """P_template = [0; p_y^T kron 1; 1 kron p_z^T]  (3 x My*Mz), eq. Ptemplate."""
    My, Mz = len(p_y), len(p_z)
    P = np.zeros((3, My * Mz))
    P[1] = np.kron(np.asarray(p_y, float), np.ones(Mz))
    P[2] = np.kron(np.ones(My), np.asarray(p_z, float))
    return P


def local_vector(p: np.ndarray, p_sfv: np.ndarray, p_pa: np.ndarray, R: np.ndarray, los: bool) -> np.ndarray:
    """r' = R^{-1} H (p - p_va)  (eq. rangep); LoS: R^{-1} (p - p_pa).  p: (..., 3)."""
    p = np.asarray(p, np.float64)
    if los:
        r = p - p_pa
        return r @ R  # R^T r for row vectors
    H = householder(p_sfv)
    r = p - virtual_anchor(p_pa, p_sfv)
    rt = np.einsum("...ij,...j->...i", H, r)
    return rt @ R


def steering(geom, j: int, p: np.ndarray, p_sfv: np.ndarray, los: bool) -> np.ndarray:
    """Steering vector psi^(j)(p, p_sfv) in C^Nz for a batch of points.

    p, p_sfv: (..., 3).  Element (f, m), flat index f*(My*Mz) + m, equals
        lambda/(4 pi |r|) * exp(-j 2 pi (fc + f_f) tau + j 2 pi/lambda (H R P_t[:, m])^T u)
    with r = p - p_va (VA to MT, global), u = r/|r|, tau = |r|/c: the VA array
    layout (eq. VA-layout-SB) under the per-PA planar wavefront of Sec. S-II with
    the spatial term taken at fc and a unit spectrum S(f) = 1 (eq. array-response)."""
    p = np.asarray(p, np.float64)
    p_pa = np.asarray(geom.p_pa[j], np.float64)
    R = np.asarray(geom.R_pa[j], np.float64)
    lam = geom.c / geom.fc
    Pt = template_layout(geom.p_y, geom.p_z)
    if los:
        va = np.broadcast_to(p_pa, p.shape)
        HRP = np.broadcast_to(R @ Pt, p.shape[:-1] + Pt.shape)
    else:
        va = virtual_anchor(p_pa, p_sfv)
        H = householder(p_sfv)
        HRP = np.einsum("...ik,kl->...il", H, R @ Pt)
    r = p - va
    d = np.linalg.norm(r, axis=-1)
    u = r / d[..., None]
    tau = d / geom.c
    spatial = (2.0 * np.pi / lam) * np.einsum("...km,...k->...m", HRP, u)   # (..., Nm)
    f = geom.freqs()
    delay = -2.0 * np.pi * (geom.fc + f)[None, :] * tau.reshape(-1, 1)       # (B, Nf)
    delay = delay.reshape(tau.shape + (len(f),))
    phase = delay[..., :, None] + spatial[..., None, :]                      # (..., Nf, Nm)
    amp = lam / (4.0 * np.pi * d)
    psi = amp[..., None, None] * np.exp(1j * phase)
    return psi.reshape(p.shape[:-1] + (geom.Nz,))


def steering_kronecker(geom, j: int, p, p_sfv, los: bool) -> np.ndarray:
    """The same vector through eq. (unit-modulus-array-response):
    (lambda/(4 pi |r'|)) (b(tau) kron a_y kron a_z) exp(-j 2 pi fc |r'|/c),
    b = exp(-j 2 pi f tau), a_y = exp(j 2pi/lambda p_y sin(theta) sin(phi)),
    a_z = exp(j 2pi/lambda p_z cos(theta)), theta = arccos(r'_z/|r'|), phi = atan2(r'_y, r'_x).
    Used only to pin `steering` (Sec. S-II)."""
    rp = local_vector(p, p_sfv, geom.p_pa[j], geom.R_pa[j], los)
    d = np.linalg.norm(rp, axis=-1)
    lam = geom.c / geom.fc
    theta = np.arccos(rp[..., 2] / d)
    phi = np.arctan2(rp[..., 1], rp[..., 0])
    tau = d / geom.c
    f = geom.freqs()
    b = np.exp(-2j * np.pi * f * tau[..., None])
    ay = np.exp(2j * np.pi / lam * np.asarray(geom.p_y) * (np.sin(theta) * np.sin(phi))[..., None])
    az = np.exp(2j * np.pi / lam * np.asarray(geom.p_z) * np.cos(theta)[..., None])
    a = (ay[..., :, None] * az[..., None, :]).reshape(ay.shape[:-1] + (-1,))
    psi_t = (b[..., :, None] * a[..., None, :]).reshape(b.shape[:-1] + (-1,))
    psi_t = psi_t * np.exp(-2j * np.pi * geom.fc * d / geom.c)[..., None]
    return (lam / (4.0 * np.pi * d))[..., None] * psi_t


def steering_spherical(geom, j: int, p, p_sfv, los: bool) -> np.ndarray:
    """Spherical-wavefront response (Sec. S-II, eq. spherical-wavefront-response):
    per-element distances |p - P_k[:, m]| to the (virtual) array elements; the
    carrier-phase/delay term exp(-j 2 pi f_pb d_m / c), amplitude at the centre.
    Used only as a far-field pin of `steering`."""
    p = np.asarray(p, np.float64)
    p_pa = np.asarray(geom.p_pa[j], np.float64)
    R = np.asarray(geom.R_pa[j], np.float64)
    Pt = template_layout(geom.p_y, geom.p_z)
    if los:
        va = p_pa
        E = va[:, None] + R @ Pt
    else:
        va = virtual_anchor(p_pa, p_sfv)
        E = va[:, None] + householder(p_sfv) @ R @ Pt
    dm = np.linalg.norm(p[:, None] - E, axis=0)                 # (Nm,)
    d0 = np.linalg.norm(p - va)
    lam = geom.c / geom.fc
    f = geom.freqs()
    ph = -2.0 * np.pi * (geom.fc + f)[:, None] * dm[None, :] / geom.c
    return (lam / (4.0 * np.pi * d0)) * np.exp(1j * ph).reshape(-1)
