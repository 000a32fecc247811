"""Oracle of the posterior Cramer-Rao lower bounds (Sec. VI; Supplementary Sec. S-VII).

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the CPU legs of
bench.py; the product path never calls it.

Global parameters (Sec. VI): eta_g = [x (6: position, velocity), the K SFV positions
(3K), phases (noncoherent: one per component and PA, K~ J; coherent: one per component,
K~), moduli (K~ J), the common noise variance eta], K~ = K + 1 components with the LoS
first.  For the bound the amplitudes absorb the path loss and the carrier phase
(Sec. S-VII), so every component's array response is the unit-modulus
b(tau) kron a_y(theta, az) kron a_z(theta) at baseband frequencies.

  * local channel FIM per PA (Table S-I): J_ch = (2/eta) Re(D^H D) over the local
    parameters [elevations, azimuths, delays, phases, moduli] (5 K~) plus Nz / eta^2 for
    eta, D holding d mu / d parameter (rho~_k times the response derivative for the
    angles and the delay, j rho~_k a_k for the phase, e^{j phi_k} a_k for the modulus);
  * Jacobians local -> global (Sec. S-VII-B): the chain H_k R_j d(angle, delay, carrier
    phase)/d r' to the MT position, the derivative of the PA-to-virtual-MT vector w.r.t.
    the SFV (sfv_block: in full, see the reading there) to the SFV positions, selectors for
    the phases (per PA or common) and moduli; moduli carry no position information (the
    path-loss derivative is neglected, as in the paper);
  * classic snapshot FIM J_C = sum_j G_j J_ch^(j) G_j^T; its Bayesian version is the mean
    of J_C over realisations of the state (Monte Carlo, as in the paper);
  * recursion J_{n|n} = J_B,n + (F J_{n-1|n-1}^-1 F^T + Q)^-1 with F = blkdiag(F_a, I_3K,
    0), Q = blkdiag(Q_a, sigma_sfv^2 I, sigma_phi^2 I, sigma_a^2 I, sigma_eta^2), and
    PEB = sqrt(tr P[0:3, 0:3]), MEB_k = sqrt(tr P[SFV k]) with P = J_{n|n}^-1.
Reading: the paper starts the recursion from J_{1|0} given by fictional starting points
at n = 0; here J_{1|0} is supplied by the caller (e.g. the inverse of a full-rank prior
covariance).
"""
from __future__ import annotations

import numpy as np

from . import geometry, model


def dims(K: int, J: int, coherent: bool):
    """Sizes and offsets of the global parameter vector."""
    Kt = K + 1
    nph = Kt if coherent else Kt * J
    o_sfv = 6
    o_ph = o_sfv + 3 * K
    o_a = o_ph + nph
    o_eta = o_a + Kt * J
    return dict(Kt=Kt, nph=nph, o_sfv=o_sfv, o_ph=o_ph, o_a=o_a, o_eta=o_eta, dim=o_eta + 1)


def local_vector(geom, j, p, sfv, los):
    """r' = R_j^T H (p - p_va) (eq. rangep) and the Householder matrix of the component."""
    p = np.asarray(p, float)
    if los:
        return geometry.local_vector(p[None], p[None], geom.p_pa[j], geom.R_pa[j], True)[0], np.eye(3)
    return (geometry.local_vector(p[None], np.asarray(sfv, float)[None], geom.p_pa[j], geom.R_pa[j], False)[0],
            geometry.householder(np.asarray(sfv, float)))


def spherical(rp):
    d = np.linalg.norm(rp)
    return d, np.arccos(rp[2] / d), np.arctan2(rp[1], rp[0])


def response(geom, tau, th, az):
    """Unit-modulus b(tau) kron a_y(theta, az) kron a_z(theta) and its derivatives w.r.t.
    theta, az, tau (Sec. S-VII-A), flat index f*(My*Mz) + y*Mz + m."""
    lam = geom.c / geom.fc
    f = geom.freqs()
    py, pz = np.asarray(geom.p_y, float), np.asarray(geom.p_z, float)
    b = np.exp(-2j * np.pi * f * tau)
    ay = np.exp(2j * np.pi / lam * py * np.sin(th) * np.sin(az))
    az_ = np.exp(2j * np.pi / lam * pz * np.cos(th))
    db = -2j * np.pi * f * b
    day_th = 2j * np.pi / lam * np.cos(th) * np.sin(az) * py * ay
    day_az = 2j * np.pi / lam * np.sin(th) * np.cos(az) * py * ay
    daz_th = -2j * np.pi / lam * np.sin(th) * pz * az_
    kr = lambda u, v, w: np.kron(u, np.kron(v, w))
    a = kr(b, ay, az_)
    a_th = kr(b, day_th, az_) + kr(b, ay, daz_th)
    a_az = kr(b, day_az, az_)
    a_tau = kr(db, ay, az_)
    return a, a_th, a_az, a_tau


def local_fim(geom, j, p, sfvs, rho_t, eta):
    """J_ch of PA j (5 K~ + 1) and the local vectors of its components.  rho_t: the K~
    complex amplitudes rho~ (path loss and carrier phase included)."""
    Kt = len(rho_t)
    Nz = geom.Nz
    D = np.zeros((Nz, 5 * Kt), complex)
    rps, Hs = [], []
    for k in range(Kt):
        rp, H = local_vector(geom, j, p, None if k == 0 else sfvs[k - 1], k == 0)
        rps.append(rp); Hs.append(H)
        d, th, az = spherical(rp)
        a, a_th, a_az, a_tau = response(geom, d / geom.c, th, az)
        r = rho_t[k]
        D[:, k] = r * a_th
        D[:, Kt + k] = r * a_az
        D[:, 2 * Kt + k] = r * a_tau
        D[:, 3 * Kt + k] = 1j * r * a
        D[:, 4 * Kt + k] = np.exp(1j * np.angle(r)) * a
    Jc = np.zeros((5 * Kt + 1, 5 * Kt + 1))
    Jc[:5 * Kt, :5 * Kt] = 2.0 / eta * np.real(D.conj().T @ D)
    Jc[5 * Kt, 5 * Kt] = Nz / eta ** 2
    return Jc, rps, Hs


def d_spherical(rp, lam, c):
    """d(theta, az, tau, carrier phase)/d r' (3 x 4)."""
    x, y, z = rp
    n2 = x * x + y * y
    d = np.linalg.norm(rp)
    g_th = np.array([x * z, y * z, -n2]) / (d * d * np.sqrt(n2))
    g_az = np.array([-y, x, 0.0]) / n2
    g_tau = rp / (c * d)
    g_ph = -2.0 * np.pi * rp / (lam * d)
    return np.stack([g_th, g_az, g_tau, g_ph], axis=1)


def sfv_block(p, sfv, H):
    """d r_breve^T / d p_sfv (3 x 3, information convention): the vector from the PA to the
    virtual MT, r_breve = H(s) p + s - p_pa with H(s) = I - 2 s s^T / |s|^2, differentiated
    in full, I - 2 p s^T / |s|^2 - 2 (p . s) / |s|^2 H.  Reading: the mapping submatrices
    of Sec. S-VII-B chain d r / d p_sfv with a fixed H; the reflection's own dependence on
    the SFV is part of the observation model, and its Fisher information (the definition of
    the bound, eq. FIMch) needs it (finite differences of the mean confirm the full form)."""
    s = np.asarray(sfv, float)
    p = np.asarray(p, float)
    n2 = s @ s
    return np.eye(3) - 2.0 * np.outer(p, s) / n2 - 2.0 * (p @ s) / n2 * H


def jacobian(geom, j, K, coherent, p, sfvs, rps, Hs):
    """G_j = d eta_ch^T / d eta_g (dim_g x (5 K~ + 1)), Sec. S-VII-B; p: MT position."""
    dd = dims(K, geom.J, coherent)
    Kt = dd["Kt"]
    lam = geom.c / geom.fc
    R = np.asarray(geom.R_pa[j], float)
    G = np.zeros((dd["dim"], 5 * Kt + 1))
    for k in range(Kt):
        ds = d_spherical(rps[k], lam, geom.c)          # columns: theta, az, tau, carrier phase
        Rd = R @ ds                                      # d(.)/d r_breve
        B = sfv_block(p, sfvs[k - 1], Hs[k]) if k > 0 else None
        for q in range(4):
            col = q * Kt + k
            G[0:3, col] = Hs[k] @ Rd[:, q]               # MT position (velocity rows stay 0)
            if k > 0:
                o = dd["o_sfv"] + 3 * (k - 1)
                G[o:o + 3, col] = B @ Rd[:, q]           # SFV k
        ph = dd["o_ph"] + (k if coherent else j * Kt + k)
        G[ph, 3 * Kt + k] = 1.0                          # phase -> nuisance phase
        G[dd["o_a"] + j * Kt + k, 4 * Kt + k] = 1.0      # modulus -> nuisance modulus of PA j
    G[dd["o_eta"], 5 * Kt] = 1.0
    return G


def snapshot_fim(geom, x, sfvs, rho_t, eta, coherent):
    """Classic snapshot FIM J_C = sum_j G_j J_ch^(j) G_j^T (eq. FIMclassic).
    x: (6,) MT state; sfvs: (K, 3); rho_t: (J, K~) complex amplitudes rho~."""
    K = len(sfvs)
    dd = dims(K, geom.J, coherent)
    Jg = np.zeros((dd["dim"], dd["dim"]))
    for j in range(geom.J):
        Jc, rps, Hs = local_fim(geom, j, x[:3], sfvs, rho_t[j], eta)
        G = jacobian(geom, j, K, coherent, x[:3], sfvs, rps, Hs)
        Jg += G @ Jc @ G.T
    return Jg


def transition(params, K, J, coherent, sigma_phi, sigma_a, sigma_eta):
    """F and Q of the global state (Sec. S-VII): NCV block, identity random walk of the
    SFVs, and nuisance parameters without memory (pseudo variances sigma_*^2)."""
    dd = dims(K, J, coherent)
    Fa, Qa = model.ncv_matrices(params.T, params.sigma_v, params.motion_dims)
    F = np.zeros((dd["dim"], dd["dim"]))
    Q = np.zeros_like(F)
    F[:6, :6] = Fa
    Q[:6, :6] = Qa
    o = dd["o_sfv"]
    F[o:o + 3 * K, o:o + 3 * K] = np.eye(3 * K)
    Q[o:o + 3 * K, o:o + 3 * K] = params.sigma_sfv ** 2 * np.eye(3 * K)
    Q[dd["o_ph"]:dd["o_a"], dd["o_ph"]:dd["o_a"]] = sigma_phi ** 2 * np.eye(dd["nph"])
    Q[dd["o_a"]:dd["o_eta"], dd["o_a"]:dd["o_eta"]] = sigma_a ** 2 * np.eye(dd["o_eta"] - dd["o_a"])
    Q[dd["o_eta"], dd["o_eta"]] = sigma_eta ** 2
    return F, Q


def recursion(J_snap, F, Q, J10):
    """J_{n|n} = J_B,n + (F J_{n-1|n-1}^-1 F^T + Q)^-1 from J_{1|0} = J10 (eq. posteriorCRLB,
    priorFIM); returns the posterior information matrices."""
    out = []
    Jpred = J10
    for n, Jb in enumerate(J_snap):
        Jpost = Jb + Jpred
        out.append(Jpost)
        Jpred = np.linalg.inv(F @ np.linalg.inv(Jpost) @ F.T + Q)
    return out


def bounds(Jpost, K):
    """PEB = sqrt(tr P[0:3, 0:3]) and MEB_k = sqrt(tr P over SFV k), P = J^-1."""
    P = np.linalg.inv(Jpost)
    peb = float(np.sqrt(np.trace(P[0:3, 0:3])))
    meb = [float(np.sqrt(np.trace(P[6 + 3 * k:9 + 3 * k, 6 + 3 * k:9 + 3 * k]))) for k in range(K)]
    return peb, meb
