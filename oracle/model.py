"""Prediction and birth (oracle, FP64 arithmetic, FP32 particle storage).

Test infrastructure only.  Follows:
  * MT NCV transition N(x; Phi_a x, sigma_v^2 Gamma Gamma^T), Gamma = [T^2/2 I, T I]^T (Sec. V-A)
  * noise variance Gamma(c_eta, eta/c_eta), gamma Gamma(c_gamma, gamma/c_gamma),
    mu ~ CN(mu, sigma_mu^2), p_sfv ~ N(p_sfv, sigma_sfv^2 I) (Sec. V-A)
  * SIR prediction with w_beta = w_x, w_xi = w_eta, w_alpha = p_S w_y (Sec. IV-D,
    eq. PR-prediction-PDF and the paragraph after it)
  * PR prediction zeta(1) = p_S^PR p~ + p_R^PR (1 - p~) (eq. zeta)
  * birth: Bernoulli with p_B = mu_B/(1+mu_B) (Sec. III-B2), particles from
    f_B = U(partition) U(0, gamma_max) U(|mu| <= mu_max), weights p_B/P,
    PR prior zeta(1) = p_B^PR (Sec. IV-B, IV-D, V-A)
Pins: P5 (NCV mean/covariance vs Kalman prediction), P6 (Gamma moments,
p_B = 1/3 at mu_B = 0.5).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import rng


@dataclasses.dataclass
class Predicted:
    """Particle representations of the prediction messages at step n."""
    n: int
    S: int
    x: np.ndarray          # (6, P) float32   particles of beta(x_n)
    phi: np.ndarray        # (S, 6, P) float32 particles of alpha(phi_s, 1)
    eta: np.ndarray        # (J, P) float32   particles of xi(eta^(j))
    w_beta: np.ndarray     # (P,)
    w_alpha: np.ndarray    # (S, P)
    w_xi: np.ndarray       # (J, P)
    zeta: np.ndarray       # (S, J)  zeta(r_s^(j) = 1)
    is_new: np.ndarray     # (S,) bool


def birth_probability(mu_B: float, Q: int) -> float:
    """p_B^(q) = mu_B^(q)/(1 + mu_B^(q)) with mu_B^(q) = mu_B/Q (equal partitions)."""
    mq = mu_B / max(Q, 1)
    return mq / (1.0 + mq)


def ncv_matrices(T: float, sigma_v: float, motion_dims: int = 3):
    """Phi_a and Q_a = sigma_v^2 Gamma Gamma^T of the NCV model (Sec. V-A)."""
    F = np.eye(6)
    F[0, 3] = F[1, 4] = F[2, 5] = T
    G = np.vstack([0.5 * T * T * np.eye(3), T * np.eye(3)])
    if motion_dims == 2:
        G[:, 2] = 0.0
    return F, sigma_v ** 2 * (G @ G.T)


def predict(state, params, J: int, seed: int, S_max: int) -> Predicted:
    """Phase (i) of the schedule (Sec. IV): prediction of every belief plus births."""
    n = state.n + 1
    P = state.x.shape[1]
    S = state.S
    idx = np.arange(P, dtype=np.uint64)
    T = params.T

    # --- MT state: x_n = Phi_a x_{n-1} + Gamma w,  w ~ N(0, sigma_v^2 I) --------
    x = state.x.astype(np.float64)
    w = np.array(rng.normals(seed, idx, n, rng.MT_PREDICT, 0, 3)) * params.sigma_v
    if params.motion_dims == 2:
        w[2] = 0.0
    xn = np.empty_like(x)
    xn[:3] = x[:3] + T * x[3:] + 0.5 * T * T * w
    xn[3:] = x[3:] + T * w

    # --- noise variances: Gamma(c_eta, eta/c_eta) ----------------------------------
    eta = state.eta.astype(np.float64)
    etan = np.empty_like(eta)
    for j in range(J):
        etan[j] = rng.gamma(seed, idx, n, rng.ETA_PREDICT, j, params.c_eta, eta[j] / params.c_eta)

    # --- legacy PFs ----------------------------------------------------------------
    S_new = min(S + params.Q, S_max) if params.Q > 0 else S
    phi = np.zeros((S_new, 6, P))
    phi[:S] = state.phi.astype(np.float64)
    for s in range(S):
        g = rng.normals(seed, idx, n, rng.PF_GAUSS, s, 5)
        if s > 0:
            for k in range(3):
                if not (params.motion_dims == 2 and k == 2):
                    phi[s, k] = phi[s, k] + params.sigma_sfv * g[k]
        phi[s, 3] = rng.gamma(seed, idx, n, rng.PF_GAMMA, s, params.c_gamma, phi[s, 3] / params.c_gamma)
        if params.zero_mean:
            phi[s, 4:] = 0.0
        else:
            sd = params.sigma_mu / np.sqrt(2.0)   # circular CN(0, sigma_mu^2)
            phi[s, 4] = phi[s, 4] + sd * g[3]
            phi[s, 5] = phi[s, 5] + sd * g[4]
    w_alpha = np.zeros((S_new, P))
    w_alpha[:S] = params.pS * state.w_y
    zeta = np.zeros((S_new, J))
    zeta[:S] = params.pS_pr * state.p_pr + params.pR_pr * (1.0 - state.p_pr)
    is_new = np.zeros(S_new, bool)

    # --- births: one PF per partition q (slabs of the birth box along x) ---------
    Q = S_new - S
    pB = birth_probability(params.mu_B, params.Q)
    blo = np.asarray(params.birth_min, float)
    bhi = np.asarray(params.birth_max, float)
    for q in range(Q):
        s = S + q
        u = rng.uniforms24(seed, idx, n, rng.BIRTH, s, 6)
        lo = blo.copy(); hi = bhi.copy()
        width = (bhi[0] - blo[0]) / params.Q
        lo[0] = blo[0] + q * width
        hi[0] = lo[0] + width
        for k in range(3):
            phi[s, k] = lo[k] + (hi[k] - lo[k]) * u[k]
        phi[s, 3] = params.gamma_max * u[3]
        if params.zero_mean:
            phi[s, 4:] = 0.0
        else:
            r = params.mu_max * np.sqrt(u[4])
            t = 2.0 * np.pi * u[5]
            phi[s, 4] = r * np.cos(t)
            phi[s, 5] = r * np.sin(t)
        w_alpha[s] = pB / P
        zeta[s] = params.pB_pr
        is_new[s] = True

    return Predicted(n=n, S=S_new, x=xn.astype(np.float32), phi=phi.astype(np.float32),
                     eta=etan.astype(np.float32), w_beta=state.w_x.copy(), w_alpha=w_alpha,
                     w_xi=state.w_eta.copy(), zeta=zeta, is_new=is_new)


def init_state(params, J: int, P: int, seed: int, S0: int = 1):
    """Time-0 beliefs (Sec. V-A): x_0 ~ U(p_min, p_max) U(-v_max, v_max),
    eta_0 ~ U(eta_min, eta_max), and the LoS (slot 0) drawn like a new PF with
    existence p_B and PR existence p_B^PR (reading R6b).  Slots 1 .. S0-1 (S0 > 1
    starts a filter with that many PFs, for the batched scenarios) are drawn from
    the birth density f_B of Sec. III-B2 over the whole birth box
    U(2 p_min, 2 p_max) x U(0, gamma_max) x uniform disc of radius mu_max, each with
    existence p_B and PR existence p_B^PR like a new PF (Sec. IV-D)."""
    from paper_2604_19723_gb300.workload import StateArrays
    idx = np.arange(P, dtype=np.uint64)
    lo, hi = np.asarray(params.p_min), np.asarray(params.p_max)
    vm = np.asarray(params.v_max)
    u = rng.uniforms24(seed, idx, 0, rng.INIT_MT, 0, 6)
    x = np.empty((6, P))
    for k in range(3):
        x[k] = lo[k] + (hi[k] - lo[k]) * u[k]
        x[3 + k] = -vm[k] + 2.0 * vm[k] * u[3 + k]
    if params.motion_dims == 2:
        x[5] = 0.0
    eta = np.empty((J, P))
    for j in range(J):
        ue = rng.uniforms24(seed, idx, 0, rng.INIT_ETA, j, 1)[0]
        eta[j] = params.eta_min + (params.eta_max - params.eta_min) * ue
    phi = np.zeros((1, 6, P))
    ub = rng.uniforms24(seed, idx, 0, rng.BIRTH, 0, 6)
    phi[0, 3] = params.gamma_max * ub[3]
    if not params.zero_mean:
        r = params.mu_max * np.sqrt(ub[4])
        t = 2.0 * np.pi * ub[5]
        phi[0, 4] = r * np.cos(t)
        phi[0, 5] = r * np.sin(t)
    if S0 > 1:
        phi = np.concatenate([phi, np.zeros((S0 - 1, 6, P))])
        blo = np.asarray(params.birth_min, float)
        bhi = np.asarray(params.birth_max, float)
        for s in range(1, S0):
            ub = rng.uniforms24(seed, idx, 0, rng.BIRTH, s, 6)
            for k in range(3):
                phi[s, k] = blo[k] + (bhi[k] - blo[k]) * ub[k]
            phi[s, 3] = params.gamma_max * ub[3]
            if not params.zero_mean:
                r = params.mu_max * np.sqrt(ub[4])
                t = 2.0 * np.pi * ub[5]
                phi[s, 4] = r * np.cos(t)
                phi[s, 5] = r * np.sin(t)
    pB = birth_probability(params.mu_B, max(params.Q, 1))
    return StateArrays(n=0, S=S0, x=x.astype(np.float32), phi=phi.astype(np.float32),
                       eta=eta.astype(np.float32), w_x=np.full(P, 1.0 / P),
                       w_y=np.full((S0, P), pB / P), w_eta=np.full((J, P), 1.0 / P),
                       p_pr=np.full((S0, J), params.pB_pr))
