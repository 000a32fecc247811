"""Beliefs, normalisation, estimates, declaration and pruning (oracle, FP64).

Test infrastructure only.  Follows:
  * particle beliefs  w~_x = w_beta prod_j iota~,  w~_y,s = w_alpha,s prod_j kappa~(., 1),
    w~_eta = w_xi nu~  (Sec. IV-D "Beliefs", Sec. S-III)
  * normalisation constants C_x = sum w~_x, C_eta = sum w~_eta and
    C_y,s = sum_p w~_y,s + (1 - sum_p w_alpha,s) prod_j kappa~(., 0) (Sec. S-IV)
  * p_s = sum_p w_y,s (eq. existenceProb)
  * PR belief p~(r = 1) = zeta omega~(1)/(zeta omega~(1) + (1 - zeta) omega~(0))
    (eq. PR-normalization), evaluated as the logistic of the log-odds (Sec. S-VI)
  * MMSE estimates (eq. stateHat, etanHat, PFphiHat), declaration p_s > T_dec,
    p^PR_s = 1 - prod_j (1 - p_s^(j)), pruning p_s < T_pru or p^PR_s < T_pru,
    never the LoS (Sec. II-C)
Pins: P7 (weights sum to one / to p_s, the S-IV identity, logistic == ratio).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def logsumexp(a, axis=None):
    a = np.asarray(a, np.float64)
    m = np.max(a, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    out = np.log(np.sum(np.exp(a - m), axis=axis, keepdims=True)) + m
    return np.squeeze(out, axis=axis) if axis is not None else float(out.reshape(()))


def logistic_from_log_odds(u):
    """sigma(u) = 1/(1 + exp(-u)), evaluated without overflow."""
    u = np.asarray(u, np.float64)
    return np.where(u >= 0, 1.0 / (1.0 + np.exp(-np.abs(u))), np.exp(-np.abs(u)) / (1.0 + np.exp(-np.abs(u))))


@dataclasses.dataclass
class Beliefs:
    w_x: np.ndarray        # (P,)   normalised
    w_y: np.ndarray        # (S, P) sums to p_s
    w_eta: np.ndarray      # (J, P) normalised per j
    p_s: np.ndarray        # (S,)
    p_pr: np.ndarray       # (S, J) p_s^(j)
    log_wx: np.ndarray     # (P,)   unnormalised log w~_x
    log_wy: np.ndarray     # (S, P) unnormalised log w~_y
    log_weta: np.ndarray   # (J, P)
    log_Cy: np.ndarray     # (S,)
    log_null: np.ndarray   # (S,)   log[(1 - W_s) prod_j kappa~(., 0)]


def pr_existence(zeta, log_omega1, log_omega0):
    """p~(r_s^(j) = 1) as sigma(log zeta/(1-zeta) + log omega~(1)/omega~(0)) (Sec. S-VI)."""
    with np.errstate(divide="ignore"):
        u = np.log(zeta) - np.log1p(-zeta) + (log_omega1 - log_omega0)
    out = logistic_from_log_odds(np.nan_to_num(u, nan=0.0, posinf=np.inf, neginf=-np.inf))
    out = np.where(zeta >= 1.0, 1.0, np.where(zeta <= 0.0, 0.0, out))
    return out


def beliefs(pred, msg) -> Beliefs:
    with np.errstate(divide="ignore"):
        log_wx = np.log(pred.w_beta) + msg.log_iota.sum(axis=0)
        log_weta = np.log(pred.w_xi) + msg.log_nu
        log_wy = np.log(pred.w_alpha) + msg.log_kappa1.sum(axis=1)
        W = pred.w_alpha.sum(axis=1)
        log_null = np.log1p(-np.minimum(W, 1.0)) + msg.log_kappa0.sum(axis=1)
    w_x = np.exp(log_wx - logsumexp(log_wx))
    w_eta = np.exp(log_weta - logsumexp(log_weta, axis=1)[:, None])
    log_Cy = np.array([logsumexp(np.concatenate([log_wy[s], [log_null[s]]])) for s in range(pred.S)])
    w_y = np.exp(log_wy - log_Cy[:, None])
    p_s = w_y.sum(axis=1)
    p_pr = pr_existence(pred.zeta, msg.log_omega1, msg.log_omega0)
    return Beliefs(w_x=w_x, w_y=w_y, w_eta=w_eta, p_s=p_s, p_pr=p_pr, log_wx=log_wx,
                   log_wy=log_wy, log_weta=log_weta, log_Cy=log_Cy, log_null=log_null)


@dataclasses.dataclass
class Estimate:
    x_hat: np.ndarray       # (6,)
    eta_hat: np.ndarray     # (J,)
    p_s: np.ndarray         # (S,)
    phi_hat: np.ndarray     # (S, 6)
    p_pr: np.ndarray        # (S, J)
    p_pr_any: np.ndarray    # (S,)  1 - prod_j (1 - p_s^(j))
    declared: np.ndarray    # (S,) bool
    ess_x: float


def estimate(pred, bel: Beliefs, params) -> Estimate:
    x = pred.x.astype(np.float64)
    x_hat = x @ bel.w_x
    eta_hat = np.sum(bel.w_eta * pred.eta.astype(np.float64), axis=1)
    phi = pred.phi.astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        phi_hat = np.einsum("skp,sp->sk", phi, bel.w_y) / bel.p_s[:, None]
    phi_hat = np.nan_to_num(phi_hat)
    p_any = 1.0 - np.prod(1.0 - bel.p_pr, axis=1)
    return Estimate(x_hat=x_hat, eta_hat=eta_hat, p_s=bel.p_s.copy(), phi_hat=phi_hat,
                    p_pr=bel.p_pr.copy(), p_pr_any=p_any, declared=bel.p_s > params.T_dec,
                    ess_x=float(1.0 / np.sum(bel.w_x ** 2)))


def survivors(est: Estimate, params) -> np.ndarray:
    """Indices of PFs kept for the next step: the LoS always, others unless
    p_s < T_pru or p^PR_s < T_pru (Sec. II-C)."""
    S = len(est.p_s)
    keep = [0] + [s for s in range(1, S)
                  if not (est.p_s[s] < params.T_pru or est.p_pr_any[s] < params.T_pru)]
    return np.asarray(keep, int)
