"""Seeded synthetic workloads: constants, scenario layout, truth and particle states.

This module is the one place both the CUDA path (through the tests and the
bench) and the FP64 oracle take their inputs from.  It holds none of the
method's arithmetic: no steering vector, no likelihood, no transition density
is evaluated here.  It only fixes numbers and draws seeded random arrays.

Paper constants (Sec. V-A, "Common Simulation Setup", and the Experiment 1/2
paragraphs of Sec. V):
  * MT prior box p_min = -[3.5 1 1], p_max = [4.5 4.5 1], |v| <= 0.5 m/s per axis
  * eta prior U(1e-9, 1e-4); c_eta = c_gamma = 100
  * p_S = 0.8, p_S^PR = 0.9, p_R^PR = 0.1, T_dec = 0.5, T_pru = 0.1
  * Q = 1 birth per step from U(2 p_min, 2 p_max) x U(0, gamma_max) x U(|mu| <= mu_max)
    with gamma_max = 5, mu_max = 1e-3, mu_B = 0.5 (so p_B = 1/3), p_B^PR = 0.3
  * Nf = 10 bins over B, fc = 3.5 GHz, J = 4 URAs of 4 x 4 at lambda/2, SNR 20 dB
  * Exp. 1: P = 30000, sigma_v = 0.5, B = 200 MHz, sigma_mu = 3e-3, sigma_sfv = 0.1 mm
  * Exp. 2: P = 15000, sigma_v = 7.7, B = 100 MHz, sigma_mu = 3e-2, sigma_sfv = 4 mm

The room geometry, PA poses and the MT trajectory of the paper exist only in
figures that are not available; the layout below is a stand-in with the same
shapes: four walls of the room (the ROI) as surface feature vectors, four PAs
inside the room facing its centre, and a smooth deterministic trajectory.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

LIGHT_SPEED = 299792458.0


# --------------------------------------------------------------------------
# configuration records
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Geometry:
    """Array / signal constants (Sec. II-B): J PAs, Nf x My x Mz samples."""
    J: int
    Nf: int
    My: int
    Mz: int
    fc: float
    B: float
    c: float
    p_pa: np.ndarray      # (J, 3)   PA centres, global frame
    R_pa: np.ndarray      # (J, 3, 3) rotation local -> global (columns = local axes)
    p_y: np.ndarray       # (My,)    template horizontal element positions
    p_z: np.ndarray       # (Mz,)    template vertical element positions

    @property
    def Nz(self) -> int:
        return self.Nf * self.My * self.Mz

    @property
    def wavelength(self) -> float:
        return self.c / self.fc

    def freqs(self) -> np.ndarray:
        """Baseband frequencies f_k = -B/2 + k B/(Nf-1), symmetric about 0."""
        if self.Nf == 1:
            return np.zeros(1)
        return -0.5 * self.B + np.arange(self.Nf) * (self.B / (self.Nf - 1))


@dataclasses.dataclass
class Params:
    """Filter parameters (Sec. III-B, Sec. V).  Field names follow the paper."""
    T: float = 0.1                 # time step [s]
    sigma_v: float = 0.5           # NCV process-noise std [m/s^2]
    motion_dims: int = 3           # 3: 3-D NCV; 2: planar (z and v_z held)
    c_eta: float = 100.0
    c_gamma: float = 100.0
    sigma_mu: float = 3e-3
    sigma_sfv: float = 1e-4
    pS: float = 0.8
    pS_pr: float = 0.9
    pR_pr: float = 0.1
    pB_pr: float = 0.3
    mu_B: float = 0.5
    Q: int = 1                     # births per step (0 disables birth)
    T_dec: float = 0.5
    T_pru: float = 0.1             # 0 disables pruning
    gamma_max: float = 5.0
    mu_max: float = 1e-3
    eta_min: float = 1e-9
    eta_max: float = 1e-4
    p_min: tuple = (-3.5, -1.0, -1.0)
    p_max: tuple = (4.5, 4.5, 1.0)
    v_max: tuple = (0.5, 0.5, 0.5)
    zero_mean: int = 0             # 1: ZM variant (mu == 0)
    mvec_scaling: int = 0          # 0: m-vectors as printed in S-V; 1: sqrt(pi) reading
    regularize: int = 1            # Gaussian-kernel jitter after resampling
    birth_proposal: int = 0        # 1: new PFs drawn from the Bartlett proposal (Sec. IV-D)
    N_g: int = 4096                # candidate positions per new PF of the proposal

    @property
    def birth_min(self):
        return tuple(2.0 * v for v in self.p_min)

    @property
    def birth_max(self):
        return tuple(2.0 * v for v in self.p_max)


@dataclasses.dataclass
class Scenario:
    """Ground truth of one synthetic run (inputs for the signal generator)."""
    geom: Geometry
    params: Params
    N: int                         # number of steps
    x_true: np.ndarray             # (N+1, 6) MT state per step (index 0 = time 0)
    sfv_true: np.ndarray           # (K, 3)   SFV positions of the K surfaces
    rho_abs: np.ndarray            # (K+1,)   |amplitude|, index 0 = LoS
    rho_phase: np.ndarray          # (N+1, J, K+1) amplitude phases [rad]
    visible: np.ndarray            # (N+1, J, K+1) bool visibility of each path
    clutter_sfv: List[np.ndarray]  # per step (Kc, 3) spurious SFVs (not in the paper)
    clutter_rho: List[np.ndarray]  # per step (Kc, J) complex spurious amplitudes
    snr_db: float
    seed: int


# --------------------------------------------------------------------------
# layout helpers (scenario setup only)
# --------------------------------------------------------------------------
def ura_template(M: int, wavelength: float) -> np.ndarray:
    """Element positions ((0..M-1) - (M-1)/2) * lambda/2, symmetric about 0."""
    return (np.arange(M) - 0.5 * (M - 1)) * (0.5 * wavelength)


def facing_rotation(p_pa: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Rotation whose local x-axis (array boresight) points horizontally at target."""
    d = np.asarray(target, float) - np.asarray(p_pa, float)
    d[2] = 0.0
    ex = d / np.linalg.norm(d)
    ez = np.array([0.0, 0.0, 1.0])
    ey = np.cross(ez, ex)
    return np.stack([ex, ey, ez], axis=1)


def room_pas(J: int, p_min, p_max, height: float = 0.5) -> np.ndarray:
    """J PA centres inside the room near its walls (corners first)."""
    lo = np.asarray(p_min, float)
    hi = np.asarray(p_max, float)
    inset = 0.3
    cands = [
        (lo[0] + inset, lo[1] + inset), (hi[0] - inset, hi[1] - inset),
        (hi[0] - inset, lo[1] + inset), (lo[0] + inset, hi[1] - inset),
        (0.5 * (lo[0] + hi[0]), lo[1] + inset), (0.5 * (lo[0] + hi[0]), hi[1] - inset),
        (lo[0] + inset, 0.5 * (lo[1] + hi[1])), (hi[0] - inset, 0.5 * (lo[1] + hi[1])),
    ]
    out = []
    for j in range(J):
        x, y = cands[j % len(cands)]
        out.append((x, y, height + 0.05 * (j // len(cands))))
    return np.asarray(out, float)


def make_geometry(J: int = 4, Nf: int = 10, My: int = 4, Mz: int = 4,
                  fc: float = 3.5e9, B: float = 200e6,
                  p_min=(-3.5, -1.0, -1.0), p_max=(4.5, 4.5, 1.0)) -> Geometry:
    lam = LIGHT_SPEED / fc
    p_pa = room_pas(J, p_min, p_max)
    centre = 0.5 * (np.asarray(p_min) + np.asarray(p_max))
    R = np.stack([facing_rotation(p_pa[j], centre) for j in range(J)])
    return Geometry(J=J, Nf=Nf, My=My, Mz=Mz, fc=fc, B=B, c=LIGHT_SPEED,
                    p_pa=p_pa, R_pa=R, p_y=ura_template(My, lam), p_z=ura_template(Mz, lam))


def room_sfvs(p_min, p_max, inset: float = 0.1) -> np.ndarray:
    """SFVs of the four vertical walls of the room: p_sfv = 2 * (wall point)."""
    lo = np.asarray(p_min, float)
    hi = np.asarray(p_max, float)
    walls = [
        np.array([lo[0] + inset, 0.0, 0.0]), np.array([hi[0] - inset, 0.0, 0.0]),
        np.array([0.0, lo[1] + inset, 0.0]), np.array([0.0, hi[1] - inset, 0.0]),
    ]
    return 2.0 * np.stack(walls)


def random_sfvs(rng: np.random.Generator, K: int, p_min, p_max, r_min: float = 1.0) -> np.ndarray:
    """K SFVs drawn inside the birth box U(2 p_min, 2 p_max), away from the origin."""
    lo = 2.0 * np.asarray(p_min, float)
    hi = 2.0 * np.asarray(p_max, float)
    out = []
    while len(out) < K:
        v = lo + (hi - lo) * rng.random(3)
        if np.linalg.norm(v) > r_min:
            out.append(v)
    return np.asarray(out, float).reshape(K, 3)


def lissajous_truth(N: int, T: float, p_min, p_max, motion_dims: int = 3,
                    phase: float = 0.0) -> np.ndarray:
    """Deterministic smooth MT trajectory inside the room, (N+1, 6) [p; v]."""
    lo = np.asarray(p_min, float)
    hi = np.asarray(p_max, float)
    c = 0.5 * (lo + hi)
    a = 0.3 * (hi - lo)
    t = np.arange(N + 1) * T
    w = np.array([0.21, 0.33, 0.17])
    ph = np.array([0.3, 1.1, 0.7]) + phase
    p = c[None, :] + a[None, :] * np.sin(w[None, :] * t[:, None] + ph[None, :])
    v = a[None, :] * w[None, :] * np.cos(w[None, :] * t[:, None] + ph[None, :])
    if motion_dims == 2:
        p[:, 2] = 0.0
        v[:, 2] = 0.0
    else:
        p[:, 2] = 0.3 * np.sin(0.11 * t + 0.2)
        v[:, 2] = 0.3 * 0.11 * np.cos(0.11 * t + 0.2)
    return np.concatenate([p, v], axis=1)


def make_scenario(geom: Geometry, params: Params, N: int, K: int, seed: int,
                  snr_db: float = 20.0, visibility: float = 1.0,
                  clutter_mean: float = 0.0, coherent: bool = True,
                  rho_los: float = 1.0, rho_mpc: float = 0.5,
                  clutter_rho: float = 0.05) -> Scenario:
    """Ground truth: trajectory, K surfaces (room walls first, then random SFVs),
    amplitude moduli/phases, per-step visibility and optional spurious paths."""
    rng = np.random.default_rng(seed)
    x_true = lissajous_truth(N, params.T, params.p_min, params.p_max, params.motion_dims)
    walls = room_sfvs(params.p_min, params.p_max)
    if K <= 4:
        sfv = walls[:K].copy()
    else:
        sfv = np.concatenate([walls, random_sfvs(rng, K - 4, params.p_min, params.p_max)])
    rho_abs = np.concatenate([[rho_los], np.full(K, rho_mpc)])
    J = geom.J
    base_phase = rng.uniform(-np.pi, np.pi, size=K + 1)
    if coherent:
        rho_phase = np.broadcast_to(base_phase, (N + 1, J, K + 1)).copy()
    else:
        rho_phase = rng.uniform(-np.pi, np.pi, size=(N + 1, J, K + 1))
    visible = rng.random((N + 1, J, K + 1)) < visibility
    cs, cr = [], []
    for n in range(N + 1):
        kc = int(rng.poisson(clutter_mean)) if clutter_mean > 0 else 0
        cs.append(random_sfvs(rng, kc, params.p_min, params.p_max))
        ph = rng.uniform(-np.pi, np.pi, size=(kc, J))
        cr.append(clutter_rho * np.exp(1j * ph))
    return Scenario(geom=geom, params=params, N=N, x_true=x_true, sfv_true=sfv,
                    rho_abs=rho_abs, rho_phase=rho_phase, visible=visible,
                    clutter_sfv=cs, clutter_rho=cr, snr_db=snr_db, seed=seed)


# --------------------------------------------------------------------------
# named workloads (shapes of the paper's experiments and of the scaled cases)
# --------------------------------------------------------------------------
def workload(name: str) -> Dict:
    """Sizes and parameters of a named workload.  Keys: geom, params, P, S_max,
    N, K (true surfaces), visibility, clutter_mean, snr_db, seed, fixed_S."""
    if name == "small_fp64":
        # one PA, planar 2-D NCV (sigma_v 0.1, T 0.1), LoS + 4 walls, 1000 particles, 50 steps
        g = make_geometry(J=1, Nf=10, My=4, Mz=4, B=200e6)
        p = Params(T=0.1, sigma_v=0.1, motion_dims=2, sigma_mu=3e-3, sigma_sfv=1e-4,
                   p_min=(-3.5, -1.0, 0.0), p_max=(4.5, 4.5, 0.0))
        return dict(geom=g, params=p, P=1000, S_max=16, N=50, K=4, visibility=0.9,
                    clutter_mean=10.0, snr_db=20.0, seed=0, fixed_S=0)
    if name == "paper_exp1":
        g = make_geometry(J=4, Nf=10, My=4, Mz=4, B=200e6)
        p = Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4)
        return dict(geom=g, params=p, P=30000, S_max=16, N=200, K=4, visibility=1.0,
                    clutter_mean=0.0, snr_db=20.0, seed=1, fixed_S=0)
    if name == "paper_exp1_proposal":
        # Experiment 1 with new PFs drawn from the Bartlett birth proposal (Sec. IV-D)
        g = make_geometry(J=4, Nf=10, My=4, Mz=4, B=200e6)
        p = Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4, birth_proposal=1, N_g=4096)
        return dict(geom=g, params=p, P=30000, S_max=16, N=200, K=4, visibility=1.0,
                    clutter_mean=0.0, snr_db=20.0, seed=1, fixed_S=0)
    if name == "paper_exp2":
        g = make_geometry(J=4, Nf=10, My=4, Mz=4, B=100e6)
        p = Params(T=0.1, sigma_v=7.7, sigma_mu=3e-2, sigma_sfv=4e-3)
        return dict(geom=g, params=p, P=15000, S_max=16, N=200, K=4, visibility=1.0,
                    clutter_mean=0.0, snr_db=20.0, seed=2, fixed_S=0)
    if name == "scale_64x100k":
        # 64 PFs held fixed (no birth, no pruning), 1e5 particles, J = 4, Nz = 160
        g = make_geometry(J=4, Nf=10, My=4, Mz=4, B=200e6)
        p = Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4, Q=0, T_pru=0.0)
        return dict(geom=g, params=p, P=100000, S_max=64, N=200, K=63, visibility=0.8,
                    clutter_mean=200.0, snr_db=20.0, seed=3, fixed_S=64)
    if name == "stress_32x262k":
        # 32 PFs, 262144 particles, Nz = 1024 (Nf = 16, 8 x 8 URA), SNR 30 dB
        g = make_geometry(J=4, Nf=16, My=8, Mz=8, B=200e6)
        p = Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4, Q=0, T_pru=0.0)
        return dict(geom=g, params=p, P=262144, S_max=32, N=200, K=31, visibility=0.8,
                    clutter_mean=500.0, snr_db=30.0, seed=4, fixed_S=32)
    raise KeyError(name)


def batched_scenarios(n: int, seed: int = 21, S_range=(1, 64), P_range=(256, 16384), Nz_range=(5, 300)) -> List[Dict]:
    """Shapes of the batched workload: n independent scenarios with S ~ U{1..64} PFs
    (held fixed: no birth, no pruning), P ~ U{256..16384} particles and Nz ~ U{5..300}
    samples per PA at J = 4.  Nz < 16 is one antenna with Nf = Nz frequencies, larger
    Nz a 2 x 2 URA with Nf = ceil(Nz / 4) (so Nz rounds up to a multiple of 4).  Each
    entry: geom, params, P, S, seed (its own Philox key and truth)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        S = int(rng.integers(S_range[0], S_range[1] + 1))
        P = int(rng.integers(P_range[0], P_range[1] + 1))
        nz = int(rng.integers(Nz_range[0], Nz_range[1] + 1))
        if nz < 16:
            g = make_geometry(J=4, Nf=nz, My=1, Mz=1, B=200e6)
        else:
            g = make_geometry(J=4, Nf=-(-nz // 4), My=2, Mz=2, B=200e6)
        prm = Params(T=0.1, sigma_v=0.5, sigma_mu=3e-3, sigma_sfv=1e-4, Q=0, T_pru=0.0)
        out.append(dict(geom=g, params=prm, P=P, S=S, seed=seed * 100003 + i))
    return out


# --------------------------------------------------------------------------
# particle states (inputs for stage-wise parity; FP32 storage as in the SoA layout)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class StateArrays:
    """One filter state in host memory.  Particles are FP32 (SoA), weights and
    existence probabilities FP64.  PF slot 0 is the LoS (its p_sfv is unused)."""
    n: int                    # index of the last completed step
    S: int                    # number of PFs including the LoS
    x: np.ndarray             # (6, P)        float32
    phi: np.ndarray           # (S, 6, P)     float32 [px py pz gamma mu_re mu_im]
    eta: np.ndarray           # (J, P)        float32
    w_x: np.ndarray           # (P,)          float64, sums to 1
    w_y: np.ndarray           # (S, P)        float64, sums to p_s
    w_eta: np.ndarray         # (J, P)        float64, sums to 1
    p_pr: np.ndarray          # (S, J)        float64, p(r_s^(j) = 1 | z_1:n)

    def copy(self) -> "StateArrays":
        return dataclasses.replace(self, x=self.x.copy(), phi=self.phi.copy(), eta=self.eta.copy(),
                                   w_x=self.w_x.copy(), w_y=self.w_y.copy(),
                                   w_eta=self.w_eta.copy(), p_pr=self.p_pr.copy())


def state_near_truth(scn: Scenario, P: int, S: int, n: int, seed: int,
                     pos_std: float = 0.02, vel_std: float = 0.05, sfv_std: float = 0.02,
                     eta_scale: float = 1.0, rho_rel_std: float = 0.1,
                     uniform_weights: bool = True, eta_true: Optional[float] = None) -> StateArrays:
    """A plausible filter state around the truth at step n (for stage-wise tests).

    MT particles ~ truth + N(0, diag(pos_std^2, vel_std^2)); PF s >= 1 tracks
    surface s-1 (cycled if S-1 > K); gamma near |rho|^2, mu near the true
    amplitude; eta around eta_true (or 1e-8).  Weights uniform (or random)."""
    rng = np.random.default_rng(seed)
    J = scn.geom.J
    K = scn.sfv_true.shape[0]
    x0 = scn.x_true[n]
    x = np.empty((6, P))
    x[:3] = x0[:3, None] + pos_std * rng.standard_normal((3, P))
    x[3:] = x0[3:, None] + vel_std * rng.standard_normal((3, P))
    if scn.params.motion_dims == 2:
        x[2] = x0[2]
        x[5] = 0.0
    phi = np.zeros((S, 6, P))
    for s in range(S):
        k = 0 if s == 0 else 1 + ((s - 1) % max(K, 1))
        if s > 0 and K > 0:
            phi[s, :3] = scn.sfv_true[k - 1][:, None] + sfv_std * rng.standard_normal((3, P))
        a = scn.rho_abs[min(k, len(scn.rho_abs) - 1)]
        ph = scn.rho_phase[n, 0, min(k, scn.rho_phase.shape[2] - 1)]
        phi[s, 3] = (a * a) * rng.uniform(0.5, 1.5, P)
        if scn.params.zero_mean:
            phi[s, 4:] = 0.0
        else:
            m = a * np.exp(1j * ph)
            d = rho_rel_std * a * (rng.standard_normal(P) + 1j * rng.standard_normal(P)) / math.sqrt(2)
            phi[s, 4] = (m + d).real
            phi[s, 5] = (m + d).imag
    et = 1e-8 if eta_true is None else eta_true
    eta = et * eta_scale * np.exp(0.3 * rng.standard_normal((J, P)))
    p_s = rng.uniform(0.3, 0.99, S)
    if uniform_weights:
        w_x = np.full(P, 1.0 / P)
        w_eta = np.full((J, P), 1.0 / P)
        w_y = p_s[:, None] * np.full((S, P), 1.0 / P)
    else:
        w_x = rng.random(P); w_x /= w_x.sum()
        w_eta = rng.random((J, P)); w_eta /= w_eta.sum(axis=1, keepdims=True)
        w_y = rng.random((S, P)); w_y *= (p_s / w_y.sum(axis=1))[:, None]
    p_pr = rng.uniform(0.2, 0.99, (S, J))
    return StateArrays(n=n, S=S, x=x.astype(np.float32), phi=phi.astype(np.float32),
                       eta=eta.astype(np.float32), w_x=w_x, w_y=w_y, w_eta=w_eta, p_pr=p_pr)


def state_from_prior(params: Params, J: int, P: int, S: int, seed: int) -> StateArrays:
    """A diffuse state: MT from the uniform prior box, PFs from the birth box."""
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(params.p_min), np.asarray(params.p_max)
    vm = np.asarray(params.v_max)
    x = np.empty((6, P))
    x[:3] = lo[:, None] + (hi - lo)[:, None] * rng.random((3, P))
    x[3:] = -vm[:, None] + 2 * vm[:, None] * rng.random((3, P))
    blo, bhi = 2 * lo, 2 * hi
    phi = np.zeros((S, 6, P))
    for s in range(S):
        if s > 0:
            phi[s, :3] = blo[:, None] + (bhi - blo)[:, None] * rng.random((3, P))
        phi[s, 3] = params.gamma_max * rng.random(P)
        if not params.zero_mean:
            r = params.mu_max * np.sqrt(rng.random(P))
            t = 2 * np.pi * rng.random(P)
            phi[s, 4] = r * np.cos(t)
            phi[s, 5] = r * np.sin(t)
    eta = params.eta_min + (params.eta_max - params.eta_min) * rng.random((J, P))
    p_s = np.full(S, 0.5)
    return StateArrays(n=0, S=S, x=x.astype(np.float32), phi=phi.astype(np.float32),
                       eta=eta.astype(np.float32), w_x=np.full(P, 1.0 / P),
                       w_y=np.full((S, P), 0.5 / P), w_eta=np.full((J, P), 1.0 / P),
                       p_pr=np.full((S, J), params.pB_pr))


# --------------------------------------------------------------------------
# proposal network: initial parameters (random inputs of training)
# --------------------------------------------------------------------------
def mlp_init(seed: int, out_scale: float = 0.1) -> np.ndarray:
    """Initial parameters of the 16-64-64-16 proposal network, packed W1, b1, W2, b2,
    W3, b3: He-uniform weights for the ReLU layers, the output layer scaled down by
    out_scale, zero biases.  FP32."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out, scale in ((16, 64, 1.0), (64, 64, 1.0), (64, 16, out_scale)):
        lim = scale * np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)).reshape(-1))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)

