"""Thin ctypes binding of libbp (include/bp.h).

Argument marshalling only: every step of the filter runs in the CUDA library.
PyTorch supplies device memory for observations and the CUDA stream.  There
is no CPU fallback: if the library cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

from .workload import Geometry, Params, StateArrays

_HERE = os.path.dirname(os.path.abspath(__file__))
# BP_CHECKED=1 selects the checked build (device-side index checks; `build --checked`)
LIB_PATH = os.path.join(_HERE, "_lib", "libbp_checked.so" if os.environ.get("BP_CHECKED") == "1" else "libbp.so")

BP_OK = 0
STATUS = {0: "BP_OK", 1: "BP_ERR_INVALID_ARG", 2: "BP_ERR_CUDA", 3: "BP_ERR_CAPACITY",
          4: "BP_ERR_NUMERIC", 5: "BP_ERR_TIMEOUT", 6: "BP_ERR_STATE"}
DIAG_TABLE, DIAG_WEIGHTS, DIAG_LOGLIK, DIAG_INDICES, DIAG_PROPOSAL, DIAG_LPROP, DIAG_IOTA = 1, 2, 3, 4, 5, 6, 7

ENTRY_POINTS = ("bp_init", "bp_predict", "bp_update", "bp_estimate", "bp_free", "bp_last_error",
                "bp_get_state", "bp_set_state", "bp_get_predicted", "bp_set_predicted", "bp_get_diag",
                "bp_synthesize", "bp_launch_count", "bp_set_profiling", "bp_get_profile",
                "bp_resample_noalloc", "bp_batch_init", "bp_batch_step", "bp_batch_z_offset", "bp_batch_z_floats",
                "bp_batch_sync", "bp_batch_handle", "bp_batch_stream_of", "bp_batch_device_bytes", "bp_batch_free",
                "bp_batch_last_error", "bp_pcrlb_fim", "bp_pcrlb_recursion",
                "bp_mlp_create", "bp_mlp_get_params", "bp_mlp_forward", "bp_mlp_grads", "bp_mlp_train_step",
                "bp_mlp_sync", "bp_mlp_free", "bp_mlp_last_error", "bp_set_mt_proposal", "bp_lp_dataset",
                "bp_selftest_wait", "bp_set_tiles", "bp_get_tiles", "bp_batch_set_tiles")
TILE_FIELDS = ("kappa_sc", "kappa_blocks", "kappa_fch", "kappa_tc", "table_chunk", "table_split")
PROFILE_STAGES = ("predict", "row_sums", "table", "stage", "kappa", "iota", "nu", "normalize", "resample")


class _Tiles(C.Structure):
    _fields_ = [(f, C.c_int) for f in TILE_FIELDS]


class BPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Geometry(C.Structure):
    _fields_ = [("J", C.c_int), ("Nf", C.c_int), ("My", C.c_int), ("Mz", C.c_int),
                ("fc", C.c_double), ("c", C.c_double), ("B", C.c_double),
                ("p_pa", C.POINTER(C.c_double)), ("R_pa", C.POINTER(C.c_double)),
                ("p_y", C.POINTER(C.c_double)), ("p_z", C.POINTER(C.c_double))]


class _Params(C.Structure):
    _fields_ = [("T", C.c_double), ("sigma_v", C.c_double), ("motion_dims", C.c_int),
                ("c_eta", C.c_double), ("c_gamma", C.c_double), ("sigma_mu", C.c_double), ("sigma_sfv", C.c_double),
                ("pS", C.c_double), ("pS_pr", C.c_double), ("pR_pr", C.c_double), ("pB_pr", C.c_double),
                ("mu_B", C.c_double), ("Q", C.c_int),
                ("T_dec", C.c_double), ("T_pru", C.c_double), ("gamma_max", C.c_double), ("mu_max", C.c_double),
                ("eta_min", C.c_double), ("eta_max", C.c_double),
                ("p_min", C.c_double * 3), ("p_max", C.c_double * 3), ("v_max", C.c_double * 3),
                ("zero_mean", C.c_int), ("mvec_scaling", C.c_int), ("regularize", C.c_int),
                ("birth_proposal", C.c_int), ("N_g", C.c_int)]


class _StateView(C.Structure):
    _fields_ = [("n", C.c_int), ("S", C.c_int), ("S_legacy", C.c_int),
                ("x", C.POINTER(C.c_float)), ("phi", C.POINTER(C.c_float)),
                ("eta", C.POINTER(C.c_float)), ("w_x", C.POINTER(C.c_double)), ("w_y", C.POINTER(C.c_double)),
                ("w_eta", C.POINTER(C.c_double)), ("p_pr", C.POINTER(C.c_double))]


class _Estimate(C.Structure):
    _fields_ = [("n", C.c_int), ("S", C.c_int), ("S_next", C.c_int), ("births_skipped", C.c_int),
                ("x_hat", C.c_double * 6), ("ess_x", C.c_double),
                ("eta_hat", C.POINTER(C.c_double)), ("p_s", C.POINTER(C.c_double)),
                ("phi_hat", C.POINTER(C.c_double)), ("p_pr", C.POINTER(C.c_double)),
                ("declared", C.POINTER(C.c_int)), ("iota_repaired", C.c_int)]


class _Scenario(C.Structure):
    _fields_ = [("geom", C.POINTER(_Geometry)), ("params", C.POINTER(_Params)), ("P", C.c_int), ("S_max", C.c_int),
                ("S0", C.c_int), ("seed", C.c_uint64)]


class _BatchOpts(C.Structure):
    _fields_ = [("n_streams", C.c_int), ("shared_workspace", C.c_int), ("use_graph", C.c_int),
                ("cuda_stream", C.c_void_p)]


_lib = None


def load() -> C.CDLL:
    """Load libbp.so (built in-tree by ``paper_2604_19723_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbp.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    lib.bp_init.argtypes = [C.POINTER(_Geometry), C.POINTER(_Params), C.c_int, C.c_int, C.c_uint64, vp, C.POINTER(vp)]
    lib.bp_predict.argtypes = [vp]
    lib.bp_update.argtypes = [vp, vp]
    lib.bp_estimate.argtypes = [vp, C.POINTER(_Estimate)]
    lib.bp_free.argtypes = [vp]
    lib.bp_last_error.argtypes = [vp]
    lib.bp_last_error.restype = C.c_char_p
    for f in ("bp_get_state", "bp_set_state", "bp_get_predicted", "bp_set_predicted"):
        getattr(lib, f).argtypes = [vp, C.POINTER(_StateView)]
    lib.bp_get_diag.argtypes = [vp, C.c_int, vp, C.c_size_t]
    lib.bp_synthesize.argtypes = [C.POINTER(_Geometry), C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int,
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int),
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double, C.c_uint64,
                                  vp, C.POINTER(C.c_double), vp]
    lib.bp_set_profiling.argtypes = [vp, C.c_int]
    lib.bp_get_profile.argtypes = [vp, C.POINTER(C.c_double), C.c_int]
    lib.bp_resample_noalloc.argtypes = [vp, C.c_int, C.c_uint64, C.c_int, C.c_int, C.c_int, vp, vp]
    lib.bp_launch_count.argtypes = [vp]
    lib.bp_launch_count.restype = C.c_longlong
    lib.bp_batch_init.argtypes = [C.POINTER(_Scenario), C.c_int, C.POINTER(_BatchOpts), C.POINTER(vp)]
    lib.bp_batch_step.argtypes = [vp, vp]
    lib.bp_batch_z_offset.argtypes = [vp, C.c_int]
    lib.bp_batch_z_offset.restype = C.c_size_t
    lib.bp_batch_z_floats.argtypes = [vp]
    lib.bp_batch_z_floats.restype = C.c_size_t
    lib.bp_batch_sync.argtypes = [vp]
    lib.bp_batch_handle.argtypes = [vp, C.c_int, C.POINTER(vp)]
    lib.bp_batch_stream_of.argtypes = [vp, C.c_int]
    lib.bp_batch_device_bytes.argtypes = [vp]
    lib.bp_batch_device_bytes.restype = C.c_size_t
    lib.bp_batch_free.argtypes = [vp]
    lib.bp_batch_last_error.argtypes = [vp]
    lib.bp_batch_last_error.restype = C.c_char_p
    lib.bp_pcrlb_fim.argtypes = [C.POINTER(_Geometry), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_double), vp]
    lib.bp_pcrlb_recursion.argtypes = [C.c_int, C.c_int, C.c_int] + [C.POINTER(C.c_double)] * 6 + [vp]
    lib.bp_mlp_create.argtypes = [C.POINTER(C.c_float), vp, C.POINTER(vp)]
    lib.bp_mlp_get_params.argtypes = [vp, C.POINTER(C.c_float)]
    lib.bp_mlp_forward.argtypes = [vp, vp, C.c_int, vp]
    lib.bp_mlp_grads.argtypes = [vp, vp, vp, C.c_int, vp, vp]
    lib.bp_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, vp]
    lib.bp_mlp_sync.argtypes = [vp]
    lib.bp_mlp_free.argtypes = [vp]
    lib.bp_mlp_last_error.argtypes = [vp]
    lib.bp_mlp_last_error.restype = C.c_char_p
    lib.bp_set_mt_proposal.argtypes = [vp, vp]
    lib.bp_selftest_wait.argtypes = [C.c_int, vp]
    lib.bp_set_tiles.argtypes = [vp, C.POINTER(_Tiles)]
    lib.bp_get_tiles.argtypes = [vp, C.POINTER(_Tiles)]
    lib.bp_batch_set_tiles.argtypes = [vp, C.c_int, C.POINTER(_Tiles)]
    lib.bp_lp_dataset.argtypes = [C.POINTER(_Geometry), C.POINTER(_Params), C.c_int, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.c_double, C.c_int] + [C.c_double] * 4 + \
                                 [C.c_int, C.c_uint64, vp, vp, vp]
    untyped = ("bp_last_error", "bp_launch_count", "bp_batch_z_offset", "bp_batch_z_floats",
               "bp_batch_device_bytes", "bp_batch_last_error", "bp_mlp_last_error")
    for f in ENTRY_POINTS:
        if f not in untyped:
            getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class _GeomHolder:
    """Keeps the host arrays referenced by a _Geometry alive."""

    def __init__(self, g: Geometry):
        self.arrs = [np.ascontiguousarray(np.asarray(a, np.float64)) for a in (g.p_pa, g.R_pa, g.p_y, g.p_z)]
        self.s = _Geometry(g.J, g.Nf, g.My, g.Mz, g.fc, g.c, g.B, *[_dptr(a) for a in self.arrs])


def _params_struct(p: Params) -> _Params:
    return _Params(p.T, p.sigma_v, p.motion_dims, p.c_eta, p.c_gamma, p.sigma_mu, p.sigma_sfv,
                   p.pS, p.pS_pr, p.pR_pr, p.pB_pr, p.mu_B, p.Q, p.T_dec, p.T_pru, p.gamma_max, p.mu_max,
                   p.eta_min, p.eta_max, (C.c_double * 3)(*p.p_min), (C.c_double * 3)(*p.p_max),
                   (C.c_double * 3)(*p.v_max), p.zero_mean, p.mvec_scaling, p.regularize,
                   p.birth_proposal, p.N_g)


def _check(lib, h, status, what):
    if status != BP_OK:
        msg = lib.bp_last_error(h)
        raise BPError(status, f"{what}: {msg.decode() if msg else ''}")


def device_array_problem(is_tensor: bool, is_cuda: bool, on_current_device: bool, contiguous: bool, dtype: str,
                         shape: tuple, want_dtypes: tuple, want_floats: int, want_cols: Optional[int] = None
                         ) -> Optional[str]:
    """Why an array cannot be handed to the library as a raw device pointer, or None.
    The library reads exactly want_floats FP32 values from it (a complex64 element is
    two) and cannot check the buffer itself: it must be a contiguous CUDA tensor on the
    current device, of one of want_dtypes, with want_floats values (and want_cols
    columns, for a row-major matrix)."""
    if not is_tensor:
        return "expected a torch tensor"
    if not is_cuda:
        return "expected a CUDA tensor (the library reads device memory)"
    if not on_current_device:
        return "the tensor is on another device than the current one"
    if dtype not in want_dtypes:
        return f"dtype {dtype}, expected one of {', '.join(want_dtypes)}"
    if not contiguous:
        return "expected a contiguous tensor"
    n = 1
    for d in shape:
        n *= int(d)
    floats = 2 * n if dtype == "complex64" else n
    if floats != want_floats:
        return f"{floats} FP32 values, expected {want_floats}"
    if want_cols is not None and (len(shape) != 2 or int(shape[1]) != want_cols):
        return f"shape {tuple(shape)}, expected (rows, {want_cols})"
    return None


def _device_array(t, what: str, want_dtypes: tuple, want_floats: int, want_cols: Optional[int] = None) -> None:
    """Raises BPError(BP_ERR_INVALID_ARG) when device_array_problem finds t unfit."""
    import torch
    is_tensor = isinstance(t, torch.Tensor)
    problem = device_array_problem(
        is_tensor, is_tensor and t.is_cuda,
        is_tensor and t.is_cuda and t.get_device() == torch.cuda.current_device(),
        is_tensor and t.is_contiguous(), str(t.dtype).replace("torch.", "") if is_tensor else "",
        tuple(t.shape) if is_tensor else (), want_dtypes, want_floats, want_cols)
    if problem:
        raise BPError(1, f"{what}: {problem}")


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


class Filter:
    """One particle BP filter on the GPU (handle of the C ABI)."""

    def __init__(self, geom: Geometry, params: Params, P: int, S_max: int, seed: int, stream=None):
        self.lib = load()
        self.geom, self.params, self.P, self.S_max, self.seed = geom, params, P, S_max, seed
        self._g = _GeomHolder(geom)
        self._p = _params_struct(params)
        self.stream = _stream_handle(stream)
        h = C.c_void_p()
        st = self.lib.bp_init(C.byref(self._g.s), C.byref(self._p), P, S_max, C.c_uint64(seed),
                              C.c_void_p(self.stream), C.byref(h))
        _check(self.lib, None, st, "bp_init")
        self.h = h

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.bp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- steps ---------------------------------------------------------------
    def predict(self):
        _check(self.lib, self.h, self.lib.bp_predict(self.h), "bp_predict")

    def update(self, z):
        """z: torch CUDA tensor of J x Nz complex64 (or J x Nz x 2 float32), contiguous."""
        _device_array(z, "bp_update: z", ("complex64", "float32"), 2 * self.geom.J * self.geom.Nz)
        _check(self.lib, self.h, self.lib.bp_update(self.h, C.c_void_p(z.data_ptr())), "bp_update")

    def step(self, z):
        self.predict()
        self.update(z)

    def launch_count(self) -> int:
        return int(self.lib.bp_launch_count(self.h))

    def set_profiling(self, on: bool):
        _check(self.lib, self.h, self.lib.bp_set_profiling(self.h, int(bool(on))), "bp_set_profiling")

    def set_tiles(self, **tiles):
        """Kernel tile requests (bp_set_tiles): any of TILE_FIELDS; fields not given keep
        their value, 0 = built-in."""
        t = self.get_tiles()
        for k, v in tiles.items():
            if k not in TILE_FIELDS:
                raise ValueError(f"unknown tile field {k}")
            t[k] = int(v)
        _check(self.lib, self.h, self.lib.bp_set_tiles(self.h, C.byref(_Tiles(**t))), "bp_set_tiles")

    def get_tiles(self) -> Dict[str, int]:
        t = _Tiles()
        _check(self.lib, self.h, self.lib.bp_get_tiles(self.h, C.byref(t)), "bp_get_tiles")
        return {f: int(getattr(t, f)) for f in TILE_FIELDS}

    def profile(self) -> Dict[str, float]:
        """Durations (ms) of each stage of the last predict and update."""
        ms = np.zeros(len(PROFILE_STAGES))
        _check(self.lib, self.h, self.lib.bp_get_profile(self.h, _dptr(ms), len(ms)), "bp_get_profile")
        return dict(zip(PROFILE_STAGES, ms.tolist()))

    # -- host views --------------------------------------------------------------
    def estimate(self) -> Dict:
        J, SM = self.geom.J, self.S_max
        eta = np.zeros(J); ps = np.zeros(SM); ph = np.zeros((SM, 6)); pr = np.zeros((SM, J))
        dec = np.zeros(SM, np.int32)
        e = _Estimate(0, 0, 0, 0, (C.c_double * 6)(), 0.0, _dptr(eta), _dptr(ps), _dptr(ph), _dptr(pr),
                      dec.ctypes.data_as(C.POINTER(C.c_int)), 0)
        _check(self.lib, self.h, self.lib.bp_estimate(self.h, C.byref(e)), "bp_estimate")
        S = e.S
        return dict(n=e.n, S=S, S_next=e.S_next, births_skipped=e.births_skipped, x_hat=np.array(e.x_hat[:]),
                    ess_x=e.ess_x, eta_hat=eta, p_s=ps[:S].copy(), phi_hat=ph[:S].copy(), p_pr=pr[:S].copy(),
                    declared=dec[:S].astype(bool), iota_repaired=e.iota_repaired)

    def _view(self, S):
        J, P = self.geom.J, self.P
        arrs = dict(x=np.zeros((6, P), np.float32), phi=np.zeros((S, 6, P), np.float32),
                    eta=np.zeros((J, P), np.float32), w_x=np.zeros(P), w_y=np.zeros((S, P)),
                    w_eta=np.zeros((J, P)), p_pr=np.zeros((S, J)))
        return arrs

    def _struct(self, n, S, a, S_legacy=0):
        return _StateView(n, S, S_legacy, _fptr(a["x"]), _fptr(a["phi"]), _fptr(a["eta"]), _dptr(a["w_x"]), _dptr(a["w_y"]),
                          _dptr(a["w_eta"]), _dptr(a["p_pr"]))

    def get_state(self) -> StateArrays:
        a = self._view(self.S_max)
        v = self._struct(0, 0, a)
        _check(self.lib, self.h, self.lib.bp_get_state(self.h, C.byref(v)), "bp_get_state")
        S = v.S
        return StateArrays(n=v.n, S=S, x=a["x"], phi=a["phi"][:S].copy(), eta=a["eta"], w_x=a["w_x"],
                           w_y=a["w_y"][:S].copy(), w_eta=a["w_eta"], p_pr=a["p_pr"][:S].copy())

    def _check_shapes(self, S, shapes):
        if not 1 <= S <= self.S_max:
            raise ValueError(f"S = {S} outside 1 .. S_max = {self.S_max}")
        for name, (arr, want) in shapes.items():
            if tuple(np.shape(arr)) != want:
                raise ValueError(f"{name} has shape {tuple(np.shape(arr))}, expected {want}")

    def set_state(self, st: StateArrays):
        J, P, S = self.geom.J, self.P, int(st.S)
        self._check_shapes(S, dict(x=(st.x, (6, P)), phi=(st.phi, (S, 6, P)), eta=(st.eta, (J, P)),
                                   w_x=(st.w_x, (P,)), w_y=(st.w_y, (S, P)), w_eta=(st.w_eta, (J, P)),
                                   p_pr=(st.p_pr, (S, J))))
        a = dict(x=np.ascontiguousarray(st.x, np.float32), phi=np.ascontiguousarray(st.phi, np.float32),
                 eta=np.ascontiguousarray(st.eta, np.float32), w_x=np.ascontiguousarray(st.w_x, np.float64),
                 w_y=np.ascontiguousarray(st.w_y, np.float64), w_eta=np.ascontiguousarray(st.w_eta, np.float64),
                 p_pr=np.ascontiguousarray(st.p_pr, np.float64))
        v = self._struct(st.n, st.S, a)
        _check(self.lib, self.h, self.lib.bp_set_state(self.h, C.byref(v)), "bp_set_state")

    def save(self, path: str):
        """Checkpoint: the belief state (particles, weights, existences, step index), P,
        S_max, the seed and the geometry's J and Nz to an .npz file.  A filter restored
        with `Filter.load` on the same geometry and parameters continues with the same
        Philox streams (keyed by seed and step).  A learned MT proposal is not part of
        the checkpoint: save() refuses while one is attached (attach it again after
        load, then save the network's parameters with the network)."""
        if getattr(self, "_lp_net", None) is not None:
            raise RuntimeError("save(): a learned MT proposal is attached; it is not part of the checkpoint")
        st = self.get_state()
        np.savez(path, n=st.n, S=st.S, x=st.x, phi=st.phi, eta=st.eta, w_x=st.w_x, w_y=st.w_y, w_eta=st.w_eta,
                 p_pr=st.p_pr, P=self.P, S_max=self.S_max, seed=self.seed, J=self.geom.J, Nz=self.geom.Nz)

    @classmethod
    def load(cls, path: str, geom: Geometry, params: Params, stream=None) -> "Filter":
        """Restores a checkpoint written by `save` into a new filter on the given geometry
        and parameters (those the checkpoint was taken with)."""
        d = np.load(path)
        if "J" not in d or int(d["J"]) != geom.J or int(d["Nz"]) != geom.Nz:
            raise ValueError(f"checkpoint {path} was taken on another geometry "
                             f"(J, Nz = {d.get('J')}, {d.get('Nz')}; here {geom.J}, {geom.Nz})")
        f = cls(geom, params, P=int(d["P"]), S_max=int(d["S_max"]), seed=int(d["seed"]), stream=stream)
        f.set_state(StateArrays(n=int(d["n"]), S=int(d["S"]), x=d["x"], phi=d["phi"], eta=d["eta"], w_x=d["w_x"],
                                w_y=d["w_y"], w_eta=d["w_eta"], p_pr=d["p_pr"]))
        return f

    def get_predicted(self) -> Dict:
        a = self._view(self.S_max)
        v = self._struct(0, 0, a)
        _check(self.lib, self.h, self.lib.bp_get_predicted(self.h, C.byref(v)), "bp_get_predicted")
        S = v.S
        return dict(n=v.n, S=S, S_legacy=v.S_legacy, x=a["x"], phi=a["phi"][:S].copy(), eta=a["eta"], w_beta=a["w_x"],
                    w_alpha=a["w_y"][:S].copy(), w_xi=a["w_eta"], zeta=a["p_pr"][:S].copy())

    def set_predicted(self, n, S, x, phi, eta, w_beta, w_alpha, w_xi, zeta, S_legacy=None):
        """S_legacy: PFs before this step's births (slots S_legacy .. S-1 are new and are
        drawn from the birth proposal in the update when it is enabled); None = no new PF."""
        a = dict(x=np.ascontiguousarray(x, np.float32), phi=np.ascontiguousarray(phi, np.float32),
                 eta=np.ascontiguousarray(eta, np.float32), w_x=np.ascontiguousarray(w_beta, np.float64),
                 w_y=np.ascontiguousarray(w_alpha, np.float64), w_eta=np.ascontiguousarray(w_xi, np.float64),
                 p_pr=np.ascontiguousarray(zeta, np.float64))
        v = self._struct(n, S, a, S if S_legacy is None else S_legacy)
        _check(self.lib, self.h, self.lib.bp_set_predicted(self.h, C.byref(v)), "bp_set_predicted")

    def _diag(self, what, nbytes, dtype):
        buf = np.zeros(nbytes // np.dtype(dtype).itemsize, dtype)
        _check(self.lib, self.h, self.lib.bp_get_diag(self.h, what, buf.ctypes.data_as(C.c_void_p), nbytes),
               "bp_get_diag")
        return buf

    def diag_table(self, S) -> Dict:
        J, Nz = self.geom.J, self.geom.Nz
        n = 4 * S * J * Nz * 2 + S + J
        b = self._diag(DIAG_TABLE, n * 8, np.float64)
        t = b[:4 * S * J * Nz * 2].reshape(4, S, J, Nz, 2)
        t = t[..., 0] + 1j * t[..., 1]
        o = 4 * S * J * Nz * 2
        return dict(m=t[0], mw=t[1], mu3=t[2], mu4=t[3], W=b[o:o + S], eta_bar=b[o + S:o + S + J])

    def diag_weights(self, S) -> Dict:
        J, P = self.geom.J, self.P
        n = P + S * P + J * P + S + S * J
        b = self._diag(DIAG_WEIGHTS, n * 8, np.float64)
        o = 0
        w_x = b[o:o + P]; o += P
        w_y = b[o:o + S * P].reshape(S, P); o += S * P
        w_eta = b[o:o + J * P].reshape(J, P); o += J * P
        p_s = b[o:o + S]; o += S
        p_pr = b[o:o + S * J].reshape(S, J)
        return dict(w_x=w_x, w_y=w_y, w_eta=w_eta, p_s=p_s, p_pr=p_pr)

    def diag_loglik(self, S) -> Dict:
        J, P = self.geom.J, self.P
        n = P + S * P + J * P + S * J
        b = self._diag(DIAG_LOGLIK, n * 8, np.float64)
        o = 0
        li = b[o:o + P]; o += P
        lk = b[o:o + S * P].reshape(S, P); o += S * P
        ln = b[o:o + J * P].reshape(J, P); o += J * P
        lw = b[o:o + S * J].reshape(S, J)
        return dict(log_iota=li, delta_kappa=lk, log_nu=ln, llr_omega=lw)

    def diag_iota(self) -> Dict:
        """The particles whose log iota was evaluated in float-float in the last update
        (S >= 24) and the error bound of every particle's FP32 value (nats)."""
        P = self.P
        b = self._diag(DIAG_IOTA, (P + 1) * 4 + P * 4, np.uint8)
        fl = np.frombuffer(b[:(P + 1) * 4].tobytes(), np.int32)
        err = np.frombuffer(b[(P + 1) * 4:].tobytes(), np.float32)
        return dict(selected=np.sort(fl[1:1 + fl[0]]), err=err.copy())

    def set_mt_proposal(self, net):
        """Attach a proposal network (Mlp) to this filter, or detach it (None)."""
        self._lp_net = net
        _check(self.lib, self.h, self.lib.bp_set_mt_proposal(self.h, net.h if net is not None else None),
               "bp_set_mt_proposal")

    def diag_lproposal(self) -> Dict:
        """The learned MT proposal of the last update: predicted mean, per-PA correlations,
        log importance ratios, network inputs and outputs."""
        J, P = self.geom.J, self.P
        nd = 6 + 4 * J + P
        nbytes = nd * 8 + 2 * P * 16 * 4
        buf = np.zeros(nbytes, np.uint8)
        _check(self.lib, self.h, self.lib.bp_get_diag(self.h, DIAG_LPROP, buf.ctypes.data_as(C.c_void_p), nbytes),
               "bp_get_diag")
        d = buf[:nd * 8].view(np.float64)
        f = buf[nd * 8:].view(np.float32)
        return dict(xbar=d[:6].copy(), cor=d[6:6 + 4 * J].reshape(J, 4).copy(), logr=d[6 + 4 * J:].copy(),
                    X=f[:P * 16].reshape(P, 16).copy(), Y=f[P * 16:].reshape(P, 16).copy())

    def diag_proposal(self, Qe: int) -> Dict:
        """Birth proposal of the last update's Qe new PFs: statistics, Bartlett costs,
        candidates, prediction weights and particle positions."""
        P, Ng = self.P, self.params.N_g
        nd = Qe * (32 + Ng + 3 * Ng + P)
        nbytes = nd * 8 + Qe * 3 * P * 4
        buf = np.zeros(nbytes, np.uint8)
        _check(self.lib, self.h, self.lib.bp_get_diag(self.h, DIAG_PROPOSAL, buf.ctypes.data_as(C.c_void_p), nbytes),
               "bp_get_diag")
        d = buf[:nd * 8].view(np.float64)
        o = 0
        st = d[o:o + 32 * Qe].reshape(Qe, 32); o += 32 * Qe
        costs = d[o:o + Qe * Ng].reshape(Qe, Ng); o += Qe * Ng
        cand = d[o:o + 3 * Qe * Ng].reshape(Qe, Ng, 3); o += 3 * Qe * Ng
        w_alpha = d[o:o + Qe * P].reshape(Qe, P)
        pos = buf[nd * 8:].view(np.float32).reshape(Qe, 3, P)
        return dict(valid=st[:, 0] != 0, i_star=st[:, 1].astype(int), cost_sum=st[:, 2], mu=st[:, 3:6],
                    C=st[:, 6:15].reshape(Qe, 3, 3), L=st[:, 15:24].reshape(Qe, 3, 3), costs=costs, cand=cand,
                    w_alpha=w_alpha, pos=pos)

    def diag_indices(self, S) -> Dict:
        J, P = self.geom.J, self.P
        n = P + S * P + J * P
        b = self._diag(DIAG_INDICES, n * 4, np.int32)
        return dict(x=b[:P], y=b[P:P + S * P].reshape(S, P), eta=b[P + S * P:].reshape(J, P))


class _BatchMember(Filter):
    """View of one scenario of a Batch: the single-handle calls (estimate, state
    export/import, launch count); the handle belongs to the batch."""

    def __init__(self, batch, i, h, geom, params, P, S_max):
        self.lib, self.h, self.geom, self.params, self.P, self.S_max = batch.lib, h, geom, params, P, S_max
        self._batch = batch   # keeps the batch (and the handle) alive
        self._i = i

    def close(self):
        self.h = None

    def set_tiles(self, **tiles):
        """Through the batch, which drops its captured graphs."""
        self._batch.set_tiles(self._i, **tiles)

    def predict(self):
        raise BPError(6, "a batch scenario steps through Batch.step")

    update = step = predict


class Batch:
    """Many independent filters stepped together (bp_batch_*): scenarios dealt over
    concurrent streams, shared per-stream workspaces, CUDA-graph replay."""

    def __init__(self, scenarios, n_streams: int = 32, shared_workspace: bool = True, use_graph: bool = True,
                 stream=None):
        """scenarios: list of (geom, params, P, S_max, S0, seed); stream: the fork/join stream
        (a torch.cuda.Stream or a raw handle; None = the current torch stream)."""
        self.lib = load()
        self.scen = list(scenarios)
        n = len(self.scen)
        self._g = [_GeomHolder(sc[0]) for sc in self.scen]
        self._p = [_params_struct(sc[1]) for sc in self.scen]
        arr = (_Scenario * n)()
        for i, (g, p, P, S_max, S0, seed) in enumerate(self.scen):
            arr[i] = _Scenario(C.pointer(self._g[i].s), C.pointer(self._p[i]), P, S_max, S0, C.c_uint64(seed))
        self._arr = arr
        self.stream = _stream_handle(stream)
        opts = _BatchOpts(n_streams, int(bool(shared_workspace)), int(bool(use_graph)), C.c_void_p(self.stream))
        b = C.c_void_p()
        st = self.lib.bp_batch_init(arr, n, C.byref(opts), C.byref(b))
        if st != BP_OK:
            msg = self.lib.bp_batch_last_error(None)
            raise BPError(st, f"bp_batch_init: {msg.decode() if msg else ''}")
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            self.lib.bp_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != BP_OK:
            msg = self.lib.bp_batch_last_error(self.b)
            raise BPError(st, f"{what}: {msg.decode() if msg else ''}")

    def __len__(self):
        return len(self.scen)

    def z_offset(self, i: int) -> int:
        return int(self.lib.bp_batch_z_offset(self.b, i))

    def z_floats(self) -> int:
        return int(self.lib.bp_batch_z_floats(self.b))

    def step(self, z):
        """z: torch CUDA float32 tensor of z_floats() values (the scenarios' J x Nz complex
        observations concatenated in scenario order)."""
        _device_array(z, "bp_batch_step: z", ("float32", "complex64"), self.z_floats())
        self._check(self.lib.bp_batch_step(self.b, C.c_void_p(z.data_ptr())), "bp_batch_step")

    def sync(self):
        self._check(self.lib.bp_batch_sync(self.b), "bp_batch_sync")

    def stream_of(self, i: int) -> int:
        return int(self.lib.bp_batch_stream_of(self.b, i))

    def device_bytes(self) -> int:
        return int(self.lib.bp_batch_device_bytes(self.b))

    def set_tiles(self, i: int, **tiles):
        """bp_batch_set_tiles on scenario i (fields not given keep their value)."""
        t = self.member(i).get_tiles()
        for k, v in tiles.items():
            if k not in TILE_FIELDS:
                raise ValueError(f"unknown tile field {k}")
            t[k] = int(v)
        self._check(self.lib.bp_batch_set_tiles(self.b, i, C.byref(_Tiles(**t))), "bp_batch_set_tiles")

    def member(self, i: int) -> Filter:
        h = C.c_void_p()
        self._check(self.lib.bp_batch_handle(self.b, i, C.byref(h)), "bp_batch_handle")
        g, p, P, S_max, _, _ = self.scen[i]
        return _BatchMember(self, i, h, g, p, P, S_max)


def pcrlb_dim(K: int, J: int, coherent: bool) -> int:
    return 6 + 3 * K + ((K + 1) if coherent else (K + 1) * J) + (K + 1) * J + 1


def pcrlb_fim(geom: Geometry, x, sfv, rho, eta: float, coherent: bool, stream=None) -> np.ndarray:
    """Bayesian snapshot FIM (bp_pcrlb_fim): mean over the M realisations in x (M, 6),
    sfv (M, K, 3), rho (M, J, K+1) complex."""
    lib = load()
    g = _GeomHolder(geom)
    x = np.ascontiguousarray(np.atleast_2d(x), np.float64)
    M = x.shape[0]
    sfv = np.ascontiguousarray(np.asarray(sfv, np.float64).reshape(M, -1, 3), np.float64)
    K = sfv.shape[1]
    rho = np.asarray(rho).reshape(M, geom.J, K + 1)
    rr = np.ascontiguousarray(np.stack([rho.real, rho.imag], -1), np.float64)
    d = pcrlb_dim(K, geom.J, coherent)
    out = np.zeros((d, d))
    st = lib.bp_pcrlb_fim(C.byref(g.s), K, int(bool(coherent)), M, _dptr(x), _dptr(sfv) if K else None, _dptr(rr),
                          float(eta), _dptr(out), C.c_void_p(_stream_handle(stream)))
    _check(lib, None, st, "bp_pcrlb_fim")
    return out


def pcrlb_recursion(F, Q, J10, Jsnap, K: int, stream=None):
    """PEB (N,) and MEB (N, K) of the recursion (bp_pcrlb_recursion)."""
    lib = load()
    F, Q, J10 = (np.ascontiguousarray(a, np.float64) for a in (F, Q, J10))
    Js = np.ascontiguousarray(np.asarray(Jsnap, np.float64))
    N, d = Js.shape[0], F.shape[0]
    peb = np.zeros(N)
    meb = np.zeros((N, max(K, 1)))
    st = lib.bp_pcrlb_recursion(d, N, K, _dptr(F), _dptr(Q), _dptr(J10), _dptr(Js), _dptr(peb), _dptr(meb),
                                C.c_void_p(_stream_handle(stream)))
    _check(lib, None, st, "bp_pcrlb_recursion")
    return peb, meb[:, :K]


MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_NPARAM = 16, 64, 16, 6288


class Mlp:
    """The proposal network on the GPU (bp_mlp_*): BF16 tensor-core forward, backward
    and Adam.  X (B x 16), T (B x 3) are torch CUDA float32 tensors."""

    def __init__(self, params: np.ndarray, stream=None):
        self.lib = load()
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == MLP_NPARAM
        h = C.c_void_p()
        st = self.lib.bp_mlp_create(_fptr(p), C.c_void_p(_stream_handle(stream)), C.byref(h))
        self._check(st, "bp_mlp_create", None)
        self.h = h

    def _check(self, st, what, h="self"):
        if st != BP_OK:
            hh = self.h if h == "self" else h
            msg = self.lib.bp_mlp_last_error(hh) if hh else b""
            raise BPError(st, f"{what}: {msg.decode() if msg else ''}")

    def params(self) -> np.ndarray:
        out = np.zeros(MLP_NPARAM, np.float32)
        self._check(self.lib.bp_mlp_get_params(self.h, _fptr(out)), "bp_mlp_get_params")
        return out

    def forward(self, X):
        import torch
        X = X.contiguous()
        _device_array(X, "bp_mlp_forward: X", ("float32",), X.numel(), MLP_IN)
        Y = torch.empty((X.shape[0], MLP_OUT), dtype=torch.float32, device=X.device)
        self._check(self.lib.bp_mlp_forward(self.h, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(Y.data_ptr())),
                    "bp_mlp_forward")
        return Y

    def grads(self, X, T):
        """(gradient of the mean loss, summed loss) without changing the parameters."""
        import torch
        X, T = X.contiguous(), T.contiguous()
        _device_array(X, "bp_mlp_grads: X", ("float32",), X.numel(), MLP_IN)
        _device_array(T, "bp_mlp_grads: T", ("float32",), 3 * X.shape[0], 3)
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=X.device)
        l = torch.empty(1, dtype=torch.float32, device=X.device)
        self._check(self.lib.bp_mlp_grads(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), X.shape[0],
                                          C.c_void_p(g.data_ptr()), C.c_void_p(l.data_ptr())), "bp_mlp_grads")
        return g.cpu().numpy(), float(l.item())

    def train_step(self, X, T, lr: float, loss_out=None):
        _device_array(X, "bp_mlp_train_step: X", ("float32",), X.numel() if hasattr(X, "numel") else -1, MLP_IN)
        _device_array(T, "bp_mlp_train_step: T", ("float32",), 3 * X.shape[0], 3)
        if loss_out is not None:
            _device_array(loss_out, "bp_mlp_train_step: loss_out", ("float32",), 1)
        self._check(self.lib.bp_mlp_train_step(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                               X.shape[0], C.c_float(lr),
                                               C.c_void_p(loss_out.data_ptr() if loss_out is not None else None)),
                    "bp_mlp_train_step")

    def sync(self):
        self._check(self.lib.bp_mlp_sync(self.h), "bp_mlp_sync")

    def close(self):
        if getattr(self, "h", None):
            self.lib.bp_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_wait(limit: int = 4096, stream=None) -> int:
    """bp_selftest_wait: the status of a bounded wait on a phase nothing completes
    (BP_ERR_TIMEOUT expected)."""
    lib = load()
    return int(lib.bp_selftest_wait(int(limit), C.c_void_p(_stream_handle(stream))))


NOALLOC_MAX_P = 1 << 20


def resample_noalloc(w, seed: int, n: int, kind: int, index: int, out=None, stream=None):
    """Systematic resampling through bp_resample_noalloc (no device allocation inside
    the library).  w: torch CUDA float64 tensor of P weights; returns int32 indices."""
    import torch
    if not (isinstance(w, torch.Tensor) and w.is_cuda and w.dtype == torch.float64 and w.dim() == 1
            and w.is_contiguous()):
        raise TypeError("resample_noalloc: w must be a 1-D contiguous CUDA float64 tensor")
    lib = load()
    P = int(w.numel())
    if out is None:
        out = torch.empty(P, dtype=torch.int32, device=w.device)
    elif not (isinstance(out, torch.Tensor) and out.device == w.device and out.dtype == torch.int32
              and out.is_contiguous() and out.numel() >= P):
        raise TypeError("resample_noalloc: out must be a contiguous int32 tensor of >= P elements on w's device")
    with torch.cuda.device(w.device):
        st = lib.bp_resample_noalloc(C.c_void_p(w.data_ptr()), P, C.c_uint64(seed), n, kind, index,
                                     C.c_void_p(out.data_ptr()), C.c_void_p(_stream_handle(stream)))
    if st != BP_OK:
        raise BPError(st, "bp_resample_noalloc" + (f": P = {P} exceeds {NOALLOC_MAX_P}" if st == 3 else ""))
    return out


def lp_dataset(geom: Geometry, params: Params, sfv: np.ndarray, rho_abs: np.ndarray, eta: float, n: int, seed: int,
               err_pos: float = 0.002, err_vel: float = 0.02, spread_pos: float = 0.003, spread_vel: float = 0.03,
               coherent: bool = True, stream=None):
    """Training samples of the proposal network (bp_lp_dataset): torch CUDA tensors
    X (n x 16) and T (n x 3); coherent: amplitude phases common to all PAs, else per PA."""
    import torch
    lib = load()
    g = _GeomHolder(geom)
    pr = _params_struct(params)
    sf = np.ascontiguousarray(np.asarray(sfv, np.float64).reshape(-1, 3))
    ra = np.ascontiguousarray(np.asarray(rho_abs, np.float64))
    X = torch.empty((n, MLP_IN), dtype=torch.float32, device="cuda")
    T = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    st = lib.bp_lp_dataset(C.byref(g.s), C.byref(pr), sf.shape[0], _dptr(sf) if sf.size else None, _dptr(ra),
                           float(eta), int(bool(coherent)), err_pos, err_vel, spread_pos, spread_vel, int(n),
                           C.c_uint64(seed),
                           C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), C.c_void_p(_stream_handle(stream)))
    _check(lib, None, st, "bp_lp_dataset")
    return X, T


def synthesize(geom: Geometry, x_pos: np.ndarray, sfv: np.ndarray, rho: np.ndarray,
               clutter_count=None, clutter_sfv=None, clutter_rho=None, snr_db: float = 20.0,
               seed: int = 0, step0: int = 1, out=None, stream=None):
    """Synthetic observations on the GPU (bp_synthesize).  x_pos (T, 3), sfv (K, 3),
    rho (T, J, K+1) complex.  Returns (z as a torch CUDA tensor (T, J, Nz) complex64, eta)."""
    import torch
    lib = load()
    g = _GeomHolder(geom)
    T = x_pos.shape[0]
    K = sfv.shape[0]
    xp = np.ascontiguousarray(x_pos, np.float64)
    sf = np.ascontiguousarray(sfv, np.float64).reshape(-1) if K else np.zeros(3)
    rh = np.ascontiguousarray(np.stack([np.real(rho), np.imag(rho)], -1), np.float64)
    cc = np.ascontiguousarray(np.zeros(T, np.int32) if clutter_count is None else clutter_count, np.int32)
    cs = np.ascontiguousarray(np.zeros((1, 3)) if clutter_sfv is None or len(clutter_sfv) == 0 else clutter_sfv, np.float64)
    cr_ = np.zeros((1, geom.J), complex) if clutter_rho is None or len(clutter_rho) == 0 else clutter_rho
    cr = np.ascontiguousarray(np.stack([np.real(cr_), np.imag(cr_)], -1), np.float64)
    if out is None:
        out = torch.empty((T, geom.J, geom.Nz), dtype=torch.complex64, device="cuda")
    eta = C.c_double()
    st = lib.bp_synthesize(C.byref(g.s), T, step0, _dptr(xp), K, _dptr(sf), _dptr(rh),
                           cc.ctypes.data_as(C.POINTER(C.c_int)), _dptr(cs), _dptr(cr), snr_db, C.c_uint64(seed),
                           C.c_void_p(out.data_ptr()), C.byref(eta), C.c_void_p(_stream_handle(stream)))
    _check(lib, None, st, "bp_synthesize")
    return out, eta.value


def scenario_arrays(scn, steps):
    """Arrays of bp_synthesize for the given scenario steps (visibility folded into rho)."""
    steps = list(steps)
    J = scn.geom.J
    K = scn.sfv_true.shape[0]
    x_pos = np.stack([scn.x_true[n, :3] for n in steps])
    rho = np.zeros((len(steps), J, K + 1), complex)
    for t, n in enumerate(steps):
        rho[t] = scn.rho_abs[None, :] * np.exp(1j * scn.rho_phase[n]) * scn.visible[n]
    cc = np.array([scn.clutter_sfv[n].shape[0] for n in steps], np.int32)
    cs = np.concatenate([scn.clutter_sfv[n] for n in steps]) if cc.sum() else np.zeros((0, 3))
    cr = np.concatenate([scn.clutter_rho[n] for n in steps]) if cc.sum() else np.zeros((0, J), complex)
    return x_pos, scn.sfv_true, rho, cc, cs, cr
