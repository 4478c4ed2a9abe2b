"""FP64 CPU oracle for the ImaSk hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does; the two share no code.

``build()`` compiles ``imask_oracle.c`` with gcc into ``liboracle.so`` beside
it; ``Oracle`` wraps the C functions with numpy arrays (float64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "imask_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, no FMA contraction) and return its path."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "imask_oracle.h")))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(
                ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                 "-o", tmp, _SRC, "-lm"], check=True)
            os.replace(tmp, _LIB)
    return _LIB


class OrcDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("n_angles", ctypes.c_int32), ("n_det", ctypes.c_int32),
        ("geometry", ctypes.c_int32),
        ("fov", ctypes.c_double), ("det_spacing", ctypes.c_double),
        ("angle_start", ctypes.c_double), ("angle_span", ctypes.c_double),
        ("src_dist", ctypes.c_double), ("det_dist", ctypes.c_double),
        ("levels", ctypes.c_int32), ("probs", ctypes.POINTER(ctypes.c_double)),
        ("reg", ctypes.c_int32), ("mu", ctypes.c_double), ("tv_lambda", ctypes.c_double),
        ("tv_eps", ctypes.c_double), ("tv_inner", ctypes.c_int32), ("sigma", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class OrcVariant(ctypes.Structure):
    _fields_ = [("sequential", ctypes.c_int32), ("theta", ctypes.c_double),
                ("snapshots", ctypes.c_int32), ("independent", ctypes.c_int32),
                ("storage", ctypes.c_int32)]


class Oracle:
    """numpy front end of the C oracle for one problem description.

    ``params`` holds the geometry and solver fields of the problem (the same
    keys as the CUDA library's descriptor: n, n_angles, n_det, geometry, fov,
    det_spacing, angle_start, angle_span, src_dist, det_dist, levels, probs,
    reg, mu, tv_lambda, tv_eps, tv_inner, sigma); reg 2 is TV with a
    nonnegativity constraint.
    """

    _lib = None

    @classmethod
    def lib(cls):
        if cls._lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "orc_splitmix64_at": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
                "orc_level_thresholds": (None, [ctypes.c_void_p, _U64]),
                "orc_level": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]),
                "orc_levels": (None, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_int64, _I32]),
                "orc_det_spacing": (ctypes.c_double, [ctypes.c_void_p]),
                "orc_ray": (None, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, _D, _D]),
                "orc_ray_is_xmajor": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32,
                                                       ctypes.c_int32]),
                "orc_joseph_ray": (ctypes.c_double, [ctypes.c_void_p, ctypes.c_int32, _D,
                                                     ctypes.c_int32, ctypes.c_int32]),
                "orc_joseph_fp": (None, [ctypes.c_void_p, ctypes.c_int32, _D, _D]),
                "orc_joseph_bp": (None, [ctypes.c_void_p, ctypes.c_int32, _D, _D]),
                "orc_block_mean": (None, [ctypes.c_int32, ctypes.c_int32, _D, _D]),
                "orc_replicate": (None, [ctypes.c_int32, ctypes.c_int32, _D, _D]),
                "orc_compensate": (None, [ctypes.c_void_p, _D, _D]),
                "orc_apply_K": (None, [ctypes.c_void_p, ctypes.c_int32, _D, _D]),
                "orc_apply_KT": (None, [ctypes.c_void_p, ctypes.c_int32, _D, _D]),
                "orc_prox": (None, [ctypes.c_void_p, ctypes.c_double, _D, _D]),
                "orc_regulariser": (ctypes.c_double, [ctypes.c_void_p, _D]),
                "orc_imask_run": (ctypes.c_int32, [ctypes.c_void_p, _D, ctypes.c_uint64,
                                                   ctypes.c_int64, ctypes.c_int32, _D, _D, _D,
                                                   _D, _I32]),
                "orc_imask_seq_run": (ctypes.c_int32, [ctypes.c_void_p, _D, ctypes.c_uint64,
                                                       ctypes.c_int64, ctypes.c_int32,
                                                       ctypes.c_double, _D, _D, _D, _D, _D,
                                                       _I32]),
                "orc_primal_seed": (ctypes.c_uint64, [ctypes.c_uint64]),
                "orc_round_format": (ctypes.c_double, [ctypes.c_double, ctypes.c_int32,
                                                       ctypes.c_int32]),
                "orc_imask_variant_run": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, _D,
                                                           ctypes.c_uint64, ctypes.c_int64,
                                                           ctypes.c_int32] + [_D] * 7
                                          + [_I32, _I32]),
                "orc_pdhg_params": (None, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           _D]),
                "orc_pdhg_run": (ctypes.c_int32, [ctypes.c_void_p, _D, ctypes.c_int32,
                                                  ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, _D, _D, _D]),
                "orc_power_eig": (ctypes.c_double, [ctypes.c_void_p, _D, ctypes.c_int32,
                                                    ctypes.c_int32, ctypes.c_int32]),
                "orc_constants_dense": (None, [_D, ctypes.c_int32, _D, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                               _D]),
                "orc_constants": (None, [ctypes.c_void_p, ctypes.c_int32, _D]),
                "orc_norm_K": (ctypes.c_double, [ctypes.c_void_p, ctypes.c_int32]),
                "orc_theta": (ctypes.c_double, [ctypes.c_double] * 7),
                "orc_eta_opt": (ctypes.c_double, [ctypes.c_double] * 6),
                "orc_optimal_step": (None, [ctypes.c_double] * 4 + [ctypes.c_int32, _D]),
                "orc_solve_quadratic": (ctypes.c_int32, [ctypes.c_void_p, _D, ctypes.c_int32,
                                                         ctypes.c_double, _D]),
                "orc_objective": (ctypes.c_double, [ctypes.c_void_p, _D, _D]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            cls._lib = lib
        return cls._lib

    def __init__(self, **params):
        self.p = dict(params)
        self.L = self.lib()
        self._probs = None
        self._desc = OrcDesc()
        self.set(**params)

    # -- descriptor -----------------------------------------------------------------
    def set(self, **params):
        self.p.update(params)
        p = self.p
        d = self._desc
        d.n = int(p["n"])
        d.n_angles = int(p["n_angles"])
        d.n_det = int(p["n_det"])
        d.geometry = int(p.get("geometry", 0))
        d.fov = float(p.get("fov", 1.0))
        d.det_spacing = float(p.get("det_spacing", 0.0))
        d.angle_start = float(p.get("angle_start", 0.0))
        d.angle_span = float(p.get("angle_span", np.pi))
        d.src_dist = float(p.get("src_dist", 2.0))
        d.det_dist = float(p.get("det_dist", 1.0))
        d.levels = int(p.get("levels", 1))
        probs = p.get("probs")
        if probs is None:
            self._probs = None
            d.probs = ctypes.cast(None, _D)
        else:
            self._probs = np.ascontiguousarray(probs, dtype=np.float64)
            d.probs = _dp(self._probs)
        d.reg = int(p.get("reg", 0))
        d.mu = float(p.get("mu", 1.0))
        d.tv_lambda = float(p.get("tv_lambda", 0.0))
        d.tv_eps = float(p.get("tv_eps", 1e-2))
        d.tv_inner = int(p.get("tv_inner", 20))
        d.sigma = float(p.get("sigma", 0.0))
        return self

    @property
    def ref(self):
        return ctypes.byref(self._desc)

    @property
    def n(self):
        return self._desc.n

    @property
    def m(self):
        return self._desc.n_angles * self._desc.n_det

    @property
    def r(self):
        return max(1, self._desc.levels)

    def probs(self):
        if self._probs is not None:
            return self._probs.copy()
        return np.full(self.r, 1.0 / self.r)

    # -- level draw -----------------------------------------------------------------
    def splitmix64_at(self, seed: int, k: int) -> int:
        return int(self.L.orc_splitmix64_at(seed, k))

    def thresholds(self) -> np.ndarray:
        t = np.zeros(max(1, self.r - 1), dtype=np.uint64)
        self.L.orc_level_thresholds(self.ref, t.ctypes.data_as(_U64))
        return t[: self.r - 1]

    def levels(self, seed: int, k0: int, n: int) -> np.ndarray:
        out = np.zeros(n, dtype=np.int32)
        self.L.orc_levels(self.ref, seed, k0, n, out.ctypes.data_as(_I32))
        return out

    # -- geometry / projector -------------------------------------------------------
    def det_spacing(self) -> float:
        return float(self.L.orc_det_spacing(self.ref))

    def ray(self, a: int, j: int):
        p0 = np.zeros(2)
        d = np.zeros(2)
        self.L.orc_ray(self.ref, a, j, _dp(p0), _dp(d))
        return p0, d

    def xmajor_table(self) -> np.ndarray:
        d = self._desc
        out = np.zeros((d.n_angles, d.n_det), dtype=np.int32)
        for a in range(d.n_angles):
            for j in range(d.n_det):
                out[a, j] = self.L.orc_ray_is_xmajor(self.ref, a, j)
        return out

    def joseph_ray(self, nl: int, img: np.ndarray, a: int, j: int) -> float:
        img = np.ascontiguousarray(img, dtype=np.float64)
        return float(self.L.orc_joseph_ray(self.ref, nl, _dp(img), a, j))

    def joseph_fp(self, img: np.ndarray) -> np.ndarray:
        img = np.ascontiguousarray(img, dtype=np.float64)
        nl = img.shape[0]
        out = np.zeros((self._desc.n_angles, self._desc.n_det))
        self.L.orc_joseph_fp(self.ref, nl, _dp(img), _dp(out))
        return out

    def joseph_bp(self, sino: np.ndarray, nl: int) -> np.ndarray:
        sino = np.ascontiguousarray(sino, dtype=np.float64)
        out = np.zeros((nl, nl))
        self.L.orc_joseph_bp(self.ref, nl, _dp(sino), _dp(out))
        return out

    # -- sketches -------------------------------------------------------------------
    def block_mean(self, x: np.ndarray, ell: int) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = x.shape[0]
        out = np.zeros((n >> ell, n >> ell))
        self.L.orc_block_mean(n, ell, _dp(x), _dp(out))
        return out

    def replicate(self, c: np.ndarray, ell: int) -> np.ndarray:
        c = np.ascontiguousarray(c, dtype=np.float64)
        n = c.shape[0] << ell
        out = np.zeros((n, n))
        self.L.orc_replicate(n, ell, _dp(c), _dp(out))
        return out

    def compensate(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        self.L.orc_compensate(self.ref, _dp(x), _dp(out))
        return out

    def K(self, ell: int, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.n, self.n)
        out = np.zeros((self._desc.n_angles, self._desc.n_det))
        self.L.orc_apply_K(self.ref, ell, _dp(x), _dp(out))
        return out

    def KT(self, ell: int, y: np.ndarray) -> np.ndarray:
        y = np.ascontiguousarray(y, dtype=np.float64).reshape(self._desc.n_angles,
                                                              self._desc.n_det)
        out = np.zeros((self.n, self.n))
        self.L.orc_apply_KT(self.ref, ell, _dp(y), _dp(out))
        return out

    # -- prox / iteration -----------------------------------------------------------
    def prox(self, tau: float, v: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(self.n, self.n)
        out = np.zeros_like(v)
        self.L.orc_prox(self.ref, tau, _dp(v), _dp(out))
        return out

    def regulariser(self, x: np.ndarray) -> float:
        x = np.ascontiguousarray(x, dtype=np.float64)
        return float(self.L.orc_regulariser(self.ref, _dp(x)))

    def new_state(self):
        n, m, r = self.n, self.m, self.r
        return {"x": np.zeros(n * n), "y": np.zeros(m), "phi": np.zeros(r * n * n),
                "psi": np.zeros(r * m), "k": 0}

    def run(self, b: np.ndarray, seed: int, iters: int, state=None):
        """Alg. 1 for ``iters`` iterations from ``state`` (default: zeros).

        Returns (state, levels); the state dict is updated in place."""
        if state is None:
            state = self.new_state()
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        lv = np.zeros(max(1, iters), dtype=np.int32)
        rc = self.L.orc_imask_run(self.ref, _dp(b), seed, state["k"], iters, _dp(state["x"]),
                                  _dp(state["y"]), _dp(state["phi"]), _dp(state["psi"]),
                                  lv.ctypes.data_as(_I32))
        if rc != 0:
            raise ValueError("oracle: sigma and mu must be positive")
        state["k"] += iters
        return state, lv[:iters]

    def run_seq(self, b: np.ndarray, seed: int, iters: int, theta: float = 1.0, state=None):
        """Alg. 7 (ImaSk-Seq) for ``iters`` iterations; the state gains ``xbar``."""
        if state is None:
            state = self.new_state()
        state.setdefault("xbar", np.zeros(self.n * self.n))
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        lv = np.zeros(max(1, iters), dtype=np.int32)
        rc = self.L.orc_imask_seq_run(self.ref, _dp(b), seed, state["k"], iters, theta,
                                      _dp(state["x"]), _dp(state["xbar"]), _dp(state["y"]),
                                      _dp(state["phi"]), _dp(state["psi"]),
                                      lv.ctypes.data_as(_I32))
        if rc != 0:
            raise ValueError("oracle: sigma and mu must be positive")
        state["k"] += iters
        return state, lv[:iters]

    @classmethod
    def round_format(cls, v: float, fmt: int) -> float:
        """bfloat16 (fmt 1) or binary16 (fmt 2) rounding of v, RNE."""
        bits, emin = (8, -126) if fmt == 1 else (11, -14)
        return float(cls.lib().orc_round_format(float(v), bits, emin))

    def primal_seed(self, seed: int) -> int:
        return int(self.L.orc_primal_seed(seed))

    def new_variant_state(self, snapshots: bool):
        n, m, r = self.n, self.m, self.r
        d = n * n
        st = {"x": np.zeros(d), "xbar": np.zeros(d), "y": np.zeros(m),
              "phi": np.zeros(r * d), "k": 0}
        if snapshots:
            st["snap"] = np.zeros(r * d)
            st["psi_mean"] = np.zeros(m)
        else:
            st["psi"] = np.zeros(r * m)
        return st

    def run_variant(self, b: np.ndarray, seed: int, iters: int, sequential=False, theta=1.0,
                    snapshots=False, independent=False, storage=0, state=None):
        """Alg. 1 / Alg. 7 with the snapshot tables and independent-draw options.

        Returns (state, dual levels, primal levels)."""
        if state is None:
            state = self.new_variant_state(snapshots)
        var = OrcVariant(int(bool(sequential)), float(theta), int(bool(snapshots)),
                         int(bool(independent)), int(storage))
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        ld = np.zeros(max(1, iters), dtype=np.int32)
        lp = np.zeros(max(1, iters), dtype=np.int32)
        null = ctypes.cast(None, _D)

        def opt(key):
            return _dp(state[key]) if key in state else null

        rc = self.L.orc_imask_variant_run(
            self.ref, ctypes.byref(var), _dp(b), seed, state["k"], iters, _dp(state["x"]),
            opt("xbar"), _dp(state["y"]), _dp(state["phi"]), opt("psi"), opt("snap"),
            opt("psi_mean"), ld.ctypes.data_as(_I32), lp.ctypes.data_as(_I32))
        if rc != 0:
            raise ValueError(f"oracle: variant run failed ({rc})")
        state["k"] += iters
        return state, ld[:iters], lp[:iters]

    # -- PDHG on Kbar (comparison method / x_nat generator) ---------------------------
    @classmethod
    def pdhg_params(cls, norm_K: float, mu: float, rho: float = 0.99):
        out = np.zeros(3)
        cls.lib().orc_pdhg_params(norm_K, mu, rho, _dp(out))
        return out   # s, t, theta

    def pdhg(self, b: np.ndarray, iters: int, s: float, t: float, theta: float, state=None):
        d, m = self.n * self.n, self.m
        if state is None:
            state = {"x": np.zeros(d), "xbar": np.zeros(d), "y": np.zeros(m), "k": 0}
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        rc = self.L.orc_pdhg_run(self.ref, _dp(b), iters, s, t, theta, _dp(state["x"]),
                                 _dp(state["xbar"]), _dp(state["y"]))
        if rc != 0:
            raise ValueError("oracle: PDHG steps must be positive")
        state["k"] += iters
        return state

    # -- step-size theory -----------------------------------------------------------
    def power_eig(self, w, cross: bool, transposed: bool, iters: int) -> float:
        w = np.ascontiguousarray(w, dtype=np.float64)
        return float(self.L.orc_power_eig(self.ref, _dp(w), int(cross), int(transposed), iters))

    def constants(self, iters: int = 100) -> np.ndarray:
        out = np.zeros(3)
        self.L.orc_constants(self.ref, iters, _dp(out))
        return out

    def norm_K(self, iters: int = 100) -> float:
        return float(self.L.orc_norm_K(self.ref, iters))

    @classmethod
    def constants_dense(cls, mats: np.ndarray, p, mu: float, iters: int = 200) -> np.ndarray:
        mats = np.ascontiguousarray(mats, dtype=np.float64)
        r, dy, dx = mats.shape
        p = np.ascontiguousarray(p, dtype=np.float64)
        out = np.zeros(3)
        cls.lib().orc_constants_dense(_dp(mats), r, _dp(p), dx, dy, mu, iters, _dp(out))
        return out

    @classmethod
    def theta(cls, eta, c, rho, L, Lbar, Lbar_p, pmin) -> float:
        return float(cls.lib().orc_theta(eta, c, rho, L, Lbar, Lbar_p, pmin))

    @classmethod
    def eta_opt(cls, c, rho, L, Lbar, Lbar_p, pmin) -> float:
        return float(cls.lib().orc_eta_opt(c, rho, L, Lbar, Lbar_p, pmin))

    @classmethod
    def optimal_step(cls, L, Lbar, Lbar_p, pmin, grid: int = 200) -> np.ndarray:
        out = np.zeros(4)
        cls.lib().orc_optimal_step(L, Lbar, Lbar_p, pmin, grid, _dp(out))
        return out

    # -- fixed point / metrics ------------------------------------------------------
    def solve_quadratic(self, b: np.ndarray, max_iter: int = 2000, tol: float = 1e-13):
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        x = np.zeros(self.n * self.n)
        its = self.L.orc_solve_quadratic(self.ref, _dp(b), max_iter, tol, _dp(x))
        return x.reshape(self.n, self.n), int(its)

    def objective(self, b: np.ndarray, x: np.ndarray) -> float:
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        return float(self.L.orc_objective(self.ref, _dp(b), _dp(x)))
