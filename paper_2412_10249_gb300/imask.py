"""Thin ctypes binding of libimask.so (include/imask.h).

Argument marshalling only: every function checks tensor dtypes, devices and
sizes, passes raw pointers and the current CUDA stream to the C ABI, and turns
a non-OK status into ``ImaskError``.  All computation happens in the library's
CUDA kernels; there is no CPU fallback, and loading fails loudly when the
library has not been built.

The module-level functions carry the C names (``imask_plan``,
``imask_project``, ...); ``Plan`` and ``State`` wrap them for convenience.
"""
from __future__ import annotations

import ctypes
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# IMASK_LIBRARY selects another build of the same library (e.g. one compiled
# with different tile constants); the default is the in-tree build.
LIB_PATH = os.environ.get("IMASK_LIBRARY") or os.path.join(_HERE, "_build", "libimask.so")

STATUS = {0: "IMASK_OK", 1: "IMASK_ERR_INVALID", 2: "IMASK_ERR_SHAPE", 3: "IMASK_ERR_OOM",
          4: "IMASK_ERR_CUDA", 5: "IMASK_ERR_TIMEOUT", 6: "IMASK_ERR_NONFINITE"}


class ImaskError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("n_angles", ctypes.c_int32), ("n_det", ctypes.c_int32),
        ("geometry", ctypes.c_int32),
        ("fov", ctypes.c_double), ("det_spacing", ctypes.c_double),
        ("angle_start", ctypes.c_double), ("angle_span", ctypes.c_double),
        ("src_dist", ctypes.c_double), ("det_dist", ctypes.c_double),
        ("levels", ctypes.c_int32), ("probs", ctypes.POINTER(ctypes.c_double)),
        ("reg", ctypes.c_int32), ("mu", ctypes.c_double), ("tv_lambda", ctypes.c_double),
        ("tv_eps", ctypes.c_double), ("tv_inner", ctypes.c_int32), ("sigma", ctypes.c_double),
        ("storage", ctypes.c_int32),
        ("variant", ctypes.c_int32), ("theta", ctypes.c_double),
        ("dual_tables", ctypes.c_int32), ("draws", ctypes.c_int32),
        ("step_rule", ctypes.c_int32), ("power_iters", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("bp_gather", ctypes.c_int32),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double), ("sigma", ctypes.c_double), ("theta", ctypes.c_double),
        ("L", ctypes.c_double), ("Lbar", ctypes.c_double), ("Lbar_p", ctypes.c_double),
        ("norm_K", ctypes.c_double), ("n_meas", ctypes.c_int64), ("n_pix", ctypes.c_int64),
        ("levels", ctypes.c_int32), ("n_xmajor_views_split", ctypes.c_int32),
        ("n_xmajor_rays", ctypes.c_int64), ("state_bytes", ctypes.c_int64),
        ("plan_bytes", ctypes.c_int64), ("autotuned", ctypes.c_int32),
        ("bp_view_groups", ctypes.c_int32 * 8),
        ("fp_strip_lines", ctypes.c_int32 * 8),
        ("bp_gather", ctypes.c_int32),
    ]


_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_DP = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); the exported C ABI
SIGNATURES = {
    "imask_plan": (_I32, [ctypes.POINTER(Desc), ctypes.POINTER(_VP)]),
    "imask_plan_destroy": (_I32, [_VP]),
    "imask_plan_get_info": (_I32, [_VP, ctypes.POINTER(PlanInfo)]),
    "imask_plan_check": (_I32, [_VP]),
    "imask_plan_axis_split": (_I32, [_VP, _I32P, _I32P]),
    "imask_geometry_axis_split": (_I32, [ctypes.POINTER(Desc), _I32P, _I32P]),
    "imask_geometry_view_groups": (_I32, [ctypes.POINTER(Desc), _I32, _I32, _I32P, _I32P,
                                          _I32P]),
    "imask_optimal_step": (_I32, [ctypes.c_double] * 4 + [_I32, _DP]),
    "imask_project": (_I32, [_VP, _I32, _VP, _VP, _VP]),
    "imask_backproject": (_I32, [_VP, _I32, _VP, _VP, _VP]),
    "imask_backproject_noalloc": (_I32, [_VP, _I32, _VP, _VP, _VP]),
    "imask_levels": (_I32, [_VP, _U64, _I64, _I64, _VP, _VP]),
    "imask_state_create": (_I32, [_VP, _VP, _U64, ctypes.POINTER(_VP), _VP]),
    "imask_step": (_I32, [_VP, _I32, _VP]),
    "imask_state_iteration": (_I64, [_VP]),
    "imask_state_get": (_I32, [_VP, _I32, _VP, _VP]),
    "imask_state_checkpoint_bytes": (_I64, [_VP]),
    "imask_state_save": (_I32, [_VP, _VP, _VP]),
    "imask_state_load": (_I32, [_VP, _VP, _VP]),
    "imask_state_get_x": (_I32, [_VP, _VP, _VP]),
    "imask_state_destroy": (_I32, [_VP]),
    "imask_solve": (_I32, [_VP, _VP, _U64, _I32, _VP, _VP]),
    "imask_objective": (_I32, [_VP, _VP, _VP, _DP, _VP]),
    "imask_rel_distance": (_I32, [_I64, _VP, _VP, _DP, _VP]),
    "imask_state_set_storage": (_I32, [_VP, _I32, _VP]),
    "imask_probe_smem": (_I32, [_DP, _VP]),
    "imask_selftest_projector_timeout": (_I32, [_VP, _VP]),
    "imask_batch_create": (_I32, [_VP, _I32, _VP]),
    "imask_batch_create_fused": (_I32, [_VP, _I32, _VP]),
    "imask_batch_step": (_I32, [_VP, _I32, _VP]),
    "imask_batch_destroy": (_I32, [_VP]),
    "imask_pdhg": (_I32, [_VP, _VP, _I32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                          _VP, _VP]),
    "imask_pdhg_params": (_I32, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP]),
    "imask_profile_enable": (_I32, [_I32]),
    "imask_profile_read": (_I32, [_DP, _I64P, _I32]),
    "imask_launch_count": (_I64, []),
    "imask_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Loads libimask.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with paper_2412_10249_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise ImaskError(status, lib().imask_last_error().decode(errors="replace"))


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor, numel: int, dtype=torch.float32, name="tensor"):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def make_desc(params: dict):
    """imask_desc from a parameter dict (keys of inputs.Problem); returns (desc, keepalive)."""
    d = Desc()
    d.n = int(params["n"])
    d.n_angles = int(params["n_angles"])
    d.n_det = int(params["n_det"])
    d.geometry = int(params.get("geometry", 0))
    d.fov = float(params.get("fov", 1.0))
    d.det_spacing = float(params.get("det_spacing", 0.0))
    d.angle_start = float(params.get("angle_start", 0.0))
    d.angle_span = float(params.get("angle_span", math.pi))
    d.src_dist = float(params.get("src_dist", 2.0))
    d.det_dist = float(params.get("det_dist", 1.0))
    d.levels = int(params.get("levels", 1))
    keep = None
    probs = params.get("probs")
    if probs is not None:
        keep = (ctypes.c_double * len(probs))(*[float(v) for v in probs])
        d.probs = ctypes.cast(keep, _DP)
    d.reg = int(params.get("reg", 0))
    d.mu = float(params.get("mu", 1.0))
    d.tv_lambda = float(params.get("tv_lambda", 0.0))
    d.tv_eps = float(params.get("tv_eps", 1e-2))
    d.tv_inner = int(params.get("tv_inner", 20))
    d.sigma = float(params.get("sigma", 0.0))
    d.storage = int(params.get("storage", 0))
    d.variant = int(params.get("variant", 0))
    d.theta = float(params.get("theta", 1.0))
    d.dual_tables = int(params.get("dual_tables", 0))
    d.draws = int(params.get("draws", 0))
    d.step_rule = int(params.get("step_rule", 0))
    d.power_iters = int(params.get("power_iters", 0))
    d.autotune = int(params.get("autotune", 0))
    d.bp_gather = int(params.get("bp_gather", 0))
    return d, keep


# ---- C-named functions ---------------------------------------------------------------

def imask_plan(params: dict) -> ctypes.c_void_p:
    d, keep = make_desc(params)
    h = ctypes.c_void_p()
    _check(lib().imask_plan(ctypes.byref(d), ctypes.byref(h)))
    del keep
    return h


def imask_plan_destroy(plan):
    _check(lib().imask_plan_destroy(plan))


def imask_plan_get_info(plan) -> dict:
    info = PlanInfo()
    _check(lib().imask_plan_get_info(plan, ctypes.byref(info)))
    out = {k: getattr(info, k) for k, _ in PlanInfo._fields_}
    out["bp_view_groups"] = list(info.bp_view_groups)
    out["fp_strip_lines"] = list(info.fp_strip_lines)
    return out


def imask_plan_check(plan):
    _check(lib().imask_plan_check(plan))


def imask_geometry_axis_split(params: dict):
    d, keep = make_desc(params)
    na = d.n_angles
    split = (ctypes.c_int32 * na)()
    fx = (ctypes.c_int32 * na)()
    _check(lib().imask_geometry_axis_split(ctypes.byref(d), split, fx))
    return list(split), list(fx)


def imask_geometry_view_groups(params: dict, role: int, n_groups: int):
    """(views of the role, group bounds) of the back-projector's split."""
    d, keep = make_desc(params)
    views = (ctypes.c_int32 * max(1, d.n_angles))()
    nv = ctypes.c_int32(0)
    bounds = (ctypes.c_int32 * (n_groups + 1))()
    _check(lib().imask_geometry_view_groups(ctypes.byref(d), role, n_groups, views,
                                            ctypes.byref(nv), bounds))
    return list(views[:nv.value]), list(bounds)


def imask_optimal_step(L, Lbar, Lbar_p, p_min, grid=200):
    out = (ctypes.c_double * 4)()
    _check(lib().imask_optimal_step(L, Lbar, Lbar_p, p_min, grid, out))
    return list(out)


def imask_project(plan, level, x, sino, n, m, stream=None):
    _check(lib().imask_project(plan, level, _ptr(x, n * n, name="x"), _ptr(sino, m, name="sino"),
                               _stream(stream)))


def imask_backproject(plan, level, y, img, n, m, stream=None):
    _check(lib().imask_backproject(plan, level, _ptr(y, m, name="y"), _ptr(img, n * n, name="img"),
                                   _stream(stream)))


def imask_backproject_noalloc(plan, level, y, img, n, m, stream=None):
    """K_level^T y without device allocation (fixed 16 MiB library array)."""
    _check(lib().imask_backproject_noalloc(plan, level, _ptr(y, m, name="y"),
                                           _ptr(img, n * n, name="img"), _stream(stream)))


def imask_levels(plan, seed, k0, n, out, stream=None):
    _check(lib().imask_levels(plan, seed, k0, n, _ptr(out, n, torch.int32, "out"), _stream(stream)))


def imask_solve(plan, b, seed, iters, x, n, m, stream=None):
    _check(lib().imask_solve(plan, _ptr(b, m, name="b"), seed, iters, _ptr(x, n * n, name="x"),
                             _stream(stream)))


def imask_pdhg_params(norm_K: float, mu: float, rho: float = 0.99):
    out = (ctypes.c_double * 3)()
    _check(lib().imask_pdhg_params(norm_K, mu, rho, out))
    return tuple(out)


def imask_rel_distance(a, b, stream=None) -> float:
    out = ctypes.c_double()
    n = a.numel()
    _check(lib().imask_rel_distance(n, _ptr(a, n, name="a"), _ptr(b, n, name="b"),
                                    ctypes.byref(out), _stream(stream)))
    return out.value


def imask_profile_enable(period):
    """0/False: off; True/1: every launch; N: every N-th solver iteration."""
    _check(lib().imask_profile_enable(int(period)))


def imask_profile_read(reset: bool = False):
    ms = (ctypes.c_double * 24)()
    cnt = (ctypes.c_int64 * 24)()
    _check(lib().imask_profile_read(ms, cnt, 1 if reset else 0))
    return list(ms), list(cnt)


def imask_probe_smem(stream=None):
    """Measured shared-memory ceilings (GB/s): conflict-free loads, private
    read-modify-writes."""
    out = (ctypes.c_double * 2)()
    _check(lib().imask_probe_smem(out, _stream(stream)))
    return tuple(out)


def imask_launch_count() -> int:
    return int(lib().imask_launch_count())


# ---- convenience wrappers --------------------------------------------------------------

class Plan:
    """An immutable plan (geometry tables on the device, step size)."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self.n = int(params["n"])
        self.m = int(params["n_angles"]) * int(params["n_det"])
        self.levels_count = int(params.get("levels", 1))
        self.handle = imask_plan(self.params)

    def close(self):
        if self.handle:
            imask_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return imask_plan_get_info(self.handle)

    def check(self):
        imask_plan_check(self.handle)

    def selftest_timeout(self, stream=None):
        """Runs the failure-detection self-test; check() then raises TIMEOUT."""
        _check(lib().imask_selftest_projector_timeout(self.handle, _stream(stream)))

    def axis_split(self):
        na = int(self.params["n_angles"])
        split = (ctypes.c_int32 * na)()
        fx = (ctypes.c_int32 * na)()
        _check(lib().imask_plan_axis_split(self.handle, split, fx))
        return list(split), list(fx)

    def project(self, level: int, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        if out is None:
            out = torch.empty(self.m, device=x.device, dtype=torch.float32)
        imask_project(self.handle, level, x, out, self.n, self.m, stream)
        return out

    def backproject(self, level: int, y: torch.Tensor, out: torch.Tensor | None = None,
                    stream=None):
        if out is None:
            out = torch.empty(self.n * self.n, device=y.device, dtype=torch.float32)
        imask_backproject(self.handle, level, y, out, self.n, self.m, stream)
        return out

    def levels(self, seed: int, k0: int, count: int, device="cuda"):
        out = torch.empty(count, device=device, dtype=torch.int32)
        imask_levels(self.handle, seed, k0, count, out)
        return out

    def solve(self, b: torch.Tensor, seed: int, iters: int, out: torch.Tensor | None = None,
              stream=None):
        if out is None:
            out = torch.empty(self.n * self.n, device=b.device, dtype=torch.float32)
        imask_solve(self.handle, b, seed, iters, out, self.n, self.m, stream)
        return out

    def objective(self, x: torch.Tensor, b: torch.Tensor, stream=None) -> float:
        out = ctypes.c_double()
        _check(lib().imask_objective(self.handle, _ptr(x, self.n * self.n, name="x"),
                                     _ptr(b, self.m, name="b"), ctypes.byref(out),
                                     _stream(stream)))
        return out.value

    def pdhg(self, b: torch.Tensor, iters: int, s: float, t: float, theta: float,
             out: torch.Tensor | None = None, stream=None):
        if out is None:
            out = torch.empty(self.n * self.n, device=b.device, dtype=torch.float32)
        _check(lib().imask_pdhg(self.handle, _ptr(b, self.m, name="b"), iters, s, t, theta,
                                _ptr(out, self.n * self.n, name="x"), _stream(stream)))
        return out

    def state(self, b: torch.Tensor, seed: int, stream=None) -> "State":
        return State(self, b, seed, stream)


class State:
    """One solve of Alg. 1 (device-resident x, y, SAGA tables)."""

    X, Y, PHI_MEAN, PSI_MEAN = 0, 1, 2, 3

    def __init__(self, plan: Plan, b: torch.Tensor, seed: int, stream=None):
        self.plan = plan
        h = ctypes.c_void_p()
        _check(lib().imask_state_create(plan.handle, _ptr(b, plan.m, name="b"), seed,
                                        ctypes.byref(h), _stream(stream)))
        self.handle = h

    def step(self, n_iters: int, stream=None):
        _check(lib().imask_step(self.handle, n_iters, _stream(stream)))

    def set_storage(self, storage: int, stream=None):
        """Converts the measurement-side tables (0 fp32, 1 bf16, 2 fp16)."""
        _check(lib().imask_state_set_storage(self.handle, storage, _stream(stream)))

    @property
    def k(self) -> int:
        return int(lib().imask_state_iteration(self.handle))

    def get(self, what: int, stream=None) -> torch.Tensor:
        n = self.plan.m if what in (self.Y, self.PSI_MEAN) else self.plan.n * self.plan.n
        out = torch.empty(n, device="cuda", dtype=torch.float32)
        _check(lib().imask_state_get(self.handle, what, _ptr(out, n, name="out"),
                                     _stream(stream)))
        return out

    def save(self, stream=None) -> torch.Tensor:
        """A checkpoint of the whole state in a device byte tensor."""
        n = int(lib().imask_state_checkpoint_bytes(self.handle))
        out = torch.empty(n, device="cuda", dtype=torch.uint8)
        _check(lib().imask_state_save(self.handle, ctypes.c_void_p(out.data_ptr()),
                                      _stream(stream)))
        return out

    def load(self, checkpoint: torch.Tensor, stream=None):
        """Restores a checkpoint of a state of a plan with the same descriptor."""
        if not (checkpoint.is_cuda and checkpoint.dtype == torch.uint8
                and checkpoint.is_contiguous()):
            raise ValueError("checkpoint must be a contiguous CUDA uint8 tensor")
        if checkpoint.numel() != int(lib().imask_state_checkpoint_bytes(self.handle)):
            raise ValueError("checkpoint size does not match this state")
        _check(lib().imask_state_load(self.handle, ctypes.c_void_p(checkpoint.data_ptr()),
                                      _stream(stream)))

    def close(self):
        if self.handle:
            _check(lib().imask_state_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent states advanced together through captured CUDA graphs:
    one graph branch per state (default), or, with ``fused=True``, one
    launch of each kernel per iteration for all states."""

    def __init__(self, states, fused: bool = False):
        self.states = list(states)
        self.fused = bool(fused)
        arr = (ctypes.c_void_p * len(self.states))(*[st.handle.value for st in self.states])
        h = ctypes.c_void_p()
        create = lib().imask_batch_create_fused if self.fused else lib().imask_batch_create
        _check(create(arr, len(self.states), ctypes.byref(h)))
        self.handle = h

    def step(self, n_iters: int, stream=None):
        _check(lib().imask_batch_step(self.handle, n_iters, _stream(stream)))
        return self

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().imask_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
