"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/imask.h declares, validates descriptors before touching a device, and
its host-side geometry and step-size logic agree with the oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import Oracle
from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def imask():
    pkg_build.build()
    from paper_2412_10249_gb300 import imask as m
    m.lib()
    return m


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "imask.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(imask_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(imask):
    syms = _declared_symbols()
    assert len(syms) >= 20
    lib = ctypes.CDLL(imask.LIB_PATH)
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    # and the binding covers them all
    assert set(syms) <= set(imask.SIGNATURES), set(syms) - set(imask.SIGNATURES)


@pytest.mark.parametrize("bad,status", [
    (dict(n=0), 2), (dict(levels=9), 1), (dict(n=60, levels=4), 2),
    (dict(probs=[0.5, 0.6]), 1), (dict(geometry=2), 1), (dict(storage=3), 1),
    (dict(storage=1, dual_tables=1), 1),
    (dict(fov=-1.0), 1), (dict(n=4096), 2), (dict(variant=2), 1),
    (dict(variant=1, theta=float("nan")), 1), (dict(dual_tables=2), 1), (dict(draws=-1), 1),
    (dict(step_rule=3), 1), (dict(reg=3), 1), (dict(reg=2, tv_inner=-1), 1),
])
def test_descriptor_validation_without_device(imask, bad, status):
    p = dict(n=64, n_angles=10, n_det=20, levels=2)
    p.update(bad)
    with pytest.raises(imask.ImaskError) as ei:
        imask.imask_geometry_axis_split(p)
    assert ei.value.status == status


@pytest.mark.parametrize("params", [
    inputs.small_problem().params(),
    inputs.Problem(n=64, n_angles=90, n_det=96, geometry=1, angle_span=2 * math.pi).params(),
    inputs.Problem(n=48, n_angles=37, n_det=75, geometry=1, angle_span=2 * math.pi,
                   angle_start=0.3).params(),
    inputs.Problem(n=32, n_angles=64, n_det=45, geometry=0, angle_span=math.pi).params(),
])
def test_axis_split_matches_oracle_bit_exact(imask, params):
    # the plan's per-view split reproduces the oracle's FP64 per-ray decision
    split, first_x = imask.imask_geometry_axis_split(params)
    table = Oracle(**params).xmajor_table()
    nd = params["n_det"]
    for a, (s, fx) in enumerate(zip(split, first_x)):
        expect = np.array([fx if j < s else 1 - fx for j in range(nd)])
        assert np.array_equal(table[a], expect), a


def test_axis_split_of_the_fan512_workload(imask):
    params = inputs.fan512_problem().params()
    split, first_x = imask.imask_geometry_axis_split(params)
    # compare a spread of views with the oracle (full table is 552960 rays)
    o = Oracle(**params)
    for a in range(0, 720, 7):
        row = [o.L.orc_ray_is_xmajor(o.ref, a, j) for j in range(768)]
        expect = [first_x[a] if j < split[a] else 1 - first_x[a] for j in range(768)]
        assert row == expect, a


@pytest.mark.parametrize("consts", [(2.46, 1.74, 1.23, 0.25), (2.46, 1.23, 2.46, 0.5),
                                    (2.41, 1.43, 2.47, 1 / 3), (2.46, 2.46, 2.46, 1.0)])
def test_host_step_solver_matches_oracle(imask, consts):
    got = imask.imask_optimal_step(*consts, 200)
    ref = Oracle.optimal_step(*consts, 200)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_pdhg_params_match_oracle(imask):
    for nk, mu, rho in ((2.46, 1.0, 0.99), (17.3, 0.4, 0.99), (1.0, 3.0, 0.5)):
        got = imask.imask_pdhg_params(nk, mu, rho)
        ref = Oracle.pdhg_params(nk, mu, rho)
        np.testing.assert_allclose(got, ref, rtol=1e-15)
    with pytest.raises(imask.ImaskError):
        imask.imask_pdhg_params(1.0, 0.0, 0.99)


def _role_rays(imask, params):
    split, first_x = imask.imask_geometry_axis_split(params)
    nd = params["n_det"]
    nx = [s if f else nd - s for s, f in zip(split, first_x)]
    return nx, [nd - v for v in nx]


@pytest.mark.parametrize("name", ["fan512", "parallel_pi", "fan_small"])
@pytest.mark.parametrize("n_groups", [1, 4, 7, 57, 400])
def test_view_groups_cover_the_axis_and_balance_its_rays(imask, name, n_groups):
    # the back-projector's view groups (host logic, no device): every view with
    # rays of a major axis is listed once, in order; the groups are consecutive
    # and cover the list; a view sits in the group of its rays' midpoint, so a
    # group's ray count is within one view's count of the even share
    if name == "fan512":
        params = dict(inputs.fan512_problem().params(), mu=1.0, sigma=0.1)
    elif name == "parallel_pi":
        params = dict(inputs.Problem(n=64, n_angles=60, n_det=92, geometry=0,
                                     levels=2).params(), mu=1.0, sigma=0.1)
    else:
        params = dict(inputs.Problem(n=32, n_angles=30, n_det=48, geometry=1,
                                     angle_span=2 * math.pi, levels=3).params(), mu=1.0,
                      sigma=0.1)
    rays = _role_rays(imask, params)
    for role in (0, 1):
        views, bounds = imask.imask_geometry_view_groups(params, role, n_groups)
        assert views == [a for a in range(params["n_angles"]) if rays[role][a] > 0]
        assert bounds[0] == 0 and bounds[-1] == len(views) and len(bounds) == n_groups + 1
        assert all(b0 <= b1 for b0, b1 in zip(bounds, bounds[1:]))
        w = [rays[role][a] for a in views]
        tot, wmax = sum(w), max(w)
        for g in range(n_groups):
            share = sum(w[bounds[g]:bounds[g + 1]])
            assert abs(share - tot / n_groups) <= wmax + 1e-9
        # the midpoint rule, view by view
        acc = 0
        for i, wi in enumerate(w):
            g = min(n_groups - 1, ((2 * acc + wi) * n_groups) // (2 * tot))
            assert bounds[g] <= i < bounds[g + 1]
            acc += wi


def test_view_groups_reject_bad_arguments(imask):
    params = dict(inputs.fan512_problem().params(), mu=1.0, sigma=0.1)
    for role, g in ((2, 4), (-1, 4), (0, 0)):
        with pytest.raises(imask.ImaskError):
            imask.imask_geometry_view_groups(params, role, g)


def test_null_handles_are_refused_without_device(imask):
    # calls on a missing state, plan or batch return INVALID (1) and never
    # touch the device
    lib = imask.lib()
    buf = ctypes.create_string_buffer(64)
    assert lib.imask_state_checkpoint_bytes(None) == -1
    assert lib.imask_state_iteration(None) == -1
    assert lib.imask_state_save(None, ctypes.cast(buf, ctypes.c_void_p), None) == 1
    assert lib.imask_state_load(None, ctypes.cast(buf, ctypes.c_void_p), None) == 1
    assert lib.imask_step(None, 1, None) == 1
    assert lib.imask_state_get(None, 0, ctypes.cast(buf, ctypes.c_void_p), None) == 1
    assert lib.imask_batch_step(None, 1, None) == 1
    assert lib.imask_state_destroy(None) == 0     # destroying nothing is fine
    assert lib.imask_plan_destroy(None) == 0
    assert lib.imask_last_error()                  # the message of the last failure


def test_null_plans_and_outputs_are_refused_without_device(imask):
    # the plan-level entry points check their handles and output pointers
    # before any device work: INVALID (1), with a message naming the argument
    lib = imask.lib()
    arr = (ctypes.c_int32 * 4)()
    buf = ctypes.cast(ctypes.create_string_buffer(64), ctypes.c_void_p)
    info = imask.PlanInfo()
    checks = {
        "imask_plan_axis_split": lambda: lib.imask_plan_axis_split(None, arr, arr),
        "imask_plan_get_info": lambda: lib.imask_plan_get_info(None, ctypes.byref(info)),
        "imask_plan_check": lambda: lib.imask_plan_check(None),
        "imask_project": lambda: lib.imask_project(None, 0, buf, buf, None),
        "imask_backproject": lambda: lib.imask_backproject(None, 0, buf, buf, None),
        "imask_backproject_noalloc": lambda: lib.imask_backproject_noalloc(None, 0, buf, buf,
                                                                           None),
        "imask_levels": lambda: lib.imask_levels(None, 0, 0, 4, buf, None),
        "imask_state_create": lambda: lib.imask_state_create(
            None, buf, 0, ctypes.byref(ctypes.c_void_p()), None),
        "imask_state_set_storage": lambda: lib.imask_state_set_storage(None, 1, None),
        "imask_batch_create": lambda: lib.imask_batch_create(None, 1, buf),
        "imask_batch_create_fused": lambda: lib.imask_batch_create_fused(None, 1, buf),
        "imask_profile_enable": lambda: lib.imask_profile_enable(-1),
    }
    for name, call in checks.items():
        assert call() == 1, name
        assert lib.imask_last_error(), name
    # a batch of one missing state
    states = (ctypes.c_void_p * 1)(None)
    out = ctypes.c_void_p()
    assert lib.imask_batch_create(ctypes.cast(states, ctypes.c_void_p), 1,
                                  ctypes.cast(ctypes.byref(out), ctypes.c_void_p)) == 1
    assert b"NULL" in lib.imask_last_error()
    assert out.value is None
