"""The index-checked build (-DIMASK_BOUNDS_CHECK): on small cases of every
geometry and iteration form, no kernel computes an index outside its buffer
(imask_plan_check stays clean) and the results still match the oracle.  The
checked library is loaded in a child process (one library per process)."""
import os
import subprocess
import sys
import textwrap

import pytest
import torch

from paper_2412_10249_gb300 import build as pkg_build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r"""
    import math, sys
    import numpy as np, torch
    sys.path.insert(0, ROOT)
    from oracle import Oracle
    from paper_2412_10249_gb300 import imask, inputs
    assert imask.LIB_PATH.endswith("checked/libimask.so"), imask.LIB_PATH

    def rel(a, b):
        a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    cases = [
        inputs.Problem(n=16, n_angles=12, n_det=24, geometry=0, levels=3),
        inputs.Problem(n=32, n_angles=30, n_det=48, geometry=1, angle_span=2 * math.pi, levels=4),
        inputs.Problem(n=48, n_angles=37, n_det=75, geometry=1, angle_span=2 * math.pi,
                       angle_start=0.3, levels=4, probs=[0.3, 0.3, 0.2, 0.2]),
        inputs.Problem(n=40, n_angles=36, n_det=61, geometry=0, levels=3),
    ]
    rng = np.random.default_rng(0)
    for prob in cases:
        params = dict(prob.params(), mu=0.1, sigma=0.04)
        o = Oracle(**params)
        extras = [{}, dict(variant=1, theta=1.0), dict(dual_tables=1, draws=1),
                  dict(reg=2, tv_lambda=0.01, tv_inner=5), dict(storage=2), dict(autotune=1)]
        if prob.geometry == 0:
            extras.append(dict(bp_gather=1))   # the pixel-driven back-projector
        for extra in extras:
            plan = imask.Plan(dict(params, **extra))
            img = rng.random((prob.n, prob.n))
            y = rng.standard_normal(o.m)
            xt = torch.as_tensor(img.ravel().astype(np.float32), device="cuda")
            yt = torch.as_tensor(y.astype(np.float32), device="cuda")
            for ell in range(-1, prob.levels):
                assert rel(plan.project(ell, xt).cpu(), o.K(ell, img)) <= 1e-5, (prob, ell)
                assert rel(plan.backproject(ell, yt).cpu(), o.KT(ell, y)) <= 1e-5, (prob, ell)
            b = o.K(-1, img).ravel()
            x = plan.solve(torch.as_tensor(b.astype(np.float32), device="cuda"), 3, 21)
            assert torch.isfinite(x).all()
            plan.check()            # raises if any index check fired
    print("checked build clean")
""").replace("ROOT", repr(ROOT))


def test_index_checked_build_is_clean():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg_build.build()
    env = dict(os.environ, IMASK_LIBRARY=pkg_build.CHECKED_LIB)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build clean" in r.stdout
