"""Failure detection without a GPU fault: a reference medium far softer than the
phases makes the basic scheme amplify instead of contract, and the solve reports
the non-finite residual as BFCS_ERR_DIVERGED; a host-side wait limit far below a
solve's duration returns BFCS_ERR_TIMEOUT while the enqueued kernels finish
normally.  In both cases the context and later solves stay usable."""
import os

import numpy as np
import pytest
import torch

from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_divergent_reference_medium_reports_diverged(precision):
    p = W.config_c1()
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, precision)
    with api.Plan(p.dims, precision) as plan:
        with pytest.raises(_lib.BfcsError) as e:
            plan.solve(ph, p.phases, (0.01, 0.005), b, tol=1e-8, maxit=2000)   # C0 ~ L / 1000
        assert e.value.code == _lib.ERR_DIVERGED
        eps, _, _, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-4, maxit=2000)
        assert info.status == _lib.OK and torch.isfinite(eps).all()


def test_host_wait_limit_returns_timeout():
    p = W.config_c2(contrast=10.0, seed=1)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp32")
    plan = api.Plan(p.dims, "fp32")
    old = os.environ.get("BFCS_WAIT_TIMEOUT_S")
    os.environ["BFCS_WAIT_TIMEOUT_S"] = "1e-6"
    try:
        with pytest.raises(_lib.BfcsError) as e:
            plan.solve(ph, p.phases, p.c0, b, tol=1e-4, maxit=20000)
        assert e.value.code == _lib.ERR_TIMEOUT
    finally:
        if old is None:
            del os.environ["BFCS_WAIT_TIMEOUT_S"]
        else:
            os.environ["BFCS_WAIT_TIMEOUT_S"] = old
        torch.cuda.synchronize()              # the enqueued work completes normally
        plan.close()
    with api.Plan(p.dims, "fp32") as fresh:
        _, _, _, info = fresh.solve(ph, p.phases, p.c0, b, tol=1e-4, maxit=20000)
    assert info.status == _lib.OK and info.resid <= 1e-4
