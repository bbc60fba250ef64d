"""The allocation-free H-solve (gadi_solve_h_2d_noalloc) for callers that
cannot call cudaMalloc: it must give what the handle-based H-solve step
(gadi_step_solve_h) gives, on two calls in a row (its scratch is a static
device array shared by every call, so the second call must not see the
first call's leftovers), and reject grids beyond its static maximum.

Collected last on purpose (file name), so a failure here comes after every
other test has run."""
import numpy as np
import pytest

import oracle as O
import paper_2512_21164_gb300 as G
from helpers import BF16, FP32, FP64, us_empty, us_to_device, us_to_host
from workloads import conv_diff_2d

TOL = {FP64: 1e-12, FP32: 2e-5, BF16: 0.06}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_21164_gb300 import build
    build.build()


def _rnd(prec, a):
    if prec == FP64:
        return np.asarray(a, np.float64)
    if prec == FP32:
        return np.asarray(a, np.float32).astype(np.float64)
    return np.array([O.round_bf16(v) for v in a])


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [FP64, FP32, BF16])
@pytest.mark.parametrize("nx,ny", [(64, 48), (37, 29)])
def test_noalloc_matches_step_solve_h(prec, nx, ny):
    import torch
    p, xt = conv_diff_2d(nx, 301, ny=ny)
    rs = _rnd(prec, xt - 0.5)
    alpha, tol, maxit, stag = 0.3, 1e-4, 200, 10
    with G.Gadi.from_problem(p) as H:
        z_ref = us_empty(p.nvec, prec)
        its_ref = H.step_solve_h(alpha, prec, us_to_device(rs, prec), z_ref, tol, maxit, stag)
    zr = us_to_host(z_ref, prec)
    for call in range(2):
        z = us_empty(p.nvec, prec)
        z.fill_(7)  # the output must be fully overwritten
        st, its = G.solve_h_2d_noalloc(nx, ny, alpha, prec, us_to_device(rs, prec), z, tol, maxit, stag)
        torch.cuda.synchronize()
        assert st == G.OK and its == its_ref, (call, its, its_ref)
        zg = us_to_host(z, prec)
        err = np.linalg.norm(zg - zr) / np.linalg.norm(zr)
        assert err <= TOL[prec], (call, err)


def test_noalloc_rejects_grids_beyond_the_maximum():
    st, _ = G.solve_h_2d_noalloc(513, 512, 0.3, FP32, 1, 1, 1e-3, 10, check=False)
    assert st == G.ERR_INVALID
    assert "static scratch maximum" in G.last_error()
