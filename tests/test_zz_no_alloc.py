"""The allocation-free H-solve (gadi_solve_h_2d_noalloc), for callers that
cannot call cudaMalloc (a fixed device-memory pool, a host program that owns
every allocation): it must give what the handle-based H-solve step
(gadi_step_solve_h) gives.  Its scratch is one static device array shared by
every call, so a call must not see what the previous call left there: two
checked calls on one grid are separated by a call on a larger grid with
another right-hand side, alpha and precision, which leaves different values in
every part of the scratch.  It must also reject grids beyond its static
maximum.

Collected last on purpose (file name), so a failure here comes after every
other test has run."""
import numpy as np
import pytest

import oracle as O
import paper_2512_21164_gb300 as G
from helpers import BF16, FP32, FP64, us_empty, us_to_device, us_to_host
from workloads import SplitMix64, conv_diff_2d

# the larger grid's reference takes the resident H-solve form (more rows
# than SMs), whose sums run in another order: compared within these bounds
# per CG step (those of the fixed-iteration H-solve step tests)
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


def _reference(nx, ny, prec, rs, alpha, tol, maxit, stag):
    p, _ = conv_diff_2d(nx, 1, ny=ny)
    with G.Gadi.from_problem(p) as H:
        z = us_empty(p.nvec, prec)
        its = H.step_solve_h(alpha, prec, us_to_device(rs, prec), z, tol, maxit, stag)
    return us_to_host(z, prec), its


def _noalloc(nx, ny, prec, rs, alpha, tol, maxit, stag):
    import torch
    z = us_empty(nx * ny, prec)
    z.fill_(7)  # the output must be fully overwritten
    st, its = G.solve_h_2d_noalloc(nx, ny, alpha, prec, us_to_device(rs, prec), z, tol, maxit, stag)
    torch.cuda.synchronize()
    assert st == G.OK, G.status_str(st)
    return us_to_host(z, prec), its


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [FP64, FP32, BF16])
@pytest.mark.parametrize("nx,ny", [(64, 48), (37, 29)])
def test_noalloc_matches_step_solve_h(prec, nx, ny):
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    rs = _rnd(prec, SplitMix64(301).uniform_array(nx * ny) - 0.5)
    args = (0.3, 1e-4, 200, 10)
    zr, its_r = _reference(nx, ny, prec, rs, *args)
    # a grid with fewer rows than SMs: both entry points run the streaming
    # H-solve on one block per SM, so the same bits are expected
    same_bits = ny < nsm
    # the larger call in between: another size, right-hand side, alpha and
    # precision (so other bytes of every work vector and control word)
    other = FP32 if prec != FP32 else BF16
    nb = 512
    rs_b = _rnd(other, (SplitMix64(302).uniform_array(nb * nb) - 0.5) * 3.0)
    args_b = (0.05, 0.0, 6, 0)  # exactly 6 CG steps
    for call in range(2):
        zg, its = _noalloc(nx, ny, prec, rs, *args)
        assert its == its_r, (call, its, its_r)
        if same_bits:
            assert np.array_equal(zg, zr), (call, np.max(np.abs(zg - zr)))
        else:
            err = np.linalg.norm(zg - zr) / np.linalg.norm(zr)
            assert err <= TOL[prec], (call, err)
        if call == 0:
            zb, its_b = _noalloc(nb, nb, other, rs_b, *args_b)
            zbr, its_br = _reference(nb, nb, other, rs_b, *args_b)
            assert its_b == its_br == 6, (its_b, its_br)
            err = np.linalg.norm(zb - zbr) / np.linalg.norm(zbr)
            assert err <= 6 * TOL[other], err


def test_noalloc_rejects_grids_beyond_the_maximum():
    st, _ = G.solve_h_2d_noalloc(513, 512, 0.3, FP32, 1, 1, 1e-3, 10, check=False)
    assert st == G.ERR_INVALID
    assert "static scratch maximum" in G.last_error()
