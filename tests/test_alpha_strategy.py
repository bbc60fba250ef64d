"""Sec. 4.3 parameter strategy: the library's closed-form condition numbers of
H = alpha I + M and S = alpha I + N (step 2) against dense condition numbers
computed from the oracle's matrices, and the alpha selection of eq. (4.1)."""
import numpy as np
import pytest

import oracle as O
import paper_2512_21164_gb300 as G
from workloads import K_3D7, Problem, complex_rd, conv_diff_2d, conv_diff_3d, random_csr

U = {G.FP64: 1.11e-16, G.FP32: 5.96e-8, G.BF16: 3.91e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_21164_gb300 import build
    build.build()


def _cases():
    return [conv_diff_2d(9, 1, beta=(30.0, 70.0), ny=7)[0], conv_diff_2d(8, 2)[0],
            Problem(K_3D7, 5, 4, 6, 1.0 / 6, (11.0, 23.0, 5.0)), complex_rd(6, 3)[0]]


@pytest.mark.parametrize("i", range(4))
@pytest.mark.parametrize("alpha", [0.01, 0.3, 4.0])
def test_condition_numbers_against_dense(i, alpha):
    p = _cases()[i]
    orc = O.Oracle(p)
    M, N = orc.dense(O.OP_M), orc.dense(O.OP_N)
    I = np.eye(M.shape[0])
    kh, ks = G.condition_numbers(p, alpha)
    assert abs(kh - np.linalg.cond(alpha * I + M)) <= 1e-9 * kh
    nn = np.linalg.norm(N, 2)
    assert abs(ks - np.sqrt(alpha ** 2 + nn ** 2) / alpha) <= 1e-9 * ks  # the stated bound, exactly
    assert ks >= np.linalg.cond(alpha * I + N) * (1 - 1e-12)               # ... and a bound


@pytest.mark.parametrize("prec", [G.FP64, G.FP32, G.BF16])
def test_select_alpha_eq_4_1(prec):
    p = conv_diff_2d(128, 4)[0]
    a0 = 1e-3
    a = G.select_alpha(p, a0, prec, 0.01)
    kh, ks = G.condition_numbers(p, a)
    assert kh * ks * U[prec] < 0.01
    if a > a0:
        kh2, ks2 = G.condition_numbers(p, a / 2)
        assert kh2 * ks2 * U[prec] >= 0.01
    assert a / a0 == 2 ** round(np.log2(a / a0))


def test_condition_numbers_unsupported_for_csr():
    import ctypes as C
    p, _ = random_csr(20, 5)
    P = G.Problem()
    P.kind, P.n = G.CSR, 20
    kh, ks = C.c_double(), C.c_double()
    assert G.lib().gadi_condition_numbers(C.byref(P), 1.0, C.byref(kh), C.byref(ks)) == G.ERR_UNSUPPORTED
