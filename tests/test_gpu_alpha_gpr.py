"""Sec. 4.2 on the GPU: a GPR trained on small instances of the paper's 2D
family predicts an alpha for a larger one whose solve moves at most 1.5x the
bytes of the best alpha a sweep finds there."""
import math

import numpy as np
import pytest

import paper_2512_21164_gb300 as G
from paper_2512_21164_gb300 import alpha_gpr as A
from workloads import alpha_star, paper_cdr_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_21164_gb300 import build
    build.build()


def test_gpr_alpha_for_a_larger_instance():
    f = np.arange(-1.0, 5.01, 0.5)
    model = A.train(paper_cdr_2d, [32, 48, 64, 96], G.FP32, 0.0, 1e-10, alpha_star, log2_factors=f)
    assert len(model.gp.x) == 4
    n = 160
    f_pred, f_std = model.predict_log2_factor(n)
    assert math.isfinite(f_pred) and f_std >= 0
    runs = A.sweep(paper_cdr_2d, n, G.FP32, 0.0, list(f) + [f_pred], 1e-10, alpha_star)
    best = min(r[1] for r in runs[:-1])
    pred = runs[-1]
    assert pred[2] == G.OK
    assert pred[1] <= 1.5 * best, (f_pred, pred[1], best)
