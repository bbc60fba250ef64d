"""The batched solve's layout rule (gadi_batch_plan, host only, no GPU).

The rule, as the header states it: every class starts at the tuned size
with the fewest block-seconds per unit; groups go to classes in proportion
to their work (units x block-seconds per unit), at least one each and no
more than the class has units, taken back from the class with the most
blocks while the grid is over-full, then added one at a time to the class
that would finish last while the grid has room; then one class at a time
moves to the size that lowers the estimated finish time (the class whose
units, in rounds of its group count, end last) most, until no move helps.

The tests restate the group assignment and the estimate in Python and
check the library's layouts against them: the groups it returns are the
rule's groups for the sizes it returns, its estimate is the model's, no
single-class move lowers that estimate, and the structural bounds hold."""
import math

import pytest

import paper_2512_21164_gb300 as G
from workloads import SplitMix64

SIZES = G.BATCH_SIZES


def _assign(sz, T, count, total):
    ncl = len(sz)
    w = [count[c] * sz[c] * T[c] for c in range(ncl)]
    ws = sum(w)
    g = [max(1, min(count[c], int(math.floor(total * w[c] / ws / sz[c])))) for c in range(ncl)]
    used = sum(g[c] * sz[c] for c in range(ncl))
    while used > total:
        pick = None
        for c in range(ncl):
            if g[c] > 1 and (pick is None or g[c] * sz[c] > g[pick] * sz[pick]):
                pick = c
        if pick is None:
            return None
        g[pick] -= 1
        used -= sz[pick]
    while True:
        pick, worst = None, -1.0
        for c in range(ncl):
            m = math.ceil(count[c] / g[c]) * T[c]
            if g[c] < count[c] and used + sz[c] <= total and m > worst:
                worst, pick = m, c
        if pick is None:
            return g
        g[pick] += 1
        used += sz[pick]


def _estimate(g, T, count):
    return max(math.ceil(count[c] / g[c]) * T[c] for c in range(len(g)))


def _random_table(seed):
    r = SplitMix64(seed)
    ncl = 1 + int(r.uniform() * 5)
    side = sorted((64 * (1 + int(r.uniform() * 16)) for _ in range(ncl)), reverse=True)
    count = [1 + int(r.uniform() * 40) for _ in range(ncl)]
    t = []
    for c in range(ncl):
        base = side[c] ** 2 * 1e-9
        row = []
        for i, s in enumerate(SIZES):
            # roughly 1/s with noise and a floor; some sizes not admitted
            v = base * (1.0 / s + 0.02) * (0.7 + 0.6 * r.uniform())
            row.append(-1.0 if r.uniform() < 0.2 else v)
        if max(row) <= 0:
            row[0] = base
        t.append(row)
    return side, count, t


@pytest.mark.parametrize("seed", range(40))
def test_layout_follows_the_rule_and_is_locally_optimal(seed):
    side, count, t = _random_table(seed)
    total = 152
    try:
        sz, gr, est = G.batch_plan(side, count, t, total=total)
    except G.GadiError:
        # only when the classes' single groups cannot fit: not with 152 blocks
        pytest.fail("no layout")
    ncl = len(side)
    assert sum(s * g for s, g in zip(sz, gr)) <= total
    idx = [SIZES.index(s) for s in sz]
    T = [t[c][idx[c]] * side[c] for c in range(ncl)]
    for c in range(ncl):
        assert t[c][idx[c]] > 0, "a size the tuner did not admit"
        assert 1 <= gr[c] <= count[c]
    assert gr == _assign(sz, T, count, total)
    assert est == pytest.approx(_estimate(gr, T, count), rel=1e-12)
    # no single-class move to another admitted size lowers the estimate
    for c in range(ncl):
        for i, s in enumerate(SIZES):
            if t[c][i] <= 0 or s == sz[c] or s > total:
                continue
            s2 = list(sz)
            s2[c] = s
            T2 = list(T)
            T2[c] = t[c][i] * side[c]
            g2 = _assign(s2, T2, count, total)
            if g2 is None:
                continue
            assert _estimate(g2, T2, count) >= est * 0.999, (c, s)


def test_layout_never_worse_than_the_cheapest_sizes():
    for seed in range(40, 80):
        side, count, t = _random_table(seed)
        sz, gr, est = G.batch_plan(side, count, t, total=152)
        start = []
        for c in range(len(side)):
            cand = [(SIZES[i] * t[c][i], -SIZES[i], i) for i in range(7) if t[c][i] > 0]
            start.append(min(cand)[2])
        s0 = [SIZES[i] for i in start]
        T0 = [t[c][start[c]] * side[c] for c in range(len(side))]
        g0 = _assign(s0, T0, count, 152)
        assert est <= _estimate(g0, T0, count) * (1 + 1e-12)


def test_fixed_size_and_errors():
    sz, gr, est = G.batch_plan([256, 128], [10, 10], None, fixed=8, total=152)
    assert sz == [8, 8] and sum(gr) * 8 <= 152 and min(gr) >= 1 and max(gr) <= 10
    # fixed sizes above the grid are clipped to it
    sz, gr, _ = G.batch_plan([64], [3], None, fixed=500, total=100)
    assert sz == [100] and gr == [1]
    # a class with no admitted size
    with pytest.raises(G.GadiError):
        G.batch_plan([64, 32], [2, 2], [[1e-3] * 7, [-1.0] * 7])
    # more classes than their single groups can fit
    with pytest.raises(G.GadiError):
        G.batch_plan([64, 32, 16], [1, 1, 1], None, fixed=64, total=100)
    with pytest.raises(G.GadiError):
        G.batch_plan([64], [0], None, fixed=4)


def test_measured_interleaved_table():
    """The tuner table of the 96-system batch with interleaved right-hand
    sides (seconds per outer iteration on 1..64 blocks, as measured): the
    class of 1024^2 units gets two groups of 64 blocks, and the 512^2 class,
    whose cheapest size (64) would leave the 1024^2 class one group, moves to
    groups of one block."""
    t = [[0.076955, 0.0350361, 0.0175946, 0.00807607, 0.00461126, 0.00223407, 0.00100264],
         [0.0150751, 0.00778185, 0.00410882, 0.00212764, 0.00102332, 0.000470422, 0.000368646],
         [0.00455326, 0.00239971, 0.00119041, 0.000545784, 0.000912806, 0.000672976, 0.000873384],
         [0.00203464, 0.000905182, 0.000611308, 0.000443614, 0.000342472, 0.000244026, 0.000114128]]
    sz, gr, est = G.batch_plan([1024, 512, 256, 128], [24, 22, 23, 27], t)
    assert sz[0] == 64 and gr[0] == 2
    assert sum(s * g for s, g in zip(sz, gr)) == 152
