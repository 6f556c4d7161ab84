"""Pins of the oracle's optimal densification (Shrivastava, ICML 2017; the
densified variant Sec. 6 says SLASH implements), against properties that do
not come from the oracle's own code."""
import numpy as np
import pytest

import oracle
from test_oracle_pins import _pair

EMPTY = 0xFFFFFFFF


def test_rows_without_empty_bins_are_not_densified():
    """Every bin holds a feature: both rules return the bin minima unchanged,
    and those equal a brute-force minimum per bin."""
    rng = np.random.default_rng(0)
    nb = 32
    for _ in range(20):
        x = rng.choice(1 << 20, size=3000, replace=False).astype(np.uint32)
        a, od, ds = (int(v) for v in rng.integers(0, 1 << 32, 3))
        c1, m1 = oracle.doph(x, nb, a, ds)
        c2, m2 = oracle.doph_opt(x, nb, a, od, ds)
        assert m1.all() and m2.all()
        h = np.array([oracle.mix32(int(f) ^ a) for f in x], dtype=np.uint64)
        b = (h * nb) >> 32
        brute = np.array([h[b == j].min() for j in range(nb)], dtype=np.uint32)
        assert np.array_equal(c1, brute) and np.array_equal(c2, brute)


def test_single_feature_row_and_empty_row():
    """One non-empty bin: every probe sequence ends there, so all codes are that
    feature's hash.  No feature: every code stays empty."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        f = int(rng.integers(0, 1 << 20))
        a, od, ds = (int(v) for v in rng.integers(0, 1 << 32, 3))
        codes, mask = oracle.doph_opt(np.array([f], np.uint32), 96, a, od, ds)
        assert mask.sum() == 1 and np.all(codes == oracle.mix32(f ^ a))
    codes, mask = oracle.doph_opt(np.zeros(0, np.uint32), 64, 1, 2, 3)
    assert not mask.any() and np.all(codes == EMPTY)


@pytest.mark.parametrize("n,s", [(12, 4), (20, 15), (24, 23)])
def test_collision_probability_is_jaccard(n, s):
    """The LSH property survives the densification: every bin, and the densified
    bins on their own, collide with probability J (nb = 64 > n leaves most bins
    of each row empty)."""
    J = s / (2 * n - s)
    nb, T = 64, 1500
    rng = np.random.default_rng(50 + n)
    hits = np.zeros(nb)
    dens_hits = dens = 0
    for _ in range(T):
        x, y = _pair(rng, n, s)
        a, od, ds = (int(v) for v in rng.integers(0, 1 << 32, 3))
        cx, mx = oracle.doph_opt(x, nb, a, od, ds)
        cy, my = oracle.doph_opt(y, nb, a, od, ds)
        eq = cx == cy
        hits += eq
        e = ~mx & ~my
        dens += e.sum()
        dens_hits += (eq & e).sum()
    sd = np.sqrt(J * (1 - J) / T)
    assert np.all(np.abs(hits / T - J) < 5 * sd + 1e-9), (hits / T, J)
    assert abs(hits.mean() / T - J) < 3 * sd
    assert dens > 1000
    assert abs(dens_hits / dens - J) < 5 * np.sqrt(J * (1 - J) / dens)


def test_lower_variance_than_the_side_rule():
    """The result the 2017 paper proves: for sparse rows, estimating J as the
    fraction of equal codes has a smaller mean squared error with optimal
    densification than with the nearest-bin rule (measured about half)."""
    rng = np.random.default_rng(9)
    nb = 128
    for n, s in [(16, 8), (16, 12)]:
        J = s / (2 * n - s)
        e_side, e_opt = [], []
        for _ in range(1500):
            x, y = _pair(rng, n, s)
            a, od, ds = (int(v) for v in rng.integers(0, 1 << 32, 3))
            e_side.append((np.mean(oracle.doph(x, nb, a, ds)[0] == oracle.doph(y, nb, a, ds)[0]) - J) ** 2)
            e_opt.append((np.mean(oracle.doph_opt(x, nb, a, od, ds)[0] ==
                                  oracle.doph_opt(y, nb, a, od, ds)[0]) - J) ** 2)
        assert np.mean(e_opt) < 0.7 * np.mean(e_side), (n, s, np.mean(e_opt), np.mean(e_side))


def test_densified_codes_come_from_non_empty_bins_of_the_row():
    rng = np.random.default_rng(3)
    for _ in range(100):
        x = rng.choice(1 << 20, size=int(rng.integers(1, 40)), replace=False).astype(np.uint32)
        a, od, ds = (int(v) for v in rng.integers(0, 1 << 32, 3))
        codes, mask = oracle.doph_opt(x, 256, a, od, ds)
        assert set(codes.tolist()) <= set(codes[mask].tolist())


def test_index_seeds_keep_the_side_rule_words():
    """The extra seed words follow the existing ones, so densify = 0 indexes
    hash exactly as before."""
    s0 = oracle.derive_seeds(11, 8, 4)["raw"]
    s1 = oracle.seeds_init(11, 8, 4, 1)
    assert np.array_equal(s1[:s0.size], s0) and s1[-1] == 1
    assert s1[-2] == oracle.splitmix64_stream(11, s0.size + 1)[-1] >> 32
