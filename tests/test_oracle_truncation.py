"""Pins of the oracle's truncation rule (oracle/dmrgu1.py select_kept).

The rule (a reading of the Numerical procedure section, which fixes the bond
dimension but not the handling of equal weights): keep the D largest
density-matrix weights across sectors; weights at or below the rounding floor
1e-14 are never kept; weights equal to 1e-8 relative that straddle the cut are
dropped together, so that the kept set never depends on rounding. Each case
below is built by hand so that the kept set is known without running the rule,
and a plausible slip (a sort in the wrong direction, a tie kept half-way, the
floor applied as >= or not at all, the discarded weight counted from the kept
states) fails one of them.
"""
import numpy as np

from oracle.dmrgu1 import TIE_REL, WEIGHT_FLOOR, select_kept


def _blocks(weights):
    """{label: weights} -> the select_kept input with singular values sqrt(w)."""
    out = {}
    for qn, ws in weights.items():
        sv = np.sqrt(np.asarray(ws, float))
        n = len(sv)
        out[qn] = (np.arange(n), np.arange(n), np.eye(n), sv, np.eye(n))
    return out


def _kept_weights(weights, kept):
    return sorted(w for qn, ks in kept.items() for k, w in enumerate(weights[qn]) if k in ks)


def test_spin_flip_pair_straddling_the_cut_is_dropped_together():
    # sectors 2Sz = +1 and -1 carry the same weight 0.2 (spin-flip symmetry); with
    # D = 2 the cut falls between them: both go, only the 0.5 state stays
    w = {(3, 1): [0.2], (3, -1): [0.2], (2, 0): [0.5, 0.1]}
    kept, disc = select_kept(_blocks(w), 2)
    assert kept == {(2, 0): [0]}
    assert abs(disc - 0.5) < 1e-15
    # D = 3: the pair is inside, kept together
    kept, disc = select_kept(_blocks(w), 3)
    assert _kept_weights(w, kept) == [0.2, 0.2, 0.5]
    assert abs(disc - 0.1) < 1e-15


def test_near_tie_within_tie_width_is_a_tie_and_outside_is_not():
    lam = 0.2
    inside = lam * (1 - 0.5 * TIE_REL)
    outside = lam * (1 - 4 * TIE_REL)
    kept, _ = select_kept(_blocks({(1, 1): [0.6, lam], (1, -1): [inside]}), 2)
    assert _kept_weights({(1, 1): [0.6, lam], (1, -1): [inside]}, kept) == [0.6]
    w = {(1, 1): [0.6, lam], (1, -1): [outside]}
    kept, disc = select_kept(_blocks(w), 2)
    assert _kept_weights(w, kept) == [lam, 0.6]
    assert abs(disc - outside) < 1e-15


def test_weights_at_the_rounding_floor_are_never_kept():
    w = {(0, 0): [0.9, 0.1 - 2e-15], (2, 0): [WEIGHT_FLOOR], (4, 0): [1e-15]}
    kept, disc = select_kept(_blocks(w), 100)
    assert kept == {(0, 0): [0, 1]}
    assert abs(disc - (WEIGHT_FLOOR + 1e-15)) < 1e-20
    # just above the floor is kept
    w2 = {(0, 0): [0.9], (2, 0): [2 * WEIGHT_FLOOR]}
    kept, _ = select_kept(_blocks(w2), 100)
    assert kept == {(0, 0): [0], (2, 0): [0]}


def test_kept_plus_discarded_is_the_total_and_matches_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(20):
        labels = [(n, s) for n in range(3) for s in (-1, 1)]
        w = {qn: list(rng.random(rng.integers(1, 5))) for qn in labels}
        tot = sum(sum(v) for v in w.values())
        w = {qn: [x / tot for x in v] for qn, v in w.items()}
        D = int(rng.integers(1, 12))
        kept, disc = select_kept(_blocks(w), D)
        flat = sorted((x for v in w.values() for x in v), reverse=True)
        # distinct random weights: the D largest, nothing else
        assert _kept_weights(w, kept) == sorted(flat[:D])
        assert abs(sum(_kept_weights(w, kept)) + disc - 1.0) < 1e-13
        for qn, ks in kept.items():
            assert ks == sorted(set(ks))


# Dynamic block-state selection (dbss_bond_dimension): the smallest D in
# [D_min, D_max] whose tail of weights beyond the D largest is at most eps.
def test_dbss_picks_the_smallest_bond_dimension_within_the_error():
    from oracle.dmrgu1 import dbss_bond_dimension
    # weights 0.5, 0.3 | 0.15 | 0.04, 0.01 over three sectors; tails after D = 1..5:
    # 0.5, 0.2, 0.05, 0.01, 0
    w = {(2, 0): [0.5, 0.04], (3, 1): [0.3, 0.01], (1, 1): [0.15]}
    b = _blocks(w)
    assert dbss_bond_dimension(b, 0.05 + 1e-15, 1, 10) == 3
    assert dbss_bond_dimension(b, 0.049, 1, 10) == 4
    assert dbss_bond_dimension(b, 0.6, 1, 10) == 1
    assert dbss_bond_dimension(b, 1e-6, 1, 10) == 5
    # bounds: D_min raises it, D_max caps it
    assert dbss_bond_dimension(b, 0.6, 4, 10) == 4
    assert dbss_bond_dimension(b, 1e-6, 1, 2) == 2
    # the selection with that D discards at most eps (no ties here)
    for eps in (0.3, 0.2, 0.05 + 1e-15, 0.011, 1e-3):
        kept, disc = select_kept(b, dbss_bond_dimension(b, eps, 1, 10))
        assert disc <= eps
        # and one state fewer would discard more than eps
        n = sum(len(v) for v in kept.values())
        if n > 1:
            _, disc1 = select_kept(b, n - 1)
            assert disc1 > eps
