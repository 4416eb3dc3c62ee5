"""Pins of the oracle's lattice tables against Table I and Eq. (NORM0).

The oracle's constants are checked against the paper's printed rationals
(tests/golden/paper_values.json) and against the exact isotropy identities
they must satisfy; the 4th-moment ratio p/w = 12/7 reproduces Eq. (EFFECTIVE).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _group_of(j):
    if j == 0:
        return "0"
    if j <= 4:
        return "1-4"
    if j <= 8:
        return "5-8"
    if j <= 12:
        return "9-12"
    if j <= 20:
        return "13-20"
    return "21-24"


@pytest.fixture(scope="module")
def tab():
    return oracle.tables()


def test_speeds_are_the_two_belts(tab):
    cx9, cy9, w9, cxf, cyf, pf, wf = tab
    vecs = list(zip(cxf.tolist(), cyf.tolist()))
    assert vecs[0] == (0, 0)
    belt1 = set(vecs[1:9])
    belt2 = set(vecs[9:25])
    assert belt1 == {(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)} - {(0, 0)}
    assert belt2 == {(a, b) for a in range(-2, 3) for b in range(-2, 3) if max(abs(a), abs(b)) == 2}
    # groups of Table I: 1..4 |c|^2 = 1, 5..8 = 2, 9..12 = 4, 13..20 = 5, 21..24 = 8
    sq = [a * a + b * b for a, b in vecs]
    assert sq[1:5] == [1] * 4 and sq[5:9] == [2] * 4 and sq[9:13] == [4] * 4
    assert sq[13:21] == [5] * 8 and sq[21:25] == [8] * 4
    # D2Q9 speeds are belt 1 in the same order, plus rest
    assert list(zip(cx9.tolist(), cy9.tolist())) == vecs[:9]


def test_weights_match_table_I(tab):
    _, _, w9, _, _, pf, wf = tab
    for j in range(25):
        expect = Fraction(GOLD["table_I_p"]["values"][_group_of(j)])
        assert pf[j] == pytest.approx(float(expect), rel=0, abs=1e-16)
    for j in range(9):
        expect = Fraction(GOLD["table_I_w"]["values"][_group_of(j)])
        assert wf[j] == pytest.approx(float(expect), rel=0, abs=1e-16)
        assert w9[j] == pytest.approx(float(expect), rel=0, abs=1e-16)
    assert np.all(wf[9:] == 0.0)


def _moment(weights, cx, cy, a, b, rng):
    return sum(Fraction(weights[_group_of(j)]) * cx[j] ** a * cy[j] ** b for j in rng)


def test_normalisation_and_isotropy_exact(tab):
    """Eq. (NORM0) and the 4th/8th-order isotropy of Sec. II, in exact rationals."""
    _, _, _, cxf, cyf, _, _ = tab
    cx = cxf.tolist()
    cy = cyf.tolist()
    P = GOLD["table_I_p"]["values"]
    W = GOLD["table_I_w"]["values"]
    cs2 = Fraction(GOLD["cs2"]["value"])
    allj = range(25)
    b1 = range(9)
    assert _moment(P, cx, cy, 0, 0, allj) == 1
    assert _moment(W, cx, cy, 0, 0, b1) == 1
    assert _moment(P, cx, cy, 2, 0, allj) == cs2
    assert _moment(W, cx, cy, 2, 0, b1) == cs2
    # 4th-order isotropy: sum c_x^4 = 3 sum c_x^2 c_y^2
    m40 = _moment(P, cx, cy, 4, 0, allj)
    m22 = _moment(P, cx, cy, 2, 2, allj)
    assert m40 == 3 * m22 and m40 == Fraction(4, 7)
    w40 = _moment(W, cx, cy, 4, 0, b1)
    w22 = _moment(W, cx, cy, 2, 2, b1)
    assert w40 == 3 * w22 and w40 == Fraction(1, 3)
    # 6th-order isotropy of the 25-speed set: c_x^6 = 5 c_x^4 c_y^2
    assert _moment(P, cx, cy, 6, 0, allj) == 5 * _moment(P, cx, cy, 4, 2, allj)
    # odd moments vanish
    for a, b in [(1, 0), (0, 1), (3, 0), (1, 2), (2, 1), (5, 0)]:
        assert _moment(P, cx, cy, a, b, allj) == 0
        assert _moment(W, cx, cy, a, b, b1) == 0


def test_fourth_moment_ratio_is_twelve_sevenths(tab):
    """The ratio of 4th moments p/w is the 12/7 of Eq. (EFFECTIVE)."""
    _, _, _, cxf, cyf, _, _ = tab
    cx = cxf.tolist()
    cy = cyf.tolist()
    P = GOLD["table_I_p"]["values"]
    W = GOLD["table_I_w"]["values"]
    ratio = _moment(P, cx, cy, 4, 0, range(25)) / _moment(W, cx, cy, 4, 0, range(9))
    assert ratio == Fraction(GOLD["isotropy_ratio_p_over_w"]["value"])
