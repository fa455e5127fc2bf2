"""Pins of the oracle's lambda_min estimate (Sec. IV-C-2, Eq.
formula_courant-fischer-3) to values fixed by hand and by closed forms.

The estimate is min over nodes p of L_G(p,p) / L_S(p,p), the weighted degrees
of the two Laplacians (the diagonal load D belongs to neither).  It is an
upper bound of the true lambda_min of the pencil (L_G, L_S): the ratio at p
is the generalized Rayleigh quotient of the indicator vector of p.

Can the bound be attained with lambda_min > 1?  No: if e_p (modulo the
all-ones vector) is a generalized eigenvector, then comparing the entries
of L_G e_p = lambda L_S e_p + c 1 at p's neighbours either forces every
edge at p into S (then the ratio at p is 1) or gives lambda < 1, which a
subgraph S of G cannot have.  So the attained case is lambda_min = 1, and
the hand-derived cases below pin the estimate's value where it is strictly
above the true lambda_min.

`_pin_failures` runs every pin against a candidate implementation; the last
test plants plausible mistakes (max for min, D added to the diagonals, the
ratio inverted, S's degrees taken over all edges) in copies of the estimate
and checks that each one fails some pin.
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth import graphs
from tests.helpers import dense_lap, gen_eigs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lambda_min_hand.json")


def _cases():
    return json.load(open(GOLDEN))["cases"]


def _build(case):
    e = np.array(case["edges"], dtype=np.float64)
    u, v, w = e[:, 0].astype(np.int64), e[:, 1].astype(np.int64), e[:, 2]
    rp, col, val = graphs.csr_from_edges(case["n"], u, v, w, np.array(case["D"]))
    g = graphs.Graph(case["name"], case["n"], rp, col, val)
    og = oracle.from_graph(g)
    mask = np.zeros(og.m, np.uint8)
    for a, b in case["s_edges"]:
        k = np.flatnonzero((og.eu == min(a, b)) & (og.ev == max(a, b)))
        assert k.shape[0] == 1
        mask[k[0]] = 1
    return og, mask


def _kn_path(n):
    """K_n with unit weights; S = the path 0-1-...-(n-1)."""
    iu = np.triu_indices(n, 1)
    rp, col, val = graphs.csr_from_edges(n, iu[0], iu[1], np.ones(iu[0].shape[0]), 0.0)
    og = oracle.from_graph(graphs.Graph(f"K{n}", n, rp, col, val))
    mask = ((og.ev - og.eu) == 1).astype(np.uint8)
    return og, mask


def _pin_failures(fn):
    """Names of the pins that estimate function fn(og, mask) fails."""
    bad = []
    for case in _cases():
        og, mask = _build(case)
        est = fn(og, mask)
        if est != pytest.approx(case["expected"], rel=1e-15, abs=0):
            bad.append(f"hand value: {case['name']}")
        lam = gen_eigs(dense_lap(og.n, og.eu, og.ev, og.ew),
                       dense_lap(og.n, og.eu, og.ev, og.ew, mask))
        if est < lam.min() * (1 - 1e-12):
            bad.append(f"upper bound: {case['name']}")
        if est < 1.0 - 1e-15:
            bad.append(f">= 1: {case['name']}")
    for n in range(4, 11):
        og, mask = _kn_path(n)
        est = fn(og, mask)
        # inner path nodes: degree n-1 in K_n, 2 in the path
        if est != pytest.approx((n - 1) / 2.0, rel=1e-15, abs=0):
            bad.append(f"K{n}/path closed form")
    return bad


def test_hand_derived_values():
    for case in _cases():
        og, mask = _build(case)
        est = oracle.lambda_min_est(og, mask)
        num, den = case["expected_fraction"]
        assert est == pytest.approx(num / den, rel=1e-15, abs=0), case["name"]
        assert est != pytest.approx(case["with_D_included"], rel=1e-6) or case["D"] == [0.0] * og.n
        if case["max_ratio"] != case["expected"]:
            assert est < case["max_ratio"]


def test_estimate_bounds_and_attains_true_lambda_min():
    for case in _cases():
        og, mask = _build(case)
        est = oracle.lambda_min_est(og, mask)
        lam = gen_eigs(dense_lap(og.n, og.eu, og.ev, og.ew),
                       dense_lap(og.n, og.eu, og.ev, og.ew, mask))
        assert est >= lam.min() * (1 - 1e-12)
        if "true_lambda_min" in case:
            assert lam.min() == pytest.approx(case["true_lambda_min"], rel=1e-12)
            if case["true_lambda_min"] == 1.0:
                assert est == 1.0            # attained: a node keeps all its edges in S


@pytest.mark.parametrize("n", [4, 5, 7, 10])
def test_complete_graph_with_path_closed_form(n):
    og, mask = _kn_path(n)
    est = oracle.lambda_min_est(og, mask)
    assert est == (n - 1) / 2.0
    # true lambda_min = n / (largest path eigenvalue 2 + 2 cos(pi/n)) < estimate
    lam = gen_eigs(dense_lap(n, og.eu, og.ev, og.ew), dense_lap(n, og.eu, og.ev, og.ew, mask))
    closed = n / (2.0 + 2.0 * np.cos(np.pi / n))
    assert lam.min() == pytest.approx(closed, rel=1e-12)
    assert est > closed


def test_oracle_passes_every_pin():
    assert _pin_failures(oracle.lambda_min_est) == []


def _degrees(og, mask=None):
    s = np.ones(og.m, bool) if mask is None else mask.astype(bool)
    return (np.bincount(og.eu[s], og.ew[s], og.n) + np.bincount(og.ev[s], og.ew[s], og.n))


def test_planted_mistakes_fail_a_pin():
    mutants = {
        "max instead of min": lambda og, m: float(np.max(_degrees(og) / _degrees(og, m))),
        "D added to both diagonals":
            lambda og, m: float(np.min((_degrees(og) + og.D) / (_degrees(og, m) + og.D))),
        "ratio inverted": lambda og, m: float(np.min(_degrees(og, m) / _degrees(og))),
        "S degrees over all edges": lambda og, m: float(np.min(_degrees(og) / _degrees(og))),
        "only u endpoints counted": lambda og, m: float(np.min(
            (np.bincount(og.eu, og.ew, og.n) + 1e-300)
            / (np.bincount(og.eu[m.astype(bool)], og.ew[m.astype(bool)], og.n) + 1e-300))),
    }
    for name, fn in mutants.items():
        with np.errstate(divide="ignore", invalid="ignore"):
            assert _pin_failures(fn), f"planted mistake not caught: {name}"
