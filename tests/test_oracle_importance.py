"""Pins of importance pruning (Eq. importance) against the paper's Table 3 and invariants.

What each test would catch:
* Table 3 (oracle, n_max <= 4)  a wrong ordering inside the cumulative sums, a missing Re, a
                                hereditary pruning rule, pruning of the n <= 1 levels, a
                                strict in place of a non-strict threshold;
* Table 3 (library host count)  the same in the C++ enumeration, up to n_max = 6 (36.7M);
* worked bosonic example        the bosonic factor (the examples only prune fermions);
* hybrid levels                 pruning of a level (m, n) in {0,1} x {0,1};
* pruned apply = projection     couplings to dropped ADOs kept, or kept couplings lost.
"""
from pathlib import Path

import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv

GOLDEN = Path(__file__).parent / "golden" / "table3_importance_counts.txt"
THRESHOLDS = [1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10, 0.0]


def _table3():
    rows = {}
    for line in GOLDEN.read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x) for x in line.split()]
        rows[v[0]] = v[1:]
    return rows


def _example1_problem(n_max):
    m = W.siam_model(eps=-5.0, U=10.0, Gamma=1.0, W=10.0, kT=0.5, mu=1.0, n_poles=6,
                     tier=n_max)
    return hy.model_to_problem(m)


def test_table3_golden_is_complete():
    t = _table3()
    assert sorted(t) == [1, 2, 3, 4, 5, 6] and all(len(r) == 9 for r in t.values())


@pytest.mark.parametrize("n_max", [1, 2, 3, 4])
def test_oracle_counts_match_table3(n_max):
    prob = _example1_problem(n_max)
    bos, fer = hy.flatten_exponents(prob)
    assert len(fer) == 56 and not bos
    full = hy.problem_hierarchy(prob)
    fe = [(e.coef, e.rate) for e in fer]
    # importance of every ADO once, then the count per threshold
    imp = np.array([np.inf if hy.always_kept(m, S) else hy.importance([], fe, m, S)
                    for (m, S) in full.ados])
    got = [int((imp >= th).sum()) for th in THRESHOLDS]
    assert got == _table3()[n_max]
    # the pruned hierarchy itself at one threshold
    assert hy.prune_hierarchy(full, [], fe, 1e-6).n_ado == _table3()[n_max][3]


def test_library_host_count_matches_table3():
    heom = pytest.importorskip("paper_2306_07522_gb300")
    from paper_2306_07522_gb300 import count_ados
    table = _table3()
    for n_max in range(1, 7):
        prob = _example1_problem(n_max)
        got = [count_ados(prob["baths"], 0, n_max, th) for th in THRESHOLDS]
        assert got == table[n_max], (n_max, got)
    assert heom is not None


def test_bosonic_importance_worked_example():
    # exponents (xi, chi) = (1, 2), (3 + 4i, 5): j listed ascending.
    # m = (2, 0): j = [0, 0]: |1 / (2 * 2)| |1 / (2 * 4)| = 1/32
    # m = (1, 1): j = [0, 1]: |1 / (2 * 2)| |(3 + 4i) / (5 * 7)| = 5/140
    # m = (0, 1) with a fermion (eta, gamma) = (2i, 4 - 1i), q = [0]: |3+4i| / 25 * 2 / 16
    be = [(1.0 + 0j, 2.0 + 0j), (3.0 + 4j, 5.0 + 0j)]
    fe = [(2j, 4.0 - 1j)]
    assert hy.importance(be, [], (2, 0), ()) == pytest.approx(1 / 32, rel=1e-15)
    assert hy.importance(be, [], (1, 1), ()) == pytest.approx(5 / 140, rel=1e-15)
    assert hy.importance(be, fe, (0, 1), (0,)) == pytest.approx(5 / 25 * 2 / 16, rel=1e-15)
    assert hy.importance([(1.0, 0.0 + 1j)], [], (1,), ()) == np.inf  # Re chi = 0


def test_hybrid_low_levels_are_always_kept():
    prob = W.random_raw_problem(3, [("RI", 2)], [4], 3, 2, seed=51)
    prob["importance_th"] = 1e30  # prunes everything that may be pruned
    h = hy.problem_hierarchy(prob)
    levels = {(sum(m), len(S)) for (m, S) in h.ados}
    assert levels == {(0, 0), (0, 1), (1, 0), (1, 1)}
    n_full = hy.problem_hierarchy(dict(prob, importance_th=0.0)).n_ado
    assert h.n_ado == sum(1 for (m, S) in hy.problem_hierarchy(dict(prob, importance_th=0.0)).ados
                          if hy.always_kept(m, S)) < n_full


@pytest.mark.parametrize("parity", [1, -1])
def test_pruned_apply_is_the_projection_of_the_full_apply(parity):
    prob = W.random_raw_problem(3, [("RI", 2), ("I", 1)], [4, 2], 3, 3, parity=parity, seed=52)
    full = hy.problem_hierarchy(prob)
    bos, fer = hy.flatten_exponents(prob)
    be = [(e.coef, e.rate) for e in bos]
    fe = [(e.coef, e.rate) for e in fer]
    imp = sorted(hy.importance(be, fe, m, S) for (m, S) in full.ados if not hy.always_kept(m, S))
    th = imp[len(imp) // 2]  # prunes about half of what may be pruned
    pr = dict(prob, importance_th=th)
    h = hy.problem_hierarchy(pr)
    assert full.n_ado > h.n_ado > 0
    keep = np.array([full.index[a] for a in h.ados])
    X = W.random_ado_vector(h.n_ado, 3, seed=53)
    Xf = np.zeros((full.n_ado, 3, 3), complex)
    Xf[keep] = X
    want = lv.apply_loop(prob, Xf, full)[keep]
    np.testing.assert_allclose(lv.apply_loop(pr, X, h), want, atol=1e-12)
    Y = lv.from_liouville(lv.build_matrix(pr, h) @ lv.to_liouville(X), 3)
    np.testing.assert_allclose(Y, want, atol=1e-12)


@pytest.mark.parametrize("seed", [71, 72])
def test_library_host_count_matches_oracle_hybrid(seed):
    """The library's host count (C++ enumeration and Eq. importance with bosonic R / I / RI
    exponents and fermions) equals the oracle's pruned hierarchy size, at thresholds between
    the oracle's own importance values (decisions far from ties)."""
    pytest.importorskip("paper_2306_07522_gb300")
    from paper_2306_07522_gb300 import count_ados
    prob = W.random_raw_problem(2, [("RI", 2), ("R", 1), ("I", 1)], [4, 2], 3, 3, seed=seed)
    full = hy.problem_hierarchy(prob)
    bos, fer = hy.flatten_exponents(prob)
    be = [(e.coef, e.rate) for e in bos]
    fe = [(e.coef, e.rate) for e in fer]
    imp = np.unique([hy.importance(be, fe, m, S) for (m, S) in full.ados if not hy.always_kept(m, S)])
    assert len(imp) > 20
    for q in (0.1, 0.35, 0.6, 0.9):
        k = int(q * (len(imp) - 1))
        th = float(np.sqrt(imp[k] * imp[k + 1]))  # strictly between two importance values
        want = hy.prune_hierarchy(full, be, fe, th).n_ado
        assert count_ados(prob["baths"], prob["tier_b"], prob["tier_f"], th) == want
    assert count_ados(prob["baths"], prob["tier_b"], prob["tier_f"], 0.0) == full.n_ado


@pytest.mark.parametrize("parity", [1, -1])
def test_pruned_integer_tables_reproduce_the_apply(parity):
    """oracle/tables.py on a pruned hierarchy (entries to dropped ADOs left out): the apply
    from the integer tables equals the loop path, which the projection test above pins."""
    from oracle import tables as tb
    prob = W.random_raw_problem(3, [("RI", 2), ("I", 1)], [4, 2], 3, 3, parity=parity, seed=54)
    full = hy.problem_hierarchy(prob)
    bos, fer = hy.flatten_exponents(prob)
    imp = sorted(hy.importance([(e.coef, e.rate) for e in bos], [(e.coef, e.rate) for e in fer], m, S)
                 for (m, S) in full.ados if not hy.always_kept(m, S))
    pr = dict(prob, importance_th=imp[len(imp) // 3])
    h = hy.problem_hierarchy(pr)
    assert full.n_ado > h.n_ado
    X = W.random_ado_vector(h.n_ado, 3, seed=55)
    Y1 = lv.apply_loop(pr, X, h)
    Y2 = tb.apply_from_tables(pr, X, h)
    assert np.abs(Y1 - Y2).max() <= 1e-13 * np.abs(Y1).max()
    # every table entry points at a kept ADO
    assert all(0 <= nb < h.n_ado for row in tb.neighbour_table(pr, h) for (nb, *_rest) in row)


def test_library_host_count_edge_cases():
    """heom_count_ados (host only): no baths, tier 0, the closed-form full count without a
    threshold, and the refusals (non-finite or negative threshold, negative tier, more than
    64 fermionic exponents)."""
    heom = pytest.importorskip("paper_2306_07522_gb300")
    from paper_2306_07522_gb300 import HeomError, count_ados
    assert count_ados([], 0, 0) == 1
    assert count_ados([], 3, 2) == 1  # tiers without exponents add nothing
    prob = W.random_raw_problem(2, [("RI", 3)], [6], 3, 2, seed=91)
    assert count_ados(prob["baths"], 0, 0) == 1
    assert count_ados(prob["baths"], 3, 2) == hy.ado_count_closed_form(3, 6, 3, 2)
    for th in (float("nan"), -1e-3):
        with pytest.raises(HeomError):
            count_ados(prob["baths"], 3, 2, th)
    with pytest.raises(HeomError):
        count_ados(prob["baths"], -1, 2)
    big = W.random_raw_problem(2, [], [66], 0, 1, seed=92)
    with pytest.raises(HeomError):
        count_ados(big["baths"], 0, 1)
    assert heom is not None
