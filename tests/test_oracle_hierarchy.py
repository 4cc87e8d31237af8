"""Pins of oracle/hierarchy.py: the paper's Table 3 counts, brute force, canonical order."""
import itertools
import os

import pytest

from oracle import hierarchy as hy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_ado_counts.txt")


def _table3():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            n, c = line.split()
            rows.append((int(n), int(c)))
    return rows


@pytest.mark.parametrize("n_max,count", [r for r in _table3() if r[0] <= 4])
def test_table3_counts_by_enumeration(n_max, count):
    """Example 1: two leads x two spins x two nu x 7 exponents = 56 fermionic exponents."""
    h = hy.build_hierarchy(0, 56, 0, n_max)
    assert h.n_ado == count


@pytest.mark.parametrize("n_max,count", _table3())
def test_table3_counts_closed_form(n_max, count):
    assert hy.ado_count_closed_form(0, 56, 0, n_max) == count


@pytest.mark.parametrize("K_b,K_f,tb,tf,count", [
    (3, 0, 4, 0, 35),      # spin-boson, tier 4
    (0, 24, 0, 2, 301),    # SIAM, tier 2
    (0, 24, 0, 3, 2325),   # SIAM, tier 3
    (0, 24, 0, 4, 12951),  # SIAM, tier 4
    (3, 12, 2, 2, 790),    # charge-cavity, tiers 2 / 2
])
def test_workload_counts(K_b, K_f, tb, tf, count):
    h = hy.build_hierarchy(K_b, K_f, tb, tf)
    assert h.n_ado == count == hy.ado_count_closed_form(K_b, K_f, tb, tf)


def test_bosonic_order_brute_force():
    K, m_max = 3, 3
    brute = [m for m in itertools.product(range(m_max + 1), repeat=K) if sum(m) <= m_max]
    brute.sort(key=lambda m: (sum(m), tuple(-v for v in m)))
    assert hy.bosonic_occupations(K, m_max) == brute
    assert hy.bosonic_occupations(K, 1) == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def test_fermionic_order_brute_force():
    K, n_max = 5, 3
    brute = [tuple(i for i in range(K) if bits >> i & 1) for bits in range(1 << K)]
    brute = [s for s in brute if len(s) <= n_max]
    brute.sort(key=lambda s: (len(s), s))
    assert hy.fermionic_subsets(K, n_max) == brute


def test_mixed_index_is_bosonic_major():
    h = hy.build_hierarchy(2, 3, 1, 2)
    nf = len(h.fer)
    for i, (m, S) in enumerate(h.ados):
        assert h.bos.index(m) * nf + h.fer.index(S) == i
        assert h.index[(m, S)] == i
