"""Neighbour and sign tables of M in integer form (oracle).

Each term of Eq. HEOM for a target ADO i is written as
    (M X)_i += -i ( mult_l * a * O X_nb + mult_r * b * X_nb O )
with the integers carrying the tier multiplicity, the parity sign (-1)^{delta_{p,-}}, the
ordering sign eps(q, S) and the P_s sign sigma = p (-1)^n; (a, b, O) depend only on the
exponent k and the direction (dir = +1: raised neighbour, a = b = 1; dir = -1: lowered).
In a pruned hierarchy (Eq. importance) an entry whose neighbour was dropped is left out.
These are the integer tables the GPU path must reproduce bit for bit. ``apply_from_tables``
evaluates M from them, which the tests pin against the two paths of liouvillian.py.
"""
from __future__ import annotations

import numpy as np

from .hierarchy import flatten_exponents, problem_hierarchy
from .liouvillian import boson_lower_coefs, damping, op_power, ordering_sign


def neighbour_table(problem: dict, hier=None):
    """List per ADO of (nb, k, dir, mult_l, mult_r); k global (bosonic first)."""
    p = problem["parity"]
    bos, fer = flatten_exponents(problem)
    hier = hier or problem_hierarchy(problem)
    Kb = len(bos)
    table = []
    for (m, S) in hier.ados:
        n = len(S)
        sigma = p * (-1) ** n
        rows = []

        def add(key, *rest):
            j = hier.index.get(key)
            if j is not None:  # a pruned neighbour contributes no entry
                rows.append((j,) + rest)

        if sum(m) < hier.tier_b:
            for k in range(Kb):
                mu = list(m)
                mu[k] += 1
                add((tuple(mu), S), k, 1, 1, -1)
        for k in range(Kb):
            if m[k] > 0:
                md = list(m)
                md[k] -= 1
                add((tuple(md), S), k, -1, m[k], -m[k])
        for q in range(len(fer)):
            eps = ordering_sign(q, S)
            if q in S:
                Sq = tuple(r for r in S if r != q)
                add((m, Sq), Kb + q, -1, p * eps, p * eps * sigma)
            elif n < hier.tier_f:
                Sq = tuple(sorted(S + (q,)))
                add((m, Sq), Kb + q, 1, p * eps, -p * eps * sigma)
        table.append(rows)
    return table


def apply_from_tables(problem: dict, X: np.ndarray, hier=None, table=None) -> np.ndarray:
    """M X evaluated term by term from the integer tables."""
    H = problem["H"]
    bos, fer = flatten_exponents(problem)
    hier = hier or problem_hierarchy(problem)
    table = table or neighbour_table(problem, hier)
    Kb = len(bos)
    Y = np.empty_like(X)
    for i, (m, S) in enumerate(hier.ados):
        acc = -1j * (H @ X[i] - X[i] @ H) - damping(m, S, bos, fer) * X[i]
        for nb, k, dr, ml, mr in table[i]:
            if k < Kb:
                e = bos[k]
                O = e.op
                a, b = (1, 1) if dr > 0 else boson_lower_coefs(e.kind, e.coef)
            else:
                e = fer[k - Kb]
                O = op_power(e.op, -e.nu if dr > 0 else e.nu)
                a, b = (1, 1) if dr > 0 else (e.coef, np.conj(e.partner_coef))
            acc = acc - 1j * (ml * a * (O @ X[nb]) + mr * b * (X[nb] @ O))
        Y[i] = acc
    return Y
