"""ADO enumeration, canonical order and raw-problem assembly (oracle).

Paper passages followed:
* Eq. HEOM and the multi-index notation below it: an ADO rho^{(m,n,p)}_{j|q} carries a
  bosonic vector j = [j_m..j_1] (a multiset: j' may repeat an element already in j) and a
  fermionic vector q = [q_n..q_1] (a set: q' not in q, Pauli exclusion). Truncation at
  tiers m_max, n_max.
* Results, "Preliminaries": a bosonic exponent is the ensemble {beta, u, l, sigma_b}, a
  fermionic one {alpha, nu, h, sigma_f}.

The paper leaves the order of the ADOs free. The canonical order fixed here (and reproduced
bit-exactly by the GPU path) is:
* exponents: bath order of the call, then the order within the bath;
* bosonic part: occupation vectors m with |m| <= m_max, by tier |m| ascending, then
  lexicographically descending in (m_1, ..., m_K) (tier 1 is e_1, e_2, ...);
* fermionic part: subsets S of {0..K_f-1}, |S| <= n_max, by size ascending, then
  lexicographically ascending as sorted tuples;
* mixed index = bosonic index * N_f + fermionic index.
The enumeration below is a plain recursive construction; the index map is a dictionary.

Importance pruning (Eq. importance and the paragraph around it): an ADO's importance is
  I = |prod_{r=1..m} xi_{j_r} / (Re chi_{j_r} sum_{x<=r} Re chi_{j_x})|
    x |prod_{w=1..n} eta_{q_w} / (Re gamma_{q_w} sum_{x<=w} Re gamma_{q_x})|,
and every ADO outside the levels (m, n) in {0, 1} x {0, 1} with I < I_th is dropped.
Readings: the paper does not fix the order of j and q inside the cumulative sums; listing
them by ascending exponent index (the canonical exponent order) reproduces every entry of
Table 3. Pruning is per ADO (not hereditary): a kept ADO keeps its equation, and the terms
that couple it to dropped ADOs vanish (a dropped ADO is zero). A zero denominator (an
undamped exponent) makes the importance infinite: the ADO is kept.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

from . import exponents as ex


def bosonic_occupations(K: int, m_max: int):
    """All m in N^K with |m| <= m_max: tier ascending, then lexicographically descending."""
    out = []
    for t in range(m_max + 1):
        if K == 0:
            if t == 0:
                out.append(())
            continue

        def rec(prefix, remaining, slots):
            if slots == 1:
                out.append(prefix + (remaining,))
                return
            for v in range(remaining, -1, -1):
                rec(prefix + (v,), remaining - v, slots - 1)

        rec((), t, K)
    return out


def fermionic_subsets(K: int, n_max: int):
    """All subsets of {0..K-1} with at most n_max elements: size ascending, then lex ascending."""
    out = []
    for n in range(min(n_max, K) + 1):
        out.extend(itertools.combinations(range(K), n))
    return out


@dataclass
class Hierarchy:
    """ADO list and dictionary (the paper's "hierarchy dictionary", Fig. 1e)."""

    K_b: int
    K_f: int
    tier_b: int
    tier_f: int
    bos: list
    fer: list
    ados: list  # list of (m tuple, S tuple)
    index: dict  # (m, S) -> ADO index

    @property
    def n_ado(self) -> int:
        return len(self.ados)


def build_hierarchy(K_b: int, K_f: int, tier_b: int, tier_f: int) -> Hierarchy:
    bos = bosonic_occupations(K_b, tier_b)
    fer = fermionic_subsets(K_f, tier_f)
    ados = [(m, S) for m in bos for S in fer]
    index = {a: i for i, a in enumerate(ados)}
    return Hierarchy(K_b, K_f, tier_b, tier_f, bos, fer, ados, index)


def importance(bos_exps, fer_exps, m, S) -> float:
    """Eq. importance of the ADO (m, S); bos_exps / fer_exps are (coef, rate) lists in the
    global exponent order, m an occupation vector, S a sorted tuple."""
    val = 1.0
    cum = 0.0
    for k, mk in enumerate(m):  # bosonic multiset j listed by ascending exponent index
        for _ in range(mk):
            xi, chi = bos_exps[k]
            cum += chi.real
            den = chi.real * cum
            if den == 0.0:
                return np.inf
            val *= abs(xi / den)
    cum = 0.0
    for q in S:  # fermionic set q listed by ascending exponent index
        eta, gam = fer_exps[q]
        cum += gam.real
        den = gam.real * cum
        if den == 0.0:
            return np.inf
        val *= abs(eta / den)
    return val


def always_kept(m, S) -> bool:
    """Levels (m, n) in {0, 1} x {0, 1} are never pruned."""
    return sum(m) <= 1 and len(S) <= 1


def prune_hierarchy(hier: Hierarchy, bos_exps, fer_exps, importance_th: float) -> Hierarchy:
    """The ADOs of hier whose importance is >= importance_th (or that are always kept), in
    the canonical order."""
    ados = [(m, S) for (m, S) in hier.ados
            if always_kept(m, S) or importance(bos_exps, fer_exps, m, S) >= importance_th]
    index = {a: i for i, a in enumerate(ados)}
    return Hierarchy(hier.K_b, hier.K_f, hier.tier_b, hier.tier_f, hier.bos, hier.fer, ados,
                     index)


def ado_count_closed_form(K_b: int, K_f: int, tier_b: int, tier_f: int) -> int:
    """C(K_b + m_max, m_max) * sum_{n <= n_max} C(K_f, n) (stars and bars; subsets)."""
    from math import comb

    nb = comb(K_b + tier_b, tier_b) if K_b > 0 else 1
    nf = sum(comb(K_f, n) for n in range(min(tier_f, K_f) + 1))
    return nb * nf


# --------------------------------------------------------------------------------------
# Raw problem: the HEOM inputs with exponents (Fig. 1a-b: "a list of exponents").
# --------------------------------------------------------------------------------------


def model_to_problem(model, parity: int = 1) -> dict:
    """Turn a physical model (workloads.Model) into the raw exponent form.

    Bosonic Drude-Lorentz baths become one combined "RI" bath each (real chi). Each
    fermionic lead on operator d becomes one bath holding nu=+1 exponents h=1..H then nu=-1
    exponents h=1..H; the partner of (nu, h) is (-nu, h).
    """
    baths = []
    for V, p in model.boson_baths:
        xi, chi = ex.drude_lorentz_exponents(p.lam, p.W, p.kT, p.n_poles, p.method)
        baths.append(dict(kind="RI", op=np.asarray(V, np.complex128), coef=xi, rate=chi))
    for dop, p in model.fermion_baths:
        ep, gp = ex.lorentz_fermion_exponents(p.Gamma, p.W, p.mu, p.kT, p.n_poles, p.method, +1)
        em, gm = ex.lorentz_fermion_exponents(p.Gamma, p.W, p.mu, p.kT, p.n_poles, p.method, -1)
        h = len(ep)
        baths.append(dict(kind="F", op=np.asarray(dop, np.complex128),
                          coef=np.concatenate([ep, em]), rate=np.concatenate([gp, gm]),
                          nu=np.array([1] * h + [-1] * h, dtype=np.int32),
                          partner=np.array(list(range(h, 2 * h)) + list(range(h)),
                                           dtype=np.int32)))
    return dict(d=model.d, H=np.asarray(model.H, np.complex128), baths=baths,
                tier_b=model.tier_b, tier_f=model.tier_f, parity=parity,
                lindblad=[dict(op=np.asarray(F, np.complex128), rate=float(g))
                          for F, g in model.lindblad])


@dataclass
class Exponent:
    """One exponent of the global list (bath order, then order within the bath)."""

    bath: int
    kind: str  # "R", "I", "RI" (bosonic) or "F"
    op: np.ndarray
    coef: complex
    rate: complex
    nu: int = 0
    partner_coef: complex = 0j  # fermionic: eta of the partner exponent (same alpha, h; -nu)


def flatten_exponents(problem: dict):
    """Split the bath list into the global bosonic and fermionic exponent lists."""
    bos, fer = [], []
    for b, bath in enumerate(problem["baths"]):
        kind = bath["kind"]
        for k in range(len(bath["coef"])):
            if kind == "F":
                fer.append(Exponent(b, kind, bath["op"], complex(bath["coef"][k]),
                                    complex(bath["rate"][k]), int(bath["nu"][k]),
                                    complex(bath["coef"][bath["partner"][k]])))
            else:
                bos.append(Exponent(b, kind, bath["op"], complex(bath["coef"][k]),
                                    complex(bath["rate"][k])))
    return bos, fer


def problem_hierarchy(problem: dict) -> Hierarchy:
    """The problem's hierarchy; pruned when it carries importance_th > 0."""
    bos, fer = flatten_exponents(problem)
    h = build_hierarchy(len(bos), len(fer), problem["tier_b"], problem["tier_f"])
    th = float(problem.get("importance_th", 0.0))
    if th > 0.0:
        h = prune_hierarchy(h, [(e.coef, e.rate) for e in bos], [(e.coef, e.rate) for e in fer],
                            th)
    return h
