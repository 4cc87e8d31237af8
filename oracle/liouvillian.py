"""The HEOM Liouvillian superoperator M (oracle, FP64), written out twice.

Paper passage: Eq. HEOM and the definitions that follow it:

  d/dt rho^{(m,n,p)}_{j|q} = -(i L_s + sum_r chi_{j_r} + sum_w gamma_{q_w}) rho
      - i sum_{q' not in q} A_{q'} rho^{(m,n+1,p)}_{j|q+}  - i sum_{j'} B_{j'} rho^{(m+1,n,p)}_{j+|q}
      - i sum_w (-1)^{n-w} C_{q_w} rho^{(m,n-1,p)}_{j|q_w^-} - i sum_r D_{j_r} rho^{(m-1,n,p)}_{j_r^-|q}

  A_q[.] = (-1)^{delta_{p,-}} { d^{nubar} [.] - P_s[[.] d^{nubar}] }
  C_q[.] = (-1)^{delta_{p,-}} { eta^{nu} d^{nu} [.] + (eta^{nubar})^* P_s[[.] d^{nu}] }
  B_j[.] = [V, .]
  D_j[.] = delta_{u,R} xi^R [V, .] + i delta_{u,I} xi^I {V, .}
  P_s[rho^{(m,n,+-)} d] = -+ (-1)^n rho^{(m,n,+-)} d,   L_s[.] = [H_s, .]

Readings (the paper fixes the operators but not an ADO order or a storage convention):
* ADOs are stored for sorted fermionic index sets S (canonical order, see hierarchy.py).
  The vector q = [q_n..q_1] lists S ascending from left to right. Then the prepended q'
  of q+ and the (-1)^{n-w} of the removal both reduce to
  eps(q, S) = (-1)^{#{r in S : r < q}}.
* The sign of P_s is evaluated from the tier of the ADO it acts on (n+1 for A, n-1 for C);
  in both cases it equals -sigma with sigma = p (-1)^n and n the tier of the ADO being
  updated, so A X = s_p (O X - sigma X O) and C X = s_p (eta O X + sigma eta_bar^* X O)
  with s_p = (-1)^{delta_{p,-}} = p.
* Bosonic multisets are stored as occupation vectors m: the raising sum over j' has one
  term per exponent k, the lowering sum over r has m_k equal terms for exponent k.
* A bosonic exponent of kind "RI" has real rate and stands for both parts of Eq.
  C_beta_RI at once: D X = Re(xi) [V, X] + i Im(xi) {V, X}.
* d^{+1} = d^dagger (nu = +1: Hermitian conjugation present), d^{-1} = d.
* No normalisation factors on the ADOs (the unnormalised form of Eq. HEOM).

Lindblad terms (Eq. Lindbladian): a problem may carry a list ``lindblad`` of jump operators
F_k with real rates gamma_k. The term sum_k gamma_k J(F_k)[X], J(F)[X] = F X F^dagger -
1/2 (F^dagger F X + X F^dagger F), is added to the equation of every ADO X, leaving the ADO set
unchanged (Results: the Lindbladian is added to the HEOMLS without extending the ADO space).
Reading: the paper gives the one form for every ADO and both parities, so no tier- or
parity-dependent sign is applied.

Pruned hierarchies (Eq. importance; hierarchy.prune_hierarchy): the terms that couple a kept
ADO to a dropped one are left out, a dropped ADO being zero.

Liouville space convention of the sparse path: column stacking, vec(A X B) =
(B^T kron A) vec(X); the ADO vector is the concatenation of vec(rho_n) in ADO order.
The loop path works on an array X[n] of d x d matrices (the GPU path's row-major layout).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .hierarchy import flatten_exponents, problem_hierarchy


def op_power(op: np.ndarray, nu: int) -> np.ndarray:
    """d^{nu}: d^{+1} = d^dagger, d^{-1} = d (Results, definition of nu)."""
    return op.conj().T if nu == 1 else op


def boson_lower_coefs(kind: str, c: complex):
    """(a, b) with D X = a V X - b X V for one bosonic exponent (definition of D_j)."""
    if kind == "R":
        return c, c
    if kind == "I":
        return 1j * c, -1j * c
    if kind == "RI":
        return c, np.conj(c)
    raise ValueError(kind)


def ordering_sign(q: int, S) -> int:
    """eps(q, S) = (-1)^{#{r in S : r < q}}."""
    return -1 if sum(1 for r in S if r < q) % 2 else 1


def damping(m, S, bos, fer) -> complex:
    """sum_r chi_{j_r} + sum_w gamma_{q_w} for the ADO (m, S)."""
    return sum(mk * e.rate for mk, e in zip(m, bos)) + sum(fer[q].rate for q in S)


# --------------------------------------------------------------------------------------
# Path 1: per-ADO loop with dense d x d products, on X[n] (shape (N, d, d)).
# --------------------------------------------------------------------------------------


def lindblad_terms(problem: dict):
    """The (gamma, F) pairs of the problem's Lindblad terms (empty list when it has none)."""
    return [(float(t["rate"]), np.asarray(t["op"], np.complex128))
            for t in problem.get("lindblad", [])]


def lindblad_apply(terms, X0: np.ndarray) -> np.ndarray:
    """sum_k gamma_k J(F_k)[X0] with J(F)[X] = F X F^dagger - 1/2 {F^dagger F, X}
    (Eq. Lindbladian)."""
    out = np.zeros_like(X0)
    for g, F in terms:
        Fd = F.conj().T
        FdF = Fd @ F
        out += g * (F @ X0 @ Fd - 0.5 * (FdF @ X0 + X0 @ FdF))
    return out


def apply_loop(problem: dict, X: np.ndarray, hier=None, only=None) -> np.ndarray:
    """Y = M X computed ADO by ADO from Eq. HEOM (target-ADO view).

    ``only``: optional list of ADO indices; then only those blocks of Y are computed (the
    others stay zero), which lets a test sample very large hierarchies.
    """
    H = problem["H"]
    p = problem["parity"]
    bos, fer = flatten_exponents(problem)
    hier = hier or problem_hierarchy(problem)
    lind = lindblad_terms(problem)
    Y = np.zeros_like(X)
    targets = range(hier.n_ado) if only is None else only
    for i in targets:
        m, S = hier.ados[i]
        n = len(S)
        X0 = X[i]
        acc = -1j * (H @ X0 - X0 @ H) - damping(m, S, bos, fer) * X0
        if lind:
            acc += lindblad_apply(lind, X0)
        if sum(m) < hier.tier_b:
            for k, e in enumerate(bos):
                mu = list(m)
                mu[k] += 1
                j = hier.index.get((tuple(mu), S))
                if j is None:  # pruned neighbour (zero)
                    continue
                Xn = X[j]
                acc += -1j * (e.op @ Xn - Xn @ e.op)
        for k, e in enumerate(bos):
            if m[k] > 0:
                md = list(m)
                md[k] -= 1
                j = hier.index.get((tuple(md), S))
                if j is None:
                    continue
                Xn = X[j]
                a, b = boson_lower_coefs(e.kind, e.coef)
                acc += -1j * m[k] * (a * (e.op @ Xn) - b * (Xn @ e.op))
        sigma = p * (-1) ** n
        if n < hier.tier_f:
            for q in range(hier.K_f):
                if q in S:
                    continue
                Sq = tuple(sorted(S + (q,)))
                j = hier.index.get((m, Sq))
                if j is None:
                    continue
                Xn = X[j]
                O = op_power(fer[q].op, -fer[q].nu)
                acc += -1j * p * ordering_sign(q, S) * (O @ Xn - sigma * (Xn @ O))
        for q in S:
            Sq = tuple(r for r in S if r != q)
            j = hier.index.get((m, Sq))
            if j is None:
                continue
            Xn = X[j]
            O = op_power(fer[q].op, fer[q].nu)
            acc += -1j * p * ordering_sign(q, S) * (
                fer[q].coef * (O @ Xn) + sigma * np.conj(fer[q].partner_coef) * (Xn @ O))
        Y[i] = acc
    return Y


# --------------------------------------------------------------------------------------
# Path 2: explicit sparse matrix in Liouville space, assembled edge by edge.
# --------------------------------------------------------------------------------------


def spre(A: np.ndarray):
    return sp.kron(sp.identity(A.shape[0], format="csr"), sp.csr_matrix(A), format="csr")


def spost(B: np.ndarray):
    return sp.kron(sp.csr_matrix(B.T), sp.identity(B.shape[0], format="csr"), format="csr")


def build_matrix(problem: dict, hier=None) -> sp.csr_matrix:
    """M as an (N d^2) x (N d^2) CSR matrix.

    Every raising edge (m,S) -> (m+e_k,S) or (m,S) -> (m,S+{q}) is visited once and fills
    both blocks it creates: the raising term (B or A) in the row of the lower ADO and the
    lowering term (D or C) in the row of the upper ADO.
    """
    d = problem["d"]
    H = problem["H"]
    p = problem["parity"]
    bos, fer = flatten_exponents(problem)
    hier = hier or problem_hierarchy(problem)
    D2 = d * d
    N = hier.n_ado
    rows, cols, vals = [], [], []

    def put(i, j, block):
        block = sp.coo_matrix(block)
        rows.append(block.row + i * D2)
        cols.append(block.col + j * D2)
        vals.append(block.data)

    LH = -1j * (spre(H) - spost(H))
    for g, F in lindblad_terms(problem):
        # vec(F X F^dagger) = (conj(F) kron F) vec(X) = spost(F^dagger) spre(F) vec(X)
        Fd = F.conj().T
        FdF = Fd @ F
        LH = LH + g * (spre(F) @ spost(Fd) - 0.5 * (spre(FdF) + spost(FdF)))
    eye = sp.identity(D2, format="csr")
    for i, (m, S) in enumerate(hier.ados):
        put(i, i, LH - damping(m, S, bos, fer) * eye)
    for i, (m, S) in enumerate(hier.ados):
        n = len(S)
        if sum(m) < hier.tier_b:
            for k, e in enumerate(bos):
                mu = list(m)
                mu[k] += 1
                j = hier.index.get((tuple(mu), S))
                if j is None:  # pruned neighbour: both blocks of the edge vanish
                    continue
                put(i, j, -1j * (spre(e.op) - spost(e.op)))
                a, b = boson_lower_coefs(e.kind, e.coef)
                put(j, i, -1j * mu[k] * (a * spre(e.op) - b * spost(e.op)))
        if n < hier.tier_f:
            for q in range(hier.K_f):
                if q in S:
                    continue
                j = hier.index.get((m, tuple(sorted(S + (q,)))))
                if j is None:
                    continue
                eps = ordering_sign(q, S)
                sig_i = p * (-1) ** n
                sig_j = p * (-1) ** (n + 1)
                O = op_power(fer[q].op, -fer[q].nu)
                put(i, j, -1j * p * eps * (spre(O) - sig_i * spost(O)))
                Od = op_power(fer[q].op, fer[q].nu)
                put(j, i, -1j * p * eps * (fer[q].coef * spre(Od)
                                            + sig_j * np.conj(fer[q].partner_coef) * spost(Od)))
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N * D2, N * D2))
    return M.tocsr()


def to_liouville(X: np.ndarray) -> np.ndarray:
    """(N, d, d) row-major blocks -> concatenated column-stacked vec(rho_n)."""
    return np.ascontiguousarray(np.swapaxes(X, -1, -2)).reshape(-1)


def from_liouville(v: np.ndarray, d: int) -> np.ndarray:
    return np.ascontiguousarray(np.swapaxes(v.reshape(-1, d, d), -1, -2))
