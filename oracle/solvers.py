"""Solvers driven by M (oracle, FP64): dynamics, stationary state, spectra, current.

Paper passages followed:
* Package architecture: dynamics by an ODE solver or by the propagator exp(M t);
  stationary states by a linear solve.
* Methods, "Numerical computation of the spectrum": the bosonic power spectrum
  pi S(w) = -Re Tr[a^dag x] with (M - i w) x = a rho (even parity), and the density of
  states pi A(w) = -Re{Tr[d x_+] + Tr[d^dag x_-]} with (M + i w) x_+ = d^dag rho and
  (M - i w) x_- = d rho, M acting on odd-parity ADOs; only the tier-0 block enters the trace.
* Methods, "Electronic current" (Eq. last): <I_alpha> = i e sum_{nu,h,sigma}
  (-1)^{delta_{nu,-}} Tr[d_sigma^{nubar} rho^{(0,1,+)}_{alpha,nu,h,sigma}].

Readings (the paper does not fix them):
* Dynamics: classical fixed-step RK4 (the paper's adaptive ODE solvers are not specified).
  A time-dependent H_s(t) (Eq. H_total) is written H + sum_k f_k(t) H_k with scalar f_k
  sampled on the half-step grid, which is where classical RK4 evaluates the right-hand side.
* Stationary state: the equation of the (0,0) element of the tier-0 ADO is replaced by the
  normalisation Tr rho_sys = 1 (that equation is redundant because M preserves the trace).
* b = O rho_n for every ADO n (left multiplication, no extra sign) in the spectra.
* Residuals: r_ss = ||M x|| / ||x|| with Tr rho_sys = 1; linear solves ||b - A x|| / ||b||.
* Large hierarchies (a fermionic tier 4: 12,951 ADOs) defeat the sparse LU (fill-in); the same
  systems are then solved by restarted GMRES (a library routine) with a diagonal
  preconditioner, pinned against the LU results on smaller hierarchies.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .liouvillian import from_liouville, to_liouville


def rk4(apply, x0: np.ndarray, dt: float, n_steps: int, save_every: int = 1,
        observe=None):
    """Classical RK4: x <- x + dt/6 (k1 + 2 k2 + 2 k3 + k4). Returns (x_end, snapshots)."""
    observe = observe or (lambda v: v.copy())
    x = x0.copy()
    snaps = [observe(x)]
    for s in range(n_steps):
        k1 = apply(x)
        k2 = apply(x + 0.5 * dt * k1)
        k3 = apply(x + 0.5 * dt * k2)
        k4 = apply(x + dt * k3)
        x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if (s + 1) % save_every == 0:
            snaps.append(observe(x))
    return x, snaps


def drive_superoperators(n_ado: int, ops):
    """-i [H_k, .] on every ADO for each drive operator H_k: a time-dependent system
    Hamiltonian H_s(t) = H + sum_k f_k(t) H_k enters Eq. HEOM only through the commutator
    L_s(t) = [H_s(t), .], which acts on every ADO alike. Column stacking, block diagonal."""
    from .liouvillian import spost, spre

    out = []
    for Hk in ops:
        Hk = np.asarray(Hk, np.complex128)
        blk = -1j * (spre(Hk) - spost(Hk))
        out.append(sp.kron(sp.identity(n_ado, format="csr"), blk, format="csr"))
    return out


def rk4_td(M0, Ls, f, x0: np.ndarray, dt: float, n_steps: int, save_every: int = 1,
           observe=lambda x: x.copy()):
    """Classical RK4 for dx/dt = (M0 + sum_k f_k(t) L_k) x. f[k][j] = f_k(t0 + j dt / 2): the
    four stages of step n evaluate the right-hand side at t_n (sample 2n), t_n + dt/2 (sample
    2n + 1, twice) and t_n + dt (sample 2n + 2)."""
    f = np.asarray(f, np.float64).reshape(len(Ls), 2 * n_steps + 1)

    def rhs(j, v):
        y = M0 @ v
        for k, L in enumerate(Ls):
            y = y + f[k, j] * (L @ v)
        return y

    x = x0.copy()
    snaps = [observe(x)]
    for n in range(n_steps):
        j = 2 * n
        k1 = rhs(j, x)
        k2 = rhs(j + 1, x + 0.5 * dt * k1)
        k3 = rhs(j + 1, x + 0.5 * dt * k2)
        k4 = rhs(j + 2, x + dt * k3)
        x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if (n + 1) % save_every == 0:
            snaps.append(observe(x))
    return x, snaps


def propagate_expm(M, v0: np.ndarray, t: float) -> np.ndarray:
    """exp(M t) v0 with a dense matrix exponential (tiny hierarchies only)."""
    Md = M.toarray() if sp.issparse(M) else np.asarray(M)
    return sla.expm(Md * t) @ v0


def initial_vector(n_ado: int, rho0: np.ndarray) -> np.ndarray:
    """All ADOs zero except the tier-0 one, which is rho0 (row-major blocks)."""
    X = np.zeros((n_ado,) + rho0.shape, dtype=np.complex128)
    X[0] = rho0
    return X


def steady_state(M, d: int) -> np.ndarray:
    """Solve M x = 0 with Tr rho_sys = 1 by sparse LU; returns (N, d, d) blocks."""
    A = sp.lil_matrix(M, dtype=np.complex128)
    trace_row = np.zeros(M.shape[1], dtype=np.complex128)
    trace_row[[i * d + i for i in range(d)]] = 1.0  # column stacking: (i,i) -> i*d + i
    A[0, :] = trace_row
    rhs = np.zeros(M.shape[0], dtype=np.complex128)
    rhs[0] = 1.0
    lu = spla.splu(sp.csc_matrix(A))
    return from_liouville(lu.solve(rhs), d)


def _stationary_system(M, d: int):
    """The stationary-state system of steady_state: M with the row of the (0,0) element of the
    tier-0 ADO replaced by the trace row (column stacking: (i, i) -> i d + i), rhs e_0."""
    A = sp.lil_matrix(M, dtype=np.complex128)
    trace_row = np.zeros(M.shape[1], dtype=np.complex128)
    trace_row[[i * d + i for i in range(d)]] = 1.0
    A[0, :] = trace_row
    rhs = np.zeros(M.shape[0], dtype=np.complex128)
    rhs[0] = 1.0
    return sp.csr_matrix(A), rhs


def _gmres(A, b, tol: float, restart: int = 300, maxiter: int = 40):
    """x with ||b - A x|| <= tol ||b|| by restarted GMRES (scipy), right-preconditioned by the
    inverse diagonal of A (1 where the diagonal is zero). For hierarchies whose sparse LU is
    out of reach (fill-in); pinned against the LU solvers on smaller hierarchies."""
    dg = A.diagonal()
    dg = np.where(np.abs(dg) > 0, dg, 1.0)
    P = spla.LinearOperator(A.shape, matvec=lambda v: v / dg, dtype=np.complex128)
    x, info = spla.gmres(A, b, rtol=tol, atol=0.0, restart=restart, maxiter=maxiter, M=P)
    res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    if not res <= 10 * tol:
        raise RuntimeError(f"oracle GMRES did not converge: info {info}, residual {res:.2e}")
    return x


def steady_state_iterative(M, d: int, tol: float = 1e-12) -> np.ndarray:
    """steady_state's system solved by GMRES instead of sparse LU; returns (N, d, d) blocks."""
    A, rhs = _stationary_system(M, d)
    return from_liouville(_gmres(A, rhs, tol), d)


def dos_iterative(M_odd, X_ss: np.ndarray, dop: np.ndarray, omegas, tol: float = 1e-12):
    """dos with every shifted system solved by GMRES instead of sparse LU."""
    d = dop.shape[0]
    bp = to_liouville(left_multiply(dop.conj().T, X_ss))
    bm = to_liouville(left_multiply(dop, X_ss))
    I = sp.identity(M_odd.shape[0], dtype=np.complex128, format="csr")
    Mc = sp.csr_matrix(M_odd)
    out = np.empty(len(omegas))
    for k, w in enumerate(omegas):
        xp = _gmres(Mc + 1j * w * I, bp, tol)
        xm = _gmres(Mc - 1j * w * I, bm, tol)
        xp0 = from_liouville(xp[: d * d], d)[0]
        xm0 = from_liouville(xm[: d * d], d)[0]
        out[k] = -np.real(np.trace(dop @ xp0) + np.trace(dop.conj().T @ xm0)) / np.pi
    return out


def steady_residual(M, X: np.ndarray) -> float:
    """r_ss = ||M x|| / ||x|| after normalising Tr rho_sys = 1."""
    X = X / np.trace(X[0])
    v = to_liouville(X)
    return float(np.linalg.norm(M @ v) / np.linalg.norm(v))


def left_multiply(op: np.ndarray, X: np.ndarray) -> np.ndarray:
    """b_n = op rho_n for every ADO n."""
    return np.einsum("ij,njk->nik", op, X)


def dos(M_odd, X_ss: np.ndarray, dop: np.ndarray, omegas, return_solutions=False):
    """Density of states A(w) of the mode dop (Methods, spectrum; fermionic case)."""
    d = dop.shape[0]
    bp = to_liouville(left_multiply(dop.conj().T, X_ss))
    bm = to_liouville(left_multiply(dop, X_ss))
    I = sp.identity(M_odd.shape[0], dtype=np.complex128, format="csc")
    Mc = sp.csc_matrix(M_odd)
    out = np.empty(len(omegas))
    sols = []
    for k, w in enumerate(omegas):
        xp = spla.splu(Mc + 1j * w * I).solve(bp)
        xm = spla.splu(Mc - 1j * w * I).solve(bm)
        xp0 = from_liouville(xp[: d * d], d)[0]
        xm0 = from_liouville(xm[: d * d], d)[0]
        out[k] = -np.real(np.trace(dop @ xp0) + np.trace(dop.conj().T @ xm0)) / np.pi
        if return_solutions:
            sols.append((xp, xm))
    return (out, sols) if return_solutions else out


def psd(M_even, X_ss: np.ndarray, aop: np.ndarray, omegas):
    """Power spectral density S(w) of the mode aop (Methods, spectrum; bosonic case)."""
    d = aop.shape[0]
    b = to_liouville(left_multiply(aop, X_ss))
    I = sp.identity(M_even.shape[0], dtype=np.complex128, format="csc")
    Mc = sp.csc_matrix(M_even)
    out = np.empty(len(omegas))
    for k, w in enumerate(omegas):
        x = spla.splu(Mc - 1j * w * I).solve(b)
        x0 = from_liouville(x[: d * d], d)[0]
        out[k] = -np.real(np.trace(aop.conj().T @ x0)) / np.pi
    return out


def current(problem: dict, hier, X_ss: np.ndarray, baths_of_lead) -> float:
    """<I_alpha> (e = 1) from the tier-1 fermionic ADOs of the baths that form lead alpha."""
    from .hierarchy import flatten_exponents
    from .liouvillian import op_power

    _, fer = flatten_exponents(problem)
    m0 = hier.bos[0]
    total = 0j
    for q, e in enumerate(fer):
        if e.bath not in baths_of_lead:
            continue
        rho_q = X_ss[hier.index[(m0, (q,))]]
        sign = 1 if e.nu == 1 else -1
        total += sign * np.trace(op_power(e.op, -e.nu) @ rho_q)
    return float(np.real(1j * total))


def solve_residual(A, x: np.ndarray, b: np.ndarray) -> float:
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
