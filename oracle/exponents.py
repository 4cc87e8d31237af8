"""Bath correlation functions as sums of exponentials (oracle, FP64).

Paper passages followed:
* Eq. C_f / Eq. C_b: the fermionic and bosonic two-time correlation functions.
* Eq. C_f_exp / Eq. C_b_exp: their exponential expansions.
* Methods, "Fermion correlation function with Lorentzian spectral density": J_alpha (Eq.
  Lorentz), the Pade form of the Fermi function and the exponents eta, gamma.
* Methods, "Boson correlation function with Drude-Lorentz spectral density": J_beta
  (Eq. Drude-Lorentz), the Pade form of the Bose function and the exponents xi, chi.

The Pade constants kappa, zeta are not printed in the paper (it cites Hu, Xu and Yan for
them). The reading used here is the [N-1/N] Pade spectrum decomposition: the poles come
from the eigenvalues of a symmetric tridiagonal matrix; the residues from a product formula.
The result is pinned by the test that the rational approximant reproduces 1/(e^x +- 1).

Matsubara: kappa = 1, zeta_j = (2j-1)pi (Fermi) or 2 pi j (Bose), j = 1..n_poles.

The printed fermionic exponent list repeats the symbol eta for the last line; that line is
the rate gamma_h = zeta_h kT - nu i mu (it follows from the residue at the Pade pole).
"""
from __future__ import annotations

import numpy as np


def _tridiag_positive_eigs(offdiag: np.ndarray) -> np.ndarray:
    """Positive eigenvalues (descending) of the zero-diagonal symmetric tridiagonal matrix."""
    n = len(offdiag) + 1
    T = np.zeros((n, n))
    for m, b in enumerate(offdiag):
        T[m, m + 1] = T[m + 1, m] = b
    lam = np.linalg.eigvalsh(T)
    return np.sort(lam[lam > 1e-12])[::-1]


def pade_constants(n_poles: int, statistics: str):
    """[N-1/N] Pade decomposition constants (kappa_j, zeta_j), j = 1..n_poles.

    Fermi: 1/(e^x+1) ~ 1/2 - sum_j 2 kappa_j x / (x^2 + zeta_j^2)
    Bose:  1/(e^x-1) ~ 1/x - 1/2 + sum_j 2 kappa_j x / (x^2 + zeta_j^2)
    (the two Pade forms printed in Methods). With b_m = 2m-1 (Fermi) or 2m+1 (Bose):
    zeta_j = 2/lambda_j for the positive eigenvalues lambda of the 2N x 2N zero-diagonal
    tridiagonal matrix with off-diagonals 1/sqrt(b_m b_{m+1}); the auxiliary roots
    zt_i = 2/lambda~_i come from the (2N-1) x (2N-1) matrix built from b_{m+1};
    kappa_j = (N b_{N+1} / 2) prod_i (zt_i^2 - zeta_j^2) / prod_{k != j} (zeta_k^2 - zeta_j^2).
    """
    if n_poles == 0:
        return np.zeros(0), np.zeros(0)
    if statistics == "fermi":
        b = lambda m: 2.0 * m - 1.0  # noqa: E731
    elif statistics == "bose":
        b = lambda m: 2.0 * m + 1.0  # noqa: E731
    else:
        raise ValueError(statistics)
    N = n_poles
    off = np.array([1.0 / np.sqrt(b(m) * b(m + 1)) for m in range(1, 2 * N)])
    zeta = 2.0 / _tridiag_positive_eigs(off)
    off_t = np.array([1.0 / np.sqrt(b(m + 1) * b(m + 2)) for m in range(1, 2 * N - 1)])
    zt = 2.0 / _tridiag_positive_eigs(off_t) if N > 1 else np.zeros(0)
    kappa = np.empty(N)
    for j in range(N):
        num = np.prod(zt ** 2 - zeta[j] ** 2)
        den = np.prod([zeta[k] ** 2 - zeta[j] ** 2 for k in range(N) if k != j])
        kappa[j] = 0.5 * N * b(N + 1) * num / den
    return kappa, zeta


def matsubara_constants(n_poles: int, statistics: str):
    """Matsubara poles: kappa_j = 1, zeta_j = (2j-1) pi (Fermi) or 2 pi j (Bose)."""
    j = np.arange(1, n_poles + 1, dtype=np.float64)
    zeta = (2 * j - 1) * np.pi if statistics == "fermi" else 2 * np.pi * j
    return np.ones(n_poles), zeta


def decomposition(n_poles: int, statistics: str, method: str):
    if method == "pade":
        return pade_constants(n_poles, statistics)
    if method == "matsubara":
        return matsubara_constants(n_poles, statistics)
    raise ValueError(method)


def fermi_approx(x, kappa, zeta):
    """n^Pade(x) = 1/2 - sum_h 2 kappa_h x / (x^2 + zeta_h^2) (Methods, fermion case)."""
    x = np.asarray(x, dtype=np.complex128)
    out = 0.5 + 0.0 * x
    for k, z in zip(kappa, zeta):
        out = out - 2.0 * k * x / (x * x + z * z)
    return out


def bose_approx(x, kappa, zeta):
    """n^Pade(x) = 1/x - 1/2 + sum_l 2 kappa_l x / (x^2 + zeta_l^2) (Methods, boson case)."""
    x = np.asarray(x, dtype=np.complex128)
    out = 1.0 / x - 0.5
    for k, z in zip(kappa, zeta):
        out = out + 2.0 * k * x / (x * x + z * z)
    return out


def lorentz_fermion_exponents(Gamma, W, mu, kT, n_poles, method, nu):
    """Exponents (eta_h, gamma_h), h = 1..n_poles+1, of C^nu_alpha (Eq. C_f_exp).

    eta_1 = (Gamma W / 2) n^Pade(i W / kT),      gamma_1 = W - nu i mu
    eta_h = -i kappa_h kT Gamma W^2 / (W^2 - (zeta_h kT)^2),   gamma_h = zeta_h kT - nu i mu
    (Methods, Lorentzian fermion exponents; with method="matsubara" kappa=1 and zeta the
    Matsubara poles, n^Pade then being the Matsubara-truncated Fermi function).
    """
    kappa, zeta = decomposition(n_poles, "fermi", method)
    eta = np.empty(n_poles + 1, dtype=np.complex128)
    gam = np.empty(n_poles + 1, dtype=np.complex128)
    eta[0] = 0.5 * Gamma * W * fermi_approx(1j * W / kT, kappa, zeta)
    gam[0] = W - nu * 1j * mu
    for h in range(n_poles):
        eta[h + 1] = -1j * kappa[h] * kT * Gamma * W ** 2 / (W ** 2 - (zeta[h] * kT) ** 2)
        gam[h + 1] = zeta[h] * kT - nu * 1j * mu
    return eta, gam


def drude_lorentz_exponents(lam, W, kT, n_poles, method):
    """Exponents (xi_l, chi_l), l = 1..n_poles+1, of C_beta (Eq. C_b_exp).

    xi_1 = lam W [cot(W / 2kT) - i],  chi_1 = W
    xi_l = -2 kappa_l kT * 2 lam W zeta_l kT / (W^2 - (zeta_l kT)^2),  chi_l = zeta_l kT
    (Methods, Drude-Lorentz exponents; lam is the coupling the paper calls Delta_beta).
    All chi are real, so the real and imaginary parts of C_beta share exponents and one
    combined ("RI") exponent per l is used (Eq. C_beta_RI with chi = chi^*).
    """
    kappa, zeta = decomposition(n_poles, "bose", method)
    xi = np.empty(n_poles + 1, dtype=np.complex128)
    chi = np.empty(n_poles + 1, dtype=np.complex128)
    xi[0] = lam * W * (1.0 / np.tan(W / (2.0 * kT)) - 1j)
    chi[0] = W
    for l in range(n_poles):
        zk = zeta[l] * kT
        xi[l + 1] = -2.0 * kappa[l] * kT * 2.0 * lam * W * zk / (W ** 2 - zk ** 2)
        chi[l + 1] = zk
    return xi, chi


def correlation_from_exponents(coef, rate, tau):
    """C(tau) = sum_k coef_k exp(-rate_k tau) (Eqs. C_f_exp, C_b_exp)."""
    tau = np.asarray(tau, dtype=np.float64)
    return sum(c * np.exp(-r * tau) for c, r in zip(coef, rate))
