"""Pins of oracle/exponents.py against the Fermi/Bose functions and quadrature of Eqs. C_f, C_b."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import exponents as ex


@pytest.mark.parametrize("N,tol", [(2, 0.13), (6, 1e-6), (10, 1e-13)])
def test_pade_fermi_reproduces_fermi_function(N, tol):
    kappa, zeta = ex.pade_constants(N, "fermi")
    x = np.linspace(-20, 20, 4001)
    approx = ex.fermi_approx(x, kappa, zeta).real
    assert np.abs(approx - 1.0 / (np.exp(x) + 1.0)).max() < tol


@pytest.mark.parametrize("N,tol", [(2, 0.06), (6, 1e-7), (10, 1e-13)])
def test_pade_bose_reproduces_bose_function(N, tol):
    kappa, zeta = ex.pade_constants(N, "bose")
    x = np.linspace(-20, 20, 4000)  # even count: x = 0 is not on the grid
    approx = ex.bose_approx(x, kappa, zeta).real
    assert np.abs(approx - 1.0 / np.expm1(x)).max() < tol


def test_pade_poles_tend_to_matsubara_poles():
    _, zf = ex.pade_constants(20, "fermi")
    _, zb = ex.pade_constants(20, "bose")
    assert np.allclose(zf[:3], [np.pi, 3 * np.pi, 5 * np.pi], rtol=1e-12)
    assert np.allclose(zb[:3], [2 * np.pi, 4 * np.pi, 6 * np.pi], rtol=1e-12)
    kf, _ = ex.pade_constants(20, "fermi")
    assert np.allclose(kf[:3], 1.0, atol=1e-12)


def test_matsubara_truncation_is_the_series():
    # 1/(e^x+1) = 1/2 - sum_j 2x/(x^2+((2j-1)pi)^2): converges like 1/n at fixed x
    k, z = ex.matsubara_constants(20000, "fermi")
    x = np.array([-3.0, 0.5, 2.0])
    assert np.abs(ex.fermi_approx(x, k, z).real - 1 / (np.exp(x) + 1)).max() < 2e-4


def _fourier(g, tau, nu):
    """(1/2pi) int_R g(w) e^{nu i w tau} dw for a real, integrable g (QAWF on [0, inf))."""
    c = quad(lambda w: g(w) + g(-w), 0, np.inf, weight="cos", wvar=tau, limlst=200)[0]
    s = quad(lambda w: g(w) - g(-w), 0, np.inf, weight="sin", wvar=tau, limlst=200)[0]
    return (c + 1j * nu * s) / (2 * np.pi)


@pytest.mark.parametrize("nu", [1, -1])
@pytest.mark.parametrize("method,N", [("pade", 2), ("pade", 5), ("matsubara", 3)])
def test_fermion_exponents_reproduce_eq_C_f(nu, method, N):
    """Sum of exponents == quadrature of Eq. C_f with the same (truncated) Fermi function."""
    Gamma, W, mu, kT = 2.0, 10.0, 1.0, 0.5
    kappa, zeta = ex.decomposition(N, "fermi", method)
    eta, gam = ex.lorentz_fermion_exponents(Gamma, W, mu, kT, N, method, nu)

    def g(w):
        J = Gamma * W ** 2 / ((w - mu) ** 2 + W ** 2)
        n = ex.fermi_approx((w - mu) / kT, kappa, zeta).real
        return J * ((1 - nu) / 2 + nu * n)

    for tau in (0.3, 1.0, 3.0):
        ref = _fourier(g, tau, nu)
        val = ex.correlation_from_exponents(eta, gam, tau)
        assert abs(val - ref) < 1e-7 * max(1.0, abs(ref)), (tau, val, ref)


@pytest.mark.parametrize("method,N,tol", [("pade", 10, 1e-8), ("matsubara", 60, 1e-8)])
def test_boson_exponents_reproduce_eq_C_b(method, N, tol):
    """Sum of exponents == quadrature of Eq. C_b with the exact Bose function."""
    lam, W, kT = 0.1, 0.5, 0.5
    xi, chi = ex.drude_lorentz_exponents(lam, W, kT, N, method)

    def J(w):
        return 4 * lam * W * w / (w * w + W * W)

    for tau in (0.3, 1.0, 3.0):
        # (1/2pi) int_0^inf J [ coth(w/2kT) cos(w tau) - i sin(w tau) ]
        re = quad(lambda w: J(w) / np.tanh(w / (2 * kT)) if w > 0 else 4 * lam * 2 * kT / W,
                  0, np.inf, weight="cos", wvar=tau, limlst=200)[0]
        im = quad(J, 0, np.inf, weight="sin", wvar=tau, limlst=200)[0]
        ref = (re - 1j * im) / (2 * np.pi)
        val = ex.correlation_from_exponents(xi, chi, tau)
        assert abs(val - ref) < tol, (tau, val, ref)


def test_fermion_eta_does_not_depend_on_nu_for_lorentzian():
    ep, gp = ex.lorentz_fermion_exponents(2.0, 10.0, 1.0, 0.5, 3, "pade", 1)
    em, gm = ex.lorentz_fermion_exponents(2.0, 10.0, 1.0, 0.5, 3, "pade", -1)
    assert np.allclose(ep, em)
    assert np.allclose(gp, np.conj(gm))
