"""Pins of oracle/liouvillian.py and oracle/solvers.py against closed forms and invariants.

What each test would catch:
* two paths        a transposed operand or a wrong block position in either assembly;
* tier-0 trace     a wrong P_s sign at tier 0 (the raising terms must be commutators);
* zero coupling    a wrong system commutator sign or H transposed;
* pure dephasing   a wrong D term (both its commutator and anticommutator parts) or damping;
* noninteracting   a wrong fermionic sign, nu / partner mix-up, or eta conjugation
  (occupation against the Keldysh integral, current against Landauer, DOS against -Im G/pi);
* relabelling      an ordering sign eps(q, S) that is not antisymmetric.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.integrate import quad

import workloads as W
from oracle import exponents as ex
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so


def _matrix_apply(prob, h, X):
    M = lv.build_matrix(prob, h)
    return lv.from_liouville(M @ lv.to_liouville(X), prob["d"])


@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("bos,fer,tb,tf", [
    ([("RI", 2), ("R", 1), ("I", 1)], [], 3, 0),
    ([], [4, 2], 0, 3),
    ([("RI", 2), ("I", 1)], [4, 2], 2, 2),
])
def test_two_paths_agree(parity, bos, fer, tb, tf):
    prob = W.random_raw_problem(3, bos, fer, tb, tf, parity=parity, seed=11)
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, seed=12)
    Y1 = lv.apply_loop(prob, X, h)
    Y2 = _matrix_apply(prob, h, X)
    assert np.abs(Y1 - Y2).max() <= 1e-13 * np.abs(Y1).max()


def test_tier0_trace_is_preserved_even_sector():
    prob = W.random_raw_problem(3, [("RI", 2)], [4], 2, 2, parity=1, seed=3)
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, seed=4)
    Y = lv.apply_loop(prob, X, h)
    assert abs(np.trace(Y[0])) < 1e-12 * np.abs(Y).max()


def test_zero_coupling_is_unitary_evolution():
    H, V, rho0 = W.spin_boson_ops(1.0)
    prob = dict(d=2, H=H, baths=[dict(kind="RI", op=V, coef=np.zeros(3, complex),
                                      rate=np.array([0.5, np.pi, 2 * np.pi]))],
                tier_b=3, tier_f=0, parity=1)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    x0 = lv.to_liouville(so.initial_vector(h.n_ado, rho0))
    t = 2.5
    U = sla.expm(-1j * H * t)
    exact = U @ rho0 @ U.conj().T
    r_expm = lv.from_liouville(so.propagate_expm(M, x0, t), 2)[0]
    _, snaps = so.rk4(lambda v: M @ v, x0, 0.01, 250, save_every=250,
                      observe=lambda v: lv.from_liouville(v, 2)[0])
    assert np.abs(r_expm - exact).max() < 1e-12
    assert np.abs(snaps[-1] - exact).max() < 1e-9


@pytest.mark.parametrize("tier,tol", [(4, 5e-5), (8, 1e-10)])
def test_pure_dephasing_closed_form(tier, tol):
    """[H, V] = 0: rho_01(t) = rho_01(0) e^{-i(E0-E1)t} exp(-(s0-s1)^2 Phi - i(s0^2-s1^2) Psi),
    Phi + i Psi = sum_k xi_k [t/chi_k - (1 - e^{-chi_k t})/chi_k^2] (second-order cumulant,
    exact for a Gaussian bath). V = diag(0, 1) so that Psi (the {V, .} part of D) enters."""
    eps, lam, Wc, kT, t = 0.7, 0.2, 1.0, 1.0, 3.0
    H = np.diag([eps / 2, -eps / 2]).astype(complex)
    V = np.diag([0.0, 1.0]).astype(complex)
    xi, chi = ex.drude_lorentz_exponents(lam, Wc, kT, 3, "pade")
    rho0 = 0.5 * np.ones((2, 2), complex)
    s, E = np.diag(V).real, np.diag(H).real
    G = [t / c - (1 - np.exp(-c * t)) / c ** 2 for c in chi.real]
    phi = sum(x.real * g for x, g in zip(xi, G))
    psi = sum(x.imag * g for x, g in zip(xi, G))
    exact = rho0[0, 1] * np.exp(-1j * (E[0] - E[1]) * t
                                - (s[0] - s[1]) ** 2 * phi - 1j * (s[0] ** 2 - s[1] ** 2) * psi)
    prob = dict(d=2, H=H, baths=[dict(kind="RI", op=V, coef=xi, rate=chi)],
                tier_b=tier, tier_f=0, parity=1)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    x0 = lv.to_liouville(so.initial_vector(h.n_ado, rho0))
    r = lv.from_liouville(so.propagate_expm(M, x0, t), 2)[0]
    assert abs(r[0, 1] - exact) < tol
    assert abs(r[0, 0] - 0.5) < 1e-12


# ---------------------------------------------------------------- noninteracting level
EPS, GAM, WB, KT, MUS, NP = 0.3, 1.0, 4.0, 0.5, (1.0, -0.5), 4


def _level(tier, parity=1):
    m = W.single_level_model(EPS, GAM, WB, KT, MUS[0], MUS[1], NP, tier)
    prob = hy.model_to_problem(m, parity)
    h = hy.problem_hierarchy(prob)
    return m, prob, h, lv.build_matrix(prob, h)


def _GR(w):
    return 1.0 / (w - EPS - sum(0.5 * GAM * WB / (w - mu + 1j * WB) for mu in MUS))


def _J(w, mu):
    return GAM * WB ** 2 / ((w - mu) ** 2 + WB ** 2)


def _f(w, mu):
    k, z = ex.pade_constants(NP, "fermi")
    return ex.fermi_approx((w - mu) / KT, k, z).real


def test_noninteracting_occupation_matches_keldysh_integral():
    """<n> = int dw/2pi |G^R|^2 sum_a J_a f_a with the Pade f (exact for these exponents)."""
    _, prob, h, M = _level(2)
    X = so.steady_state(M, 2)
    ref = quad(lambda w: abs(_GR(w)) ** 2 * sum(_J(w, mu) * _f(w, mu) for mu in MUS)
               / (2 * np.pi), -np.inf, np.inf, limit=500, epsabs=1e-14)[0]
    assert abs(X[0][1, 1].real - ref) < 1e-10
    assert so.steady_residual(M, X) < 1e-12
    # the hierarchy closes at tier 2 for a noninteracting level
    _, _, _, M3 = _level(3)
    X3 = so.steady_state(M3, 2)
    assert np.abs(X3[0] - X[0]).max() < 1e-11


def test_noninteracting_current_matches_landauer():
    _, prob, h, M = _level(2)
    X = so.steady_state(M, 2)
    IL = so.current(prob, h, X, [0])
    IR = so.current(prob, h, X, [1])
    ref = quad(lambda w: abs(_GR(w)) ** 2 * _J(w, MUS[0]) * _J(w, MUS[1])
               * (_f(w, MUS[0]) - _f(w, MUS[1])) / (2 * np.pi),
               -np.inf, np.inf, limit=500, epsabs=1e-14)[0]
    assert abs(IL - ref) < 1e-9
    assert abs(IL + IR) < 1e-12


def test_noninteracting_dos_matches_green_function():
    m, prob, h, M = _level(2)
    X = so.steady_state(M, 2)
    _, probo, ho, Mo = _level(2, parity=-1)
    om = np.array([-6.0, -1.0, 0.0, 0.3, 1.7, 5.0])
    A = so.dos(Mo, X, m.fermion_baths[0][0], om)
    ref = np.array([-_GR(w).imag / np.pi for w in om])
    assert np.abs(A - ref).max() < 1e-11


def test_fermionic_relabelling_leaves_physics_unchanged():
    """Reversing the bath order and the exponent order inside each bath permutes the ADOs
    with ordering signs; the reduced state and the current must not change (SIAM, tier 2)."""
    model = W.siam_model(tier=2, U=4.0, Gamma=1.0, kT=1.0)
    prob = hy.model_to_problem(model)
    rev = dict(prob)
    baths = []
    for b in reversed(prob["baths"]):
        k = len(b["coef"])
        perm = np.arange(k)[::-1]
        inv = np.empty(k, int)
        inv[perm] = np.arange(k)
        baths.append(dict(kind="F", op=b["op"], coef=b["coef"][perm], rate=b["rate"][perm],
                          nu=b["nu"][perm], partner=inv[b["partner"][perm]].astype(np.int32)))
    rev["baths"] = baths
    res = []
    for p, leads in ((prob, ([0, 1], [2, 3])), (rev, ([2, 3], [0, 1]))):
        h = hy.problem_hierarchy(p)
        M = lv.build_matrix(p, h)
        X = so.steady_state(M, 4)
        res.append((X[0], so.current(p, h, X, leads[0]), so.current(p, h, X, leads[1])))
    assert np.abs(res[0][0] - res[1][0]).max() < 1e-11
    assert abs(res[0][1] - res[1][1]) < 1e-11
    assert abs(res[0][1] + res[0][2]) < 1e-10


# ---------------------------------------------------------------- dynamics and spectra
def test_rk4_matches_propagator_and_preserves_trace():
    """RK4 conserves the (linear) trace exactly, keeps rho Hermitian, and converges to
    exp(Mt) x0 at fourth order: halving dt divides the error by ~16."""
    model = W.spin_boson_model(tier=2)
    prob = hy.model_to_problem(model)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    x0 = lv.to_liouville(so.initial_vector(h.n_ado, model.rho0))
    obs = lambda v: lv.from_liouville(v, 2)[0]  # noqa: E731
    errs = []
    for dt in (0.02, 0.01):
        n = int(round(2.0 / dt))
        _, snaps = so.rk4(lambda v: M @ v, x0, dt, n, save_every=n // 4, observe=obs)
        err = 0.0
        for k, r in enumerate(snaps):
            assert abs(np.trace(r) - 1) < 1e-13
            assert np.abs(r - r.conj().T).max() < 1e-13
            err = max(err, np.abs(r - obs(so.propagate_expm(M, x0, 0.5 * k))).max())
        errs.append(err)
    assert errs[1] < 1e-9
    assert 12.0 < errs[0] / errs[1] < 20.0


def test_even_sector_has_one_stationary_mode():
    model = W.spin_boson_model(tier=2)
    prob = hy.model_to_problem(model)
    h = hy.problem_hierarchy(prob)
    lam = np.linalg.eigvals(lv.build_matrix(prob, h).toarray())
    small = np.abs(lam) < 1e-9
    assert small.sum() == 1
    assert lam[~small].real.max() < 0


def test_tier_convergence_spin_boson():
    model = W.spin_boson_model(tier=7)
    errs = []
    ref = None
    for tier in (7, 1, 2, 3, 4):
        model.tier_b = tier
        prob = hy.model_to_problem(model)
        h = hy.problem_hierarchy(prob)
        M = lv.build_matrix(prob, h)
        x0 = lv.to_liouville(so.initial_vector(h.n_ado, model.rho0))
        r = lv.from_liouville(so.propagate_expm(M, x0, 5.0), 2)[0]
        if ref is None:
            ref = r
        else:
            errs.append(np.abs(r - ref).max())
    assert all(errs[i + 1] <= errs[i] for i in range(len(errs) - 1))


def test_siam_stationary_state_is_a_density_matrix():
    model = W.siam_model(tier=2)
    prob = hy.model_to_problem(model)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    X = so.steady_state(M, 4)
    r = X[0]
    assert abs(np.trace(r) - 1) < 1e-13
    assert np.abs(r - r.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh(0.5 * (r + r.conj().T)).min() > -1e-10
    assert so.steady_residual(M, X) < 1e-12
    IL = so.current(prob, h, X, [0, 1])
    IR = so.current(prob, h, X, [2, 3])
    assert abs(IL + IR) < 1e-10 and IL > 0  # mu_L > mu_R: electrons flow L -> R


def test_siam_dos_symmetry_and_hubbard_peaks():
    """eps = -U/2 makes the model particle-hole symmetric, so A(w) = A(-w) exactly; the
    Hubbard peaks sit near eps and eps + U (Example 1, qualitative; Gamma = 1 as in Table 1)."""
    model = W.siam_model(tier=2, Gamma=1.0)
    prob = hy.model_to_problem(model)
    h = hy.problem_hierarchy(prob)
    X = so.steady_state(lv.build_matrix(prob, h), 4)
    Mo = lv.build_matrix(hy.model_to_problem(model, -1), h)
    om = np.linspace(-10, 10, 41)
    A = so.dos(Mo, X, model.fermion_baths[0][0], om)
    assert A.min() > 0
    assert np.abs(A - A[::-1]).max() < 1e-10
    left = om[np.argmax(np.where(om < -2, A, 0))]
    assert -7.5 <= left <= -4.0


@pytest.mark.parametrize("parity", [1, -1])
def test_integer_tables_reproduce_the_apply(parity):
    """oracle/tables.py (the integer tables the GPU must match) against the loop path."""
    from oracle import tables as tb
    prob = W.random_raw_problem(3, [("RI", 2), ("I", 1)], [4, 2], 2, 2, parity=parity, seed=21)
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, seed=22)
    Y1 = lv.apply_loop(prob, X, h)
    Y3 = tb.apply_from_tables(prob, X, h)
    assert np.abs(Y1 - Y3).max() <= 1e-13 * np.abs(Y1).max()


def test_psd_sum_rule_spin_boson():
    """The PSD is the real part of the Laplace transform of the correlation function
    C(t) = Tr[a^dag e^{Mt}(a rho_ss)], so its integral over all frequencies is Re C(0) =
    <a^dag a> when the stationary <a> vanishes. Spin-boson with H = (Delta/2) sigma_x: the
    stationary <sigma_z> is 0 by symmetry and <sigma_z sigma_z> = 1."""
    m = W.spin_boson_model(tier=4)
    prob = hy.model_to_problem(m, 1)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    X = so.steady_state(M, m.d)
    sz = np.diag([1.0, -1.0]).astype(complex)
    assert abs(np.trace(sz @ X[0])) < 1e-12
    om = np.linspace(-50, 50, 4000)  # an even count: omega = 0 (the zero mode) is not sampled
    S = so.psd(M, X, sz, om)
    assert abs(np.trapezoid(S, om) - 1.0) < 1e-6


def test_iterative_solvers_match_sparse_lu():
    """The GMRES path of the oracle (for hierarchies whose sparse LU fills in beyond reach)
    solves the same systems as the LU path: on SIAM tier 2 (301 ADOs) the stationary state and
    the DOS agree with the LU results to 1e-11, and on the noninteracting level the GMRES DOS
    equals -Im G^R(w) / pi."""
    m = W.siam_model(tier=2, U=5.0, mu=1.5, kT=0.5)
    pe = hy.model_to_problem(m, 1)
    h = hy.problem_hierarchy(pe)
    Me = lv.build_matrix(pe, h)
    Mo = lv.build_matrix(hy.model_to_problem(m, -1), h)
    X = so.steady_state(Me, 4)
    Xi = so.steady_state_iterative(Me, 4)
    assert np.abs(Xi - X).max() < 1e-11 * np.abs(X).max()
    om = np.array([-7.0, 0.3, 6.0])
    dop = m.fermion_baths[0][0]
    A = so.dos(Mo, X, dop, om)
    Ai = so.dos_iterative(Mo, X, dop, om)
    assert np.abs(Ai - A).max() < 1e-11 * np.abs(A).max()
    # noninteracting level: A(w) = -Im G^R(w) / pi (closed form)
    lvl, _, _, Ml = _level(2)
    Xl = so.steady_state_iterative(Ml, 2)
    _, _, _, Mlo = _level(2, parity=-1)
    w = np.array([-2.0, 0.1, 0.9, 3.0])
    Al = so.dos_iterative(Mlo, Xl, lvl.fermion_baths[0][0], w)
    assert np.abs(Al - np.array([-_GR(x).imag / np.pi for x in w])).max() < 1e-10
