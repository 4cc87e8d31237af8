"""Parity of the CUDA solvers (RK4, stationary state, density of states) with the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so
from tests.helpers import rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


def _oracle_rk4(prob, h, rho0, dt, n_steps, save_every):
    M = lv.build_matrix(prob, h)
    x0 = lv.to_liouville(so.initial_vector(h.n_ado, rho0))
    d = rho0.shape[0]
    _, snaps = so.rk4(lambda v: M @ v, x0, dt, n_steps, save_every,
                      observe=lambda v: lv.from_liouville(v[: d * d], d)[0])
    return np.array(snaps)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_evolve_spin_boson_matches_oracle_rk4(heom, prec, tol):
    """Spin-boson, tier 4 (35 ADOs), dt = 0.01 to t = 10, snapshots every 0.5."""
    import torch
    m = W.spin_boson_model(tier=4)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    ref = _oracle_rk4(prob, h, m.rho0, 0.01, 1000, 50)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    x = to_dev(so.initial_vector(h.n_ado, m.rho0), torch.complex128 if prec == "fp64" else torch.complex64)
    traj = heom.evolve(g, x, 0.01, 1000, 50)
    got = traj.cpu().numpy().astype(np.complex128)
    assert got.shape == ref.shape
    assert rel_err(got, ref) < tol
    tr = np.trace(got, axis1=1, axis2=2)
    assert np.abs(tr - 1).max() < (1e-12 if prec == "fp64" else 1e-5)


def test_evolve_wide_batch_matches_oracle(heom):
    """32 columns (the tiled kernel's launch shape), FP32 and FP64, against the oracle RK4."""
    import torch
    m = W.siam_model(tier=2)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    scales = np.linspace(0.2, 1.0, 32)
    X = np.stack([so.initial_vector(h.n_ado, np.diag([1 - s, 0.5 * s, 0.5 * s, 0]).astype(complex))
                  for s in scales], axis=-1)
    ref0 = _oracle_rk4(prob, h, np.diag([1 - scales[0], 0.5 * scales[0], 0.5 * scales[0], 0]).astype(complex), 0.005, 100, 50)
    ref9 = _oracle_rk4(prob, h, np.diag([1 - scales[9], 0.5 * scales[9], 0.5 * scales[9], 0]).astype(complex), 0.005, 100, 50)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    for dt_, tol in ((torch.complex128, 1e-10), (torch.complex64, 1e-5)):
        x = to_dev(X, dt_)
        got = heom.evolve(g, x, 0.005, 100, 50).cpu().numpy().astype(np.complex128)
        assert rel_err(got[..., 0], ref0) < tol and rel_err(got[..., 9], ref9) < tol


def test_evolve_batched_columns_are_independent(heom):
    import torch
    m = W.siam_model(tier=2)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    rhos = [np.diag(v).astype(complex) for v in ([1, 0, 0, 0], [0, 0.5, 0.5, 0], [0, 0, 0, 1])]
    X = np.stack([so.initial_vector(h.n_ado, r) for r in rhos], axis=-1)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    x = to_dev(X, torch.complex128)
    traj = heom.evolve(g, x, 0.005, 200, 100)
    got = traj.cpu().numpy()
    for j, r in enumerate(rhos):
        ref = _oracle_rk4(prob, h, r, 0.005, 200, 100)
        assert rel_err(got[..., j], ref) < 1e-10


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("name,model", [
    ("spin_boson_t4", lambda: W.spin_boson_model(tier=4)),
    ("siam_t2", lambda: W.siam_model(tier=2)),
    ("siam_t3", lambda: W.siam_model(tier=3)),
])
def test_steady_matches_oracle(heom, prec, name, model):
    import torch
    m = model()
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    Xo = so.steady_state(M, m.d)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    x = torch.zeros((h.n_ado, m.d, m.d), dtype=torch.complex128, device="cuda")
    st, stats = heom.steady(g, x, tol=1e-10, max_iter=3000, prec=getattr(heom, prec),
                            raise_on_error=False)
    X = x.cpu().numpy()
    assert st == heom.OK, stats
    assert stats[0]["residual"] <= 1e-10
    assert abs(np.trace(X[0]) - 1) < 1e-12
    # the oracle's own residual of the GPU solution (independent check of r_ss)
    assert so.steady_residual(M, X) <= 1.5e-10
    assert rel_err(X[0], Xo[0]) < 1e-7


def test_steady_batched_parameter_sets(heom):
    """Three SIAM parameter sets (different U, bias) solved as one batch."""
    import torch
    models = [W.siam_model(tier=2, U=u, mu=mu) for u, mu in ((10.0, 1.0), (4.0, 0.3), (7.0, 2.0))]
    g = heom.build_hierarchy(heom.problem_from_model(models[0]))
    Hs, coefs, rates = [], [], []
    for m in models:
        p = heom.problem_from_model(m)
        Hs.append(p["H"])
        coefs.append(np.concatenate([b["coef"] for b in p["baths"]]))
        rates.append(np.concatenate([b["rate"] for b in p["baths"]]))
    heom.set_params(g, np.array(Hs), np.array(coefs), np.array(rates))
    x = torch.zeros((g.n_ado, 4, 4, 3), dtype=torch.complex128, device="cuda")
    st, stats = heom.steady(g, x, tol=1e-9, max_iter=3000, prec=heom.MIXED)
    X = x.cpu().numpy()
    for j, m in enumerate(models):
        prob = hy.model_to_problem(m)
        h = hy.problem_hierarchy(prob)
        M = lv.build_matrix(prob, h)
        assert stats[j]["residual"] <= 1e-9
        assert rel_err(X[..., j][0], so.steady_state(M, 4)[0]) < 1e-6


def test_steady_warm_start_from_solution_needs_no_iterations(heom):
    import torch
    m = W.siam_model(tier=2)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    Xo = so.steady_state(lv.build_matrix(prob, h), 4)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    x0 = to_dev(Xo, torch.complex128)
    x = torch.zeros_like(x0)
    st, stats = heom.steady(g, x, x0=x0, tol=1e-8, prec=heom.MIXED)
    assert stats[0]["iterations"] == 0 and stats[0]["residual"] < 1e-8


@pytest.mark.parametrize("prec", ["FP64", "MIXED", "SHIFTED"])
def test_dos_noninteracting_level_closed_form(heom, prec):
    """A(w) = -Im G^R(w) / pi for a noninteracting level (odd-parity HEOM, tier 2)."""
    import torch
    eps, G, Wd, kT, mus = 0.3, 1.0, 4.0, 0.5, (1.0, -0.5)
    m = W.single_level_model(eps, G, Wd, kT, mus[0], mus[1], 4, 2)
    even = heom.build_hierarchy(heom.problem_from_model(m, 1))
    odd = heom.build_hierarchy(heom.problem_from_model(m, -1))
    x = torch.zeros((even.n_ado, 2, 2), dtype=torch.complex128, device="cuda")
    heom.steady(even, x, tol=1e-12, max_iter=4000, prec=heom.FP64)
    om = np.linspace(-6, 6, 25)
    A, st, stats = heom.spectrum(odd, x, m.fermion_baths[0][0], om, tol=1e-10, max_iter=4000,
                                 prec=getattr(heom, prec))
    GR = 1.0 / (om - eps - sum(0.5 * G * Wd / (om - mu + 1j * Wd) for mu in mus))
    assert np.abs(A - (-GR.imag / np.pi)).max() < 1e-8
    assert max(s["residual"] for s in stats) <= 1e-10


@pytest.mark.parametrize("prec", ["MIXED", "SHIFTED"])
def test_dos_siam_matches_oracle(heom, prec):
    import torch
    m = W.siam_model(tier=2)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    Xo = so.steady_state(M, 4)
    Mo = lv.build_matrix(hy.model_to_problem(m, -1), h)
    om = np.array([-12.0, -5.0, -1.0, 0.0, 0.7, 3.0, 9.0])
    Ao = so.dos(Mo, Xo, m.fermion_baths[0][0], om)
    odd = heom.build_hierarchy(heom.problem_from_model(m, -1))
    A, st, stats = heom.spectrum(odd, to_dev(Xo, torch.complex128), m.fermion_baths[0][0], om,
                                 tol=1e-10, max_iter=4000, prec=getattr(heom, prec))
    assert np.abs(A - Ao).max() < 1e-8 * np.abs(Ao).max()
    assert max(x["residual"] for x in stats) <= 1e-10


def test_dos_siam_tier3_many_frequencies_shifted(heom):
    """The benchmark shape: tier 3 (2,325 ADOs), 400 frequencies on [-20, 20]; sampled
    frequencies against the oracle's sparse-LU DOS."""
    import torch
    m = W.siam_model(tier=3)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    Xo = so.steady_state(lv.build_matrix(prob, h), 4)
    om = np.linspace(-20, 20, 400)
    odd = heom.build_hierarchy(heom.problem_from_model(m, -1))
    A, st, stats = heom.spectrum(odd, to_dev(Xo, torch.complex128), m.fermion_baths[0][0], om,
                                 tol=1e-8, max_iter=1000, prec=heom.SHIFTED)
    assert st == heom.OK and max(x["residual"] for x in stats) <= 1e-8
    idx = np.array([0, 57, 199, 200, 311, 399])
    Mo = lv.build_matrix(hy.model_to_problem(m, -1), h)
    Ao = so.dos(Mo, Xo, m.fermion_baths[0][0], om[idx])
    assert np.abs(A[idx] - Ao).max() < 1e-7 * np.abs(Ao).max()


def _set_params_of(heom, g, models, parity):
    Hs, coefs, rates = [], [], []
    for m in models:
        p = heom.problem_from_model(m, parity)
        Hs.append(p["H"])
        coefs.append(np.concatenate([b["coef"] for b in p["baths"]]))
        rates.append(np.concatenate([b["rate"] for b in p["baths"]]))
    heom.set_params(g, np.array(Hs), np.array(coefs), np.array(rates))


def test_dos_parameter_sets_shifted(heom):
    """Three SIAM parameter sets in one shift-invariant solve (two Krylov processes per set):
    every set's A(w) against the oracle's sparse-LU DOS of that set."""
    import torch
    models = [W.siam_model(tier=2, U=u, mu=mu, eps=e) for u, mu, e in
              ((10.0, 1.0, -5.0), (4.0, 0.3, -2.0), (7.0, 2.0, -3.5))]
    even = heom.build_hierarchy(heom.problem_from_model(models[0], 1))
    _set_params_of(heom, even, models, 1)
    odd = heom.build_hierarchy(heom.problem_from_model(models[0], -1))
    _set_params_of(heom, odd, models, -1)
    x = torch.zeros((even.n_ado, 4, 4, 3), dtype=torch.complex128, device="cuda")
    heom.steady(even, x, tol=1e-10, max_iter=3000, prec=heom.FP64)
    om = np.linspace(-15, 15, 61)
    A, st, stats = heom.spectrum(odd, x, models[0].fermion_baths[0][0], om, tol=1e-9,
                                 max_iter=1500, prec=heom.SHIFTED)
    assert A.shape == (3, 61) and len(stats) == 3 * 2 * 61
    assert st == heom.OK and max(s_["residual"] for s_ in stats) <= 1e-9
    idx = np.array([0, 13, 30, 31, 47, 60])
    for j, m in enumerate(models):
        prob = hy.model_to_problem(m)
        h = hy.problem_hierarchy(prob)
        Xo = so.steady_state(lv.build_matrix(prob, h), 4)
        Mo = lv.build_matrix(hy.model_to_problem(m, -1), h)
        Ao = so.dos(Mo, Xo, m.fermion_baths[0][0], om[idx])
        assert np.abs(A[j, idx] - Ao).max() < 1e-7 * np.abs(Ao).max(), j


def test_dos_two_parameter_sets_shifted(heom):
    """Two parameter sets (four Krylov processes, a column count the single-set persistent
    Arnoldi would take): each set's A(w) against the oracle's sparse-LU DOS of that set, so a
    solve that used one set's coefficients for every column fails."""
    import torch
    models = [W.siam_model(tier=2, U=u, mu=mu, eps=e) for u, mu, e in
              ((10.0, 1.0, -5.0), (3.0, 0.2, -1.5))]
    even = heom.build_hierarchy(heom.problem_from_model(models[0], 1))
    _set_params_of(heom, even, models, 1)
    odd = heom.build_hierarchy(heom.problem_from_model(models[0], -1))
    _set_params_of(heom, odd, models, -1)
    x = torch.zeros((even.n_ado, 4, 4, 2), dtype=torch.complex128, device="cuda")
    heom.steady(even, x, tol=1e-10, max_iter=3000, prec=heom.FP64)
    om = np.array([-9.0, -2.5, 0.0, 4.0, 11.0])
    A, st, stats = heom.spectrum(odd, x, models[0].fermion_baths[0][0], om, tol=1e-9,
                                 max_iter=1500, prec=heom.SHIFTED)
    assert st == heom.OK and A.shape == (2, 5)
    for j, m in enumerate(models):
        prob = hy.model_to_problem(m)
        h = hy.problem_hierarchy(prob)
        Xo = so.steady_state(lv.build_matrix(prob, h), 4)
        Ao = so.dos(lv.build_matrix(hy.model_to_problem(m, -1), h), Xo, m.fermion_baths[0][0], om)
        assert np.abs(A[j] - Ao).max() < 1e-7 * np.abs(Ao).max(), j


def test_current_matches_oracle(heom):
    """Lead currents from the tier-1 ADOs of GPU stationary states (one parameter set, then
    three biases batched as parameter sets) against the oracle's current of its own sparse-LU
    stationary states; I_L + I_R = 0."""
    import torch
    biases = (1.0, 0.4, 2.2)
    models = [W.siam_model(tier=2, mu=mu) for mu in biases]
    g = heom.build_hierarchy(heom.problem_from_model(models[0]))
    x = torch.zeros((g.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
    heom.steady(g, x, tol=1e-10, max_iter=3000, prec=heom.FP64)
    IL1 = heom.current(g, x, [0, 1])[0]
    IR1 = heom.current(g, x, [2, 3])[0]
    gb = heom.build_hierarchy(heom.problem_from_model(models[0]))
    _set_params_of(heom, gb, models, 1)
    xb = torch.zeros((gb.n_ado, 4, 4, 3), dtype=torch.complex128, device="cuda")
    heom.steady(gb, xb, tol=1e-10, max_iter=3000, prec=heom.FP64)
    IL = heom.current(gb, xb, [0, 1])
    IR = heom.current(gb, xb, [2, 3])
    for j, m in enumerate(models):
        prob = hy.model_to_problem(m)
        h = hy.problem_hierarchy(prob)
        X = so.steady_state(lv.build_matrix(prob, h), 4)
        il, ir = so.current(prob, h, X, [0, 1]), so.current(prob, h, X, [2, 3])
        assert abs(IL[j] - il) <= 1e-7 * abs(il), (j, IL[j], il)
        assert abs(IR[j] - ir) <= 1e-7 * abs(ir), (j, IR[j], ir)
        assert abs(IL[j] + IR[j]) <= 1e-7 * abs(il)
    assert abs(IL1 - IL[0]) <= 1e-8 * abs(IL[0]) and abs(IR1 - IR[0]) <= 1e-8 * abs(IR[0])


def test_psd_matches_oracle_and_sum_rule(heom):
    """Bosonic power spectrum by the shift-invariant solver: spin-boson sigma_z against the
    oracle's sparse-LU PSD at sampled frequencies and, over 4,000 frequencies, the sum rule
    (integral of S = <sigma_z sigma_z> = 1 since the stationary <sigma_z> vanishes); SIAM
    spin-up occupation against the oracle."""
    import torch
    m = W.spin_boson_model(tier=4)
    prob = hy.model_to_problem(m, 1)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    Xo = so.steady_state(M, m.d)
    g = heom.build_hierarchy(heom.problem_from_model(m, 1))
    x = torch.zeros((g.n_ado, 2, 2), dtype=torch.complex128, device="cuda")
    heom.steady(g, x, tol=1e-11, max_iter=3000, prec=heom.FP64)
    sz = np.diag([1.0, -1.0]).astype(complex)
    om = np.linspace(-50, 50, 4000)
    S, st, stats = heom.psd(g, x, sz, om, tol=1e-10, max_iter=1500)
    assert st == heom.OK and max(s_["residual"] for s_ in stats) <= 1e-10
    idx = np.array([0, 700, 1500, 1999, 2000, 2600, 3999])
    So = so.psd(M, Xo, sz, om[idx])
    assert np.abs(S[idx] - So).max() < 1e-7 * np.abs(So).max()
    assert abs(np.trapezoid(S, om) - 1.0) < 1e-6
    # SIAM (tier 2): occupation of the spin-up level, n = d^dag d
    ms = W.siam_model(tier=2)
    ps = hy.model_to_problem(ms, 1)
    hs = hy.problem_hierarchy(ps)
    Ms = lv.build_matrix(ps, hs)
    Xs = so.steady_state(Ms, 4)
    dup = ms.fermion_baths[0][0]
    nup = dup.conj().T @ dup
    gs = heom.build_hierarchy(heom.problem_from_model(ms, 1))
    xs = torch.zeros((gs.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
    heom.steady(gs, xs, tol=1e-11, max_iter=3000, prec=heom.FP64)
    oms = np.array([-12.0, -5.0, -1.3, 0.7, 3.0, 9.0])
    Sg, st, stats = heom.psd(gs, xs, nup, oms, tol=1e-10, max_iter=1500)
    assert st == heom.OK
    Sso = so.psd(Ms, Xs, nup, oms)
    assert np.abs(Sg - Sso).max() < 1e-7 * np.abs(Sso).max()


def test_spectrum_batched_over_hierarchies_of_different_shapes(heom):
    """heom_spectrum_batched over SIAM tier 1, a single level (d = 2, its own exponents) and
    SIAM tier 2: every hierarchy's result equals its own heom_spectrum call bit for bit, and
    the SIAM ones match the oracle's sparse LU."""
    import torch
    models = [W.siam_model(tier=1), W.single_level_model(tier=2), W.siam_model(tier=2)]
    om = np.array([-9.0, -3.0, 0.4, 5.0])
    odds, sss, ops, singles = [], [], [], []
    for m in models:
        even = heom.build_hierarchy(heom.problem_from_model(m, 1))
        odd = heom.build_hierarchy(heom.problem_from_model(m, -1))
        x = torch.zeros((even.n_ado, m.d, m.d), dtype=torch.complex128, device="cuda")
        heom.steady(even, x, tol=1e-11, max_iter=3000, prec=heom.FP64)
        dop = m.fermion_baths[0][0]
        A1, st, _ = heom.spectrum(odd, x, dop, om, tol=1e-10, max_iter=2000, prec=heom.SHIFTED)
        assert st == heom.OK
        odds.append(odd)
        sss.append(x)
        ops.append(dop)
        singles.append(A1)
    As, st, stats = heom.spectrum_batched(odds, sss, ops, om, tol=1e-10, max_iter=2000)
    assert st == heom.OK and len(stats) == 2 * len(om) * 3
    for A, A1 in zip(As, singles):
        assert np.array_equal(A, A1)
    for i in (0, 2):
        m = models[i]
        prob = hy.model_to_problem(m)
        h = hy.problem_hierarchy(prob)
        Xo = so.steady_state(lv.build_matrix(prob, h), m.d)
        Ao = so.dos(lv.build_matrix(hy.model_to_problem(m, -1), h), Xo, m.fermion_baths[0][0], om)
        assert np.abs(As[i] - Ao).max() < 1e-8 * np.abs(Ao).max()


def test_steady_fp64_strict_matches_oracle(heom):
    """HEOM_FP64_STRICT (FP64 applies everywhere, no float-float persistent kernel): one column
    and two columns against the oracle's sparse-LU stationary state, SIAM tier 2."""
    import torch
    m = W.siam_model(tier=2)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    M = lv.build_matrix(prob, h)
    Xo = so.steady_state(M, 4)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    for shape in ((h.n_ado, 4, 4), (h.n_ado, 4, 4, 2)):
        x = torch.zeros(shape, dtype=torch.complex128, device="cuda")
        st, stats = heom.steady(g, x, tol=1e-10, max_iter=4000, prec=heom.FP64_STRICT)
        assert st == heom.OK and all(s_["residual"] <= 1e-10 for s_ in stats)
        X = x.cpu().numpy()
        X = X if X.ndim == 3 else X[..., 1]
        assert np.abs(X - Xo).max() < 1e-8 * np.abs(Xo).max()
