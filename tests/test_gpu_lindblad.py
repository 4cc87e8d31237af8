"""Parity of the Lindblad terms (Eq. Lindbladian) on the GPU with the oracle and closed forms.

The terms enter every kernel through the ADO-local system superoperator, so each path is
exercised: the per-element apply (batch < 16) and the tiled apply (batch >= 16), RK4
dynamics, the persistent and batched stationary solvers, and both spectra (the
shift-invariant solver on the odd sector for the DOS, on the even sector for the PSD).
Tolerances are those of the plain apply tests (FP64 1e-10, FP32 1e-5, relative to max|y|) and
of the solver tests (residual 1e-10; tier-0 block 1e-7; spectra 1e-7 relative).
"""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so
from tests.helpers import oracle_apply_batched, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


def _apply(heom, g, X, prec):
    import torch
    x = to_dev(X, torch.complex128 if prec == "fp64" else torch.complex64)
    y = torch.empty_like(x)
    heom.apply(g, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("batch", [1, 5, 64])
@pytest.mark.parametrize("parity", [1, -1])
def test_apply_with_lindblad_random(heom, prec, batch, parity):
    prob = W.random_raw_problem(3, [("RI", 2), ("I", 1)], [4, 2], 2, 2, parity=parity,
                                seed=41, n_lindblad=3)
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, batch, seed=42)
    Y = oracle_apply_batched(prob, h, X)
    g = heom.build_hierarchy(prob)
    Yg = _apply(heom, g, X if batch > 1 else X[..., 0], prec)
    if batch == 1:
        Yg = Yg[..., None]
    assert rel_err(Yg, Y) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_charge_cavity_master_equation_full_size(heom, prec):
    """Example 2's master-equation variant at d = 24 (12 Fock states), fermionic tier 2."""
    m = W.charge_cavity_me_model()
    prob_o = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob_o)
    X = W.random_ado_vector(h.n_ado, m.d, 16, seed=43)
    Y = oracle_apply_batched(prob_o, h, X)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    assert g.n_ado == h.n_ado
    assert rel_err(_apply(heom, g, X, prec), Y) < TOL[prec]


def test_set_lindblad_replace_remove_and_reject(heom):
    """Removing the terms restores the plain apply bit for bit; the terms survive
    heom_set_params; a rejected call leaves the previous terms in place."""
    prob = W.random_raw_problem(3, [("RI", 2)], [4], 2, 1, seed=44, n_lindblad=2)
    plain = dict(prob, lindblad=[])
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, 3, seed=45)
    g0 = heom.build_hierarchy(plain)
    g = heom.build_hierarchy(prob)
    y_l = _apply(heom, g, X, "fp64")
    heom.set_lindblad(g, [], [])
    assert np.array_equal(_apply(heom, g, X, "fp64"), _apply(heom, g0, X, "fp64"))
    ops = [t["op"] for t in prob["lindblad"]]
    rates = [t["rate"] for t in prob["lindblad"]]
    heom.set_lindblad(g, ops, rates)
    assert np.array_equal(_apply(heom, g, X, "fp64"), y_l)
    with pytest.raises(heom.HeomError):
        heom.set_lindblad(g, ops, [rates[0], float("nan")])
    assert np.array_equal(_apply(heom, g, X, "fp64"), y_l)
    K = 4 + 2
    coef = np.concatenate([b["coef"] for b in prob["baths"]])[None]
    rate = np.concatenate([b["rate"] for b in prob["baths"]])[None]
    assert coef.shape == (1, K)
    heom.set_params(g, prob["H"][None], coef, rate)
    assert rel_err(_apply(heom, g, X, "fp64"), y_l) < 1e-14


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_evolve_two_level_decay_closed_form(heom, prec, tol):
    """No baths (one ADO): rho_11 = rho_11(0) e^{-gamma t}, rho_01 = rho_01(0) e^{-i w t -
    gamma t / 2} for H = (w/2) sz and F = |0><1|; RK4 at dt = 0.01 to t = 5."""
    import torch
    w, gam = 1.3, 0.4
    prob = dict(d=2, H=0.5 * w * W.SZ, baths=[], tier_b=0, tier_f=0, parity=1,
                lindblad=[dict(op=W.SM, rate=gam)])
    g = heom.build_hierarchy(prob)
    assert g.n_ado == 1
    rho0 = np.array([[0.3, 0.2 + 0.1j], [0.2 - 0.1j, 0.7]])
    x = to_dev(rho0[None], torch.complex128 if prec == "fp64" else torch.complex64)
    traj = heom.evolve(g, x, 0.01, 500, 100).cpu().numpy().astype(np.complex128)
    for s, rho in enumerate(traj):
        t = s * 1.0
        p1 = 0.7 * np.exp(-gam * t)
        c = rho0[0, 1] * np.exp(-1j * w * t - 0.5 * gam * t)
        want = np.array([[1 - p1, c], [np.conj(c), p1]])
        assert np.abs(rho - want).max() < tol


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_steady_thermal_oscillator_closed_form(heom, prec):
    """Loss a at gamma (n+1), gain a^dag at gamma n: p_k ~ (n / (n+1))^k (detailed balance of
    the truncated chain)."""
    import torch
    nf, w, gam, nth = 10, 1.0, 0.3, 0.6
    a = W.destroy(nf)
    prob = dict(d=nf, H=w * W.dag(a) @ a, baths=[], tier_b=0, tier_f=0, parity=1,
                lindblad=[dict(op=a, rate=gam * (nth + 1)), dict(op=W.dag(a), rate=gam * nth)])
    g = heom.build_hierarchy(prob)
    x = torch.zeros((1, nf, nf), dtype=torch.complex128, device="cuda")
    st, stats = heom.steady(g, x, tol=1e-11, max_iter=3000, prec=getattr(heom, prec))
    assert st == heom.OK and stats[0]["residual"] <= 1e-11
    p = (nth / (nth + 1)) ** np.arange(nf)
    assert np.abs(x.cpu().numpy()[0] - np.diag(p / p.sum())).max() < 1e-9


@pytest.fixture(scope="module")
def cc_me():
    """Charge-cavity master-equation model, 4 Fock states (d = 8), tier 2: oracle stationary
    state, even and odd sector matrices."""
    m = W.charge_cavity_me_model(n_fock=4, tier_f=2)
    pe = hy.model_to_problem(m, 1)
    po = hy.model_to_problem(m, -1)
    he = hy.problem_hierarchy(pe)
    Me = lv.build_matrix(pe, he)
    Mo = lv.build_matrix(po, hy.problem_hierarchy(po))
    return m, he, Me, Mo, so.steady_state(Me, m.d)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_steady_charge_cavity_master_equation(heom, cc_me, prec):
    import torch
    m, he, Me, _, Xo = cc_me
    g = heom.build_hierarchy(heom.problem_from_model(m, 1))
    x = torch.zeros((he.n_ado, m.d, m.d), dtype=torch.complex128, device="cuda")
    st, stats = heom.steady(g, x, tol=1e-10, max_iter=3000, prec=getattr(heom, prec))
    X = x.cpu().numpy()
    assert st == heom.OK and stats[0]["residual"] <= 1e-10
    assert so.steady_residual(Me, X) <= 1.5e-10
    assert rel_err(X[0], Xo[0]) < 1e-7


def test_spectra_charge_cavity_master_equation(heom, cc_me):
    """Cavity PSD (a) on the even sector and charge DOS (d) on the odd sector, both with the
    Lindblad terms, against the oracle's sparse LU at sampled frequencies."""
    import torch
    m, he, Me, Mo, Xo = cc_me
    pe = heom.problem_from_model(m, 1)
    po = heom.problem_from_model(m, -1)
    ge, go = heom.build_hierarchy(pe), heom.build_hierarchy(po)
    x = torch.zeros((he.n_ado, m.d, m.d), dtype=torch.complex128, device="cuda")
    heom.steady(ge, x, tol=1e-11, max_iter=3000, prec=heom.FP64)
    a = np.kron(np.eye(2), W.destroy(4))
    d = np.kron(W.SM, np.eye(4))
    om = np.array([-3.0, -0.4, 0.2, 0.6, 1.0, 1.7, 4.0])
    S, st, stats = heom.psd(ge, x, a, om, tol=1e-10, max_iter=1500)
    assert st == heom.OK
    So = so.psd(Me, Xo, a, om)
    assert np.abs(S - So).max() < 1e-7 * np.abs(So).max()
    # w = 0: (M - i w) x = a rho_ss has no solution when <a> = Tr(a rho_ss) != 0 (the trace
    # functional is a left null vector of M); the coherent part is a delta at w = 0. That
    # frequency reports ENOCONV, the other one of the same call still converges.
    assert abs(np.trace(a @ Xo[0])) > 0.1
    S0, st, stats = heom.psd(ge, x, a, np.array([0.0, 1.0]), tol=1e-8, max_iter=400,
                             raise_on_error=False)
    assert st == heom.ENOCONV
    assert stats[0]["status"] == heom.ENOCONV and stats[1]["status"] == heom.OK
    assert abs(S0[1] - so.psd(Me, Xo, a, [1.0])[0]) < 1e-6 * abs(So).max()
    A, st, _ = heom.spectrum(go, x, d, om, tol=1e-10, max_iter=1500, prec=heom.SHIFTED)
    assert st == heom.OK
    Ao = so.dos(Mo, Xo, d, om)
    assert np.abs(A - Ao).max() < 1e-7 * np.abs(Ao).max()
