"""Pins of the oracle's Lindblad terms (Eq. Lindbladian) against closed forms and invariants.

What each test would catch:
* two-level decay      F and F^dagger swapped (pumping instead of decay), a missing 1/2 on the
                       anticommutator (coherences decay at gamma, trace lost), a wrong sign;
* thermal oscillator   rates attached to the wrong operator (inverted Boltzmann ratio);
* trace / Hermiticity  F X F in place of F X F^dagger, F F^dagger in place of F^dagger F;
* block structure      Lindblad terms added to some ADOs only, or ADOs added for them;
* charge-cavity at g=0 the master-equation workload's rates (the cavity marginal of the
                       stationary state must be the truncated thermal distribution).
"""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so


def _bare(d, H, lind):
    return dict(d=d, H=np.asarray(H, np.complex128), baths=[], tier_b=0, tier_f=0, parity=1,
                lindblad=[dict(op=np.asarray(F, np.complex128), rate=g) for F, g in lind])


def test_two_level_decay_closed_form():
    # H = (w/2) sz: E_0 = w/2, E_1 = -w/2; F = |0><1| decays level 1 at rate gamma:
    # rho_11(t) = rho_11(0) e^{-gamma t}, rho_01(t) = rho_01(0) e^{-i w t - gamma t / 2}.
    w, gam = 1.3, 0.4
    prob = _bare(2, 0.5 * w * W.SZ, [(W.SM, gam)])
    h = hy.problem_hierarchy(prob)
    assert h.n_ado == 1
    M = lv.build_matrix(prob, h)
    rho0 = np.array([[0.3, 0.2 + 0.1j], [0.2 - 0.1j, 0.7]])
    for t in (0.5, 2.0, 7.0):
        rho = lv.from_liouville(so.propagate_expm(M, lv.to_liouville(rho0[None]), t), 2)[0]
        p1 = 0.7 * np.exp(-gam * t)
        c = rho0[0, 1] * np.exp(-1j * w * t - 0.5 * gam * t)
        want = np.array([[1 - p1, c], [np.conj(c), p1]])
        np.testing.assert_allclose(rho, want, atol=1e-12)


def test_truncated_oscillator_thermal_state():
    # Loss a at gamma (n+1), gain a^dag at gamma n, H = w a^dag a: the stationary state of
    # the truncated birth-death chain obeys detailed balance, p_k ~ (n / (n + 1))^k.
    nf, w, gam, nth = 8, 1.0, 0.3, 0.6
    a = W.destroy(nf)
    prob = _bare(nf, w * W.dag(a) @ a, [(a, gam * (nth + 1)), (W.dag(a), gam * nth)])
    X = so.steady_state(lv.build_matrix(prob), nf)[0]
    p = (nth / (nth + 1)) ** np.arange(nf)
    np.testing.assert_allclose(X, np.diag(p / p.sum()), atol=1e-12)


def test_lindblad_preserves_trace_and_hermiticity():
    rng = np.random.default_rng(5)
    d = 5
    lind = [(W.random_complex((d, d), rng), float(rng.uniform(0.1, 1.0))) for _ in range(3)]
    terms = [(g, F) for F, g in lind]
    X = W.random_hermitian(d, rng)
    Y = lv.lindblad_apply(terms, X)
    assert abs(np.trace(Y)) < 1e-12 * np.abs(Y).max()
    np.testing.assert_allclose(Y, Y.conj().T, atol=1e-12)
    # non-Hermitian X: still traceless (Tr F X F^dagger = Tr F^dagger F X)
    Xc = W.random_complex((d, d), rng)
    assert abs(np.trace(lv.lindblad_apply(terms, Xc))) < 1e-12 * np.abs(Xc).max() * 10


@pytest.mark.parametrize("parity", [1, -1])
def test_lindblad_is_the_same_block_on_every_ado(parity):
    prob = W.random_raw_problem(3, [("RI", 2)], [4], 2, 2, parity=parity, seed=21,
                                n_lindblad=2)
    plain = dict(prob, lindblad=[])
    h = hy.problem_hierarchy(prob)
    assert h.n_ado == hy.problem_hierarchy(plain).n_ado
    diff = (lv.build_matrix(prob, h) - lv.build_matrix(plain, h)).toarray()
    # the Lindbladian alone on one ADO (no baths, H = 0)
    L1 = lv.build_matrix(_bare(3, np.zeros((3, 3)), [(t["op"], t["rate"])
                                                     for t in prob["lindblad"]])).toarray()
    D2 = 9
    for i in range(h.n_ado):
        for j in range(h.n_ado):
            blk = diff[i * D2:(i + 1) * D2, j * D2:(j + 1) * D2]
            np.testing.assert_allclose(blk, L1 if i == j else 0.0, atol=1e-13)
    # the loop path agrees with the matrix path
    X = W.random_ado_vector(h.n_ado, 3, seed=22)
    Y1 = lv.apply_loop(prob, X, h)
    Y2 = lv.from_liouville(lv.build_matrix(prob, h) @ lv.to_liouville(X), 3)
    np.testing.assert_allclose(Y1, Y2, atol=1e-12)


def test_charge_cavity_master_equation_decoupled_cavity_is_thermal():
    # g = 0: the cavity only meets its Lindblad terms, so the stationary state's cavity
    # marginal is the truncated thermal distribution with n = n_BE(w_c) whatever the leads do.
    nf = 4
    model = W.charge_cavity_me_model(g=0.0, n_fock=nf, tier_f=2)
    prob = hy.model_to_problem(model)
    X = so.steady_state(lv.build_matrix(prob), model.d)[0]
    cav = X.reshape(2, nf, 2, nf).trace(axis1=0, axis2=2)
    nth = W.bose_einstein(1.0, 0.5)
    p = (nth / (nth + 1)) ** np.arange(nf)
    np.testing.assert_allclose(cav, np.diag(p / p.sum()), atol=1e-10)
    np.testing.assert_allclose(np.trace(X), 1.0, atol=1e-12)
