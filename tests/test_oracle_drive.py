"""Pins of the oracle's time-dependent system Hamiltonian H(t) = H + sum_k f_k(t) H_k.

What each test would catch:
* Rabi closed form         a wrong sign of the drive commutator, f_k applied to the wrong
                           operator, a drive missing from some stage;
* fourth order in dt       f_k sampled at the wrong stage times (every stage at t_n makes the
                           scheme first order in the time dependence);
* Bloch steady state       a drive that breaks with Lindblad terms or baths on other ADOs;
* constant drive           a drive that differs from adding c H_k to H.
"""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so


def _circular(w, Om, dt, n_steps):
    """H(t) = (w/2) sz + (Om/2)(cos(w t) sx + sin(w t) sy): in the frame rotating with
    exp(i w t sz / 2) the Hamiltonian is (Om/2) sx exactly (no rotating-wave step)."""
    t = 0.5 * dt * np.arange(2 * n_steps + 1)
    return [0.5 * Om * W.SX, 0.5 * Om * W.SY], np.stack([np.cos(w * t), np.sin(w * t)])


def _bare(H, lind=()):
    return dict(d=2, H=H, baths=[], tier_b=0, tier_f=0, parity=1,
                lindblad=[dict(op=F, rate=g) for F, g in lind])


def _rabi_error(dt, T=5.0, w=2.0, Om=1.3):
    n = int(round(T / dt))
    ops, f = _circular(w, Om, dt, n)
    prob = _bare(0.5 * w * W.SZ)
    M0 = lv.build_matrix(prob)
    Ls = so.drive_superoperators(1, ops)
    x0 = lv.to_liouville(np.array([[[1, 0], [0, 0]]], complex))
    x, _ = so.rk4_td(M0, Ls, f, x0, dt, n)
    rho = lv.from_liouville(x, 2)[0]
    t = n * dt
    p1 = np.sin(0.5 * Om * t) ** 2
    c = 0.5j * np.sin(Om * t) * np.exp(-1j * w * t)
    want = np.array([[1 - p1, c], [np.conj(c), p1]])
    return np.abs(rho - want).max()


def test_rabi_closed_form_and_fourth_order():
    e1, e2 = _rabi_error(0.05), _rabi_error(0.025)
    assert e2 < 1e-6
    assert e1 / e2 > 12.0  # 2^4 = 16 for a fourth-order scheme


def test_driven_decay_reaches_bloch_steady_state():
    # excited level 0 (energy +w/2) decays to 1 with F = |1><0| at rate g; on resonance the
    # stationary excited population is Om^2 / (g^2 + 2 Om^2)
    # (RK4 at dt = 0.02 leaves 6e-9; the other jump direction would give 1 - 0.409)
    w, Om, g, dt, n = 2.0, 1.5, 1.0, 0.02, 3000
    ops, f = _circular(w, Om, dt, n)
    prob = _bare(0.5 * w * W.SZ, [(W.SM.T.copy(), g)])
    M0 = lv.build_matrix(prob)
    x0 = lv.to_liouville(np.array([[[0, 0], [0, 1]]], complex))
    x, _ = so.rk4_td(M0, so.drive_superoperators(1, ops), f, x0, dt, n)
    assert abs(lv.from_liouville(x, 2)[0][0, 0] - Om ** 2 / (g ** 2 + 2 * Om ** 2)) < 1e-7


def test_constant_drive_equals_static_hamiltonian():
    m = W.spin_boson_model(tier=3)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    c, dt, n = 0.7, 0.01, 200
    Hk = W.SZ
    M0 = lv.build_matrix(prob, h)
    x0 = lv.to_liouville(so.initial_vector(h.n_ado, m.rho0))
    x_td, _ = so.rk4_td(M0, so.drive_superoperators(h.n_ado, [Hk]),
                        np.full((1, 2 * n + 1), c), x0, dt, n)
    Ms = lv.build_matrix(dict(prob, H=prob["H"] + c * Hk), h)
    x_st, _ = so.rk4(lambda v: Ms @ v, x0, dt, n)
    np.testing.assert_allclose(x_td, x_st, atol=1e-13)
