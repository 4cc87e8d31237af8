"""Time-dependent system Hamiltonian H(t) = H + sum_k f_k(t) H_k (heom_set_drive,
heom_evolve_td) on the GPU against closed forms and the oracle's RK4.

Tolerances: against the oracle FP64 1e-10 and FP32 1e-5 relative to max|rho|, as for the
time-independent RK4; against closed forms the RK4 truncation error bounds them.
"""
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


def _circular(w, Om, dt, n_steps):
    t = 0.5 * dt * np.arange(2 * n_steps + 1)
    return [0.5 * Om * W.SX, 0.5 * Om * W.SY], np.stack([np.cos(w * t), np.sin(w * t)])


@pytest.mark.parametrize("prec,tol,tol_o", [("fp64", 3e-9, 1e-12), ("fp32", 2e-5, 2e-5)])
def test_rabi_closed_form(heom, prec, tol, tol_o):
    """Circularly driven two-level system (no baths): P_1 = sin^2(Om t / 2) and rho_01 =
    (i/2) sin(Om t) e^{-i w t}, to within RK4's truncation error at dt = 0.005 (about 1e-9 at
    t = 6, from the oracle's measured fourth-order convergence), and the oracle's RK4 itself
    to rounding; 1,200 steps cross two chunks of drive samples."""
    import torch
    w, Om, dt, n = 2.0, 1.3, 0.005, 1200
    prob = dict(d=2, H=0.5 * w * W.SZ, baths=[], tier_b=0, tier_f=0, parity=1)
    g = heom.build_hierarchy(prob)
    ops, f = _circular(w, Om, dt, n)
    heom.set_drive(g, ops)
    x = to_dev(np.array([[[1, 0], [0, 0]]], complex),
               torch.complex128 if prec == "fp64" else torch.complex64)
    traj = heom.evolve_td(g, x, dt, n, f, save_every=100).cpu().numpy().astype(complex)
    x0 = lv.to_liouville(np.array([[[1, 0], [0, 0]]], complex))
    _, snaps = so.rk4_td(lv.build_matrix(prob), so.drive_superoperators(1, ops), f, x0, dt, n, 100,
                         observe=lambda v: lv.from_liouville(v, 2)[0])
    assert np.abs(traj - np.array(snaps)).max() < tol_o
    for s_, rho in enumerate(traj):
        t = s_ * 100 * dt
        p1 = np.sin(0.5 * Om * t) ** 2
        c = 0.5j * np.sin(Om * t) * np.exp(-1j * w * t)
        assert np.abs(rho - np.array([[1 - p1, c], [np.conj(c), p1]])).max() < tol, s_


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("batch", [1, 32])
def test_driven_spin_boson_matches_oracle(heom, prec, tol, batch):
    """Spin-boson (tier 4, 35 ADOs) with a pulsed sigma_x drive and a cosine sigma_z drive;
    batch 32 runs the tiled stage kernel."""
    import torch
    m = W.spin_boson_model(tier=4)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    dt, n = 0.01, 600
    t = 0.5 * dt * np.arange(2 * n + 1)
    f = np.stack([0.8 * np.exp(-((t - 2.0) / 0.7) ** 2), 0.3 * np.cos(1.7 * t)])
    ops = [W.SX, W.SZ]
    x0 = lv.to_liouville(so.initial_vector(h.n_ado, m.rho0))
    _, snaps = so.rk4_td(lv.build_matrix(prob, h), so.drive_superoperators(h.n_ado, ops), f, x0,
                         dt, n, 50, observe=lambda v: lv.from_liouville(v[:4], 2)[0])
    ref = np.array(snaps)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    heom.set_drive(g, ops)
    X0 = so.initial_vector(h.n_ado, m.rho0)
    if batch > 1:
        X0 = np.repeat(X0[..., None], batch, axis=-1)
    x = to_dev(X0, torch.complex128 if prec == "fp64" else torch.complex64)
    got = heom.evolve_td(g, x, dt, n, f, save_every=50).cpu().numpy().astype(complex)
    if batch > 1:
        assert np.abs(got - got[..., :1]).max() == 0.0  # identical columns, identical results
        got = got[..., 0]
    assert rel_err(got, ref) < tol


def test_zero_drive_is_heom_evolve_bit_for_bit(heom):
    import torch
    m = W.spin_boson_model(tier=4)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    heom.set_drive(g, [W.SX])
    X0 = so.initial_vector(g.n_ado, m.rho0)
    x1 = to_dev(X0, torch.complex128)
    x2 = to_dev(X0, torch.complex128)
    n = 300
    heom.evolve_td(g, x1, 0.01, n, np.zeros((1, 2 * n + 1)))
    heom.evolve(g, x2, 0.01, n)
    assert torch.equal(x1, x2)


def test_drive_with_parameter_sets(heom):
    """Two parameter sets (different H) share the drive; each column follows its own H(t)."""
    import torch
    m = W.spin_boson_model(tier=3)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    Hs = [prob["H"], prob["H"] + 0.4 * W.SZ]
    prob_g = heom.problem_from_model(m)
    coef = np.concatenate([b["coef"] for b in prob_g["baths"]])
    rate = np.concatenate([b["rate"] for b in prob_g["baths"]])
    dt, n = 0.01, 400
    t = 0.5 * dt * np.arange(2 * n + 1)
    f = np.sin(2.3 * t)[None]
    g = heom.build_hierarchy(prob_g)
    heom.set_params(g, np.stack(Hs), np.stack([coef, coef]), np.stack([rate, rate]))
    heom.set_drive(g, [W.SX])
    X0 = np.repeat(so.initial_vector(h.n_ado, m.rho0)[..., None], 2, axis=-1)
    x = to_dev(X0, torch.complex128)
    heom.evolve_td(g, x, dt, n, f)
    got = x.cpu().numpy()
    x0 = lv.to_liouville(so.initial_vector(h.n_ado, m.rho0))
    for s_, H in enumerate(Hs):
        M0 = lv.build_matrix(dict(prob, H=H), h)
        xe, _ = so.rk4_td(M0, so.drive_superoperators(h.n_ado, [W.SX]), f, x0, dt, n)
        assert rel_err(got[..., s_], lv.from_liouville(xe, 2)) < 1e-10
