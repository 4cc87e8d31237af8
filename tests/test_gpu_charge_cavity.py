"""The charge-cavity workload end to end: a spinless level coupled to a cavity mode truncated
at 12 Fock states (d = 24), a Drude-Lorentz cavity-loss bath (3 exponents, tier 2) and two
Lorentzian leads (12 exponents, tier 2): 790 ADOs of 24 x 24 (Example 2, Table 1 row 2).
RK4 (dt = 0.01 to t = 5) against the oracle's RK4, FP64 and FP32; the stationary state
(FP64 and mixed precision) through the oracle's assembled M: Tr rho = 1, rho Hermitian and
r_ss = ||M x|| / ||x|| at the solver's tolerance. The stationary state is M's unique null
vector of unit trace, so the residual pins it; the oracle's own GMRES solve of these
455,040 unknowns takes minutes, its sparse LU longer."""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so

pytestmark = pytest.mark.gpu

DT, STEPS, SAVE = 0.01, 500, 100


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


@pytest.fixture(scope="module")
def cavity():
    m = W.charge_cavity_model()
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    assert (h.n_ado, m.d) == (790, 24)
    M = lv.build_matrix(prob, h)
    x0 = lv.to_liouville(so.initial_vector(h.n_ado, m.rho0))
    _, snaps = so.rk4(lambda v: M @ v, x0, DT, STEPS, SAVE,
                      observe=lambda v: lv.from_liouville(v[:m.d ** 2], m.d)[0])
    return m, h, M, np.array(snaps)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_charge_cavity_rk4_matches_oracle(heom, cavity, prec, tol):
    import torch
    m, h, M, snaps = cavity
    g = heom.build_hierarchy(heom.problem_from_model(m))
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    x = torch.from_numpy(so.initial_vector(h.n_ado, m.rho0)).to("cuda", dt)
    traj = heom.evolve(g, x, DT, STEPS, SAVE).cpu().numpy().astype(np.complex128)
    assert traj.shape == snaps.shape
    err = np.abs(traj - snaps).max() / np.abs(snaps).max()
    assert err < tol, err
    tr = np.trace(traj, axis1=1, axis2=2)
    assert np.abs(tr - 1).max() < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_charge_cavity_stationary_state(heom, cavity, prec):
    import torch
    m, h, M, _ = cavity
    g = heom.build_hierarchy(heom.problem_from_model(m))
    x = torch.zeros((h.n_ado, 24, 24), dtype=torch.complex128, device="cuda")
    st, stats = heom.steady(g, x, tol=1e-9, max_iter=6000, prec=getattr(heom, prec))
    assert st == heom.OK
    X = x.cpu().numpy()
    rho = X[0]
    assert abs(np.trace(rho) - 1) < 1e-12
    assert np.abs(rho - rho.conj().T).max() < 1e-8
    assert np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min() > -1e-8
    assert so.steady_residual(M, X) < 2e-9
