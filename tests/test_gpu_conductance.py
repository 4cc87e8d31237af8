"""Differential conductance G = dI/dPhi (Methods, electronic current) by heom_conductance:
one batched stationary solve over bias pairs, lead currents, difference quotients. Checked
against the oracle's difference quotient of its own sparse-LU currents (SIAM), and against
the Landauer formula's difference quotient for a noninteracting level, where the current with
the Pade Fermi function of the truncated exponents is exact."""
import numpy as np
import pytest
from scipy.integrate import quad

import workloads as W
from oracle import exponents as ex
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


def _pairs(heom, build, phis, dphi):
    """An even hierarchy holding sets at Phi_k and Phi_k + dphi (mu_L = +Phi/2, mu_R = -Phi/2)."""
    models = []
    for p in phis:
        models += [build(p / 2), build((p + dphi) / 2)]
    g = heom.build_hierarchy(heom.problem_from_model(models[0], 1))
    heom.set_params_from_models(g, models, 1)
    return g, models


def test_conductance_siam_matches_oracle_difference_quotient(heom):
    phis, dphi = np.array([1.0, 3.0, 6.0]), 0.04
    g, models = _pairs(heom, lambda mu: W.siam_model(tier=2, mu=mu), phis, dphi)
    G, I, st, stats = heom.conductance(g, np.full(3, dphi), [0, 1], tol=1e-11)
    assert st == heom.OK
    for k in range(3):
        Io = []
        for m in models[2 * k:2 * k + 2]:
            prob = hy.model_to_problem(m)
            h = hy.problem_hierarchy(prob)
            X = so.steady_state(lv.build_matrix(prob, h), 4)
            Io.append(so.current(prob, h, X, [0, 1]))
        assert abs(I[2 * k] - Io[0]) < 1e-8 and abs(I[2 * k + 1] - Io[1]) < 1e-8
        Go = (Io[1] - Io[0]) / dphi
        assert abs(G[k] - Go) < 1e-6 * max(abs(Go), 1e-3), (k, G[k], Go)
    # the right lead carries the opposite current, so the opposite conductance
    GR, _, _, _ = heom.conductance(g, np.full(3, dphi), [2, 3], tol=1e-11)
    assert np.abs(GR + G).max() < 1e-6 * np.abs(G).max()
    with pytest.raises(ValueError):
        heom.conductance(g, np.full(2, dphi), [0, 1])


def test_conductance_noninteracting_level_matches_landauer(heom):
    eps, gam, wb, kt, npol = 0.3, 1.0, 4.0, 0.5, 4
    phis, dphi = np.array([0.4, 1.2, 2.5]), 0.02

    def build(mu):
        return W.single_level_model(eps, gam, wb, kt, mu, -mu, npol, tier=2)

    g, _ = _pairs(heom, build, phis, dphi)
    G, I, st, _ = heom.conductance(g, np.full(3, dphi), [0], tol=1e-12)
    assert st == heom.OK
    kap, zet = ex.pade_constants(npol, "fermi")

    def landauer(phi):
        mu = (phi / 2, -phi / 2)
        J = lambda w, m: gam * wb ** 2 / ((w - m) ** 2 + wb ** 2)
        GR = lambda w: 1.0 / (w - eps - sum(0.5 * gam * wb / (w - m + 1j * wb) for m in mu))
        f = lambda w, m: ex.fermi_approx((w - m) / kt, kap, zet).real
        return quad(lambda w: abs(GR(w)) ** 2 * J(w, mu[0]) * J(w, mu[1]) * (f(w, mu[0]) - f(w, mu[1]))
                    / (2 * np.pi), -np.inf, np.inf, limit=500, epsabs=1e-14)[0]

    for k, p in enumerate(phis):
        I0, I1 = landauer(p), landauer(p + dphi)
        assert abs(I[2 * k] - I0) < 1e-9 and abs(I[2 * k + 1] - I1) < 1e-9
        assert abs(G[k] - (I1 - I0) / dphi) < 1e-6, (k, G[k], (I1 - I0) / dphi)
