"""Per-set truncation (heom_set_truncation): parameter sets of different depths in one
hierarchy of the deepest structure. Each set's columns must equal the oracle's result for that
set's own, shallower hierarchy -- apply, stationary state and density of states -- and the
batched-spectra workload (64 SIAM sets, tiers 2 to 4, 4,096 frequencies) is checked on sampled
(set, frequency) pairs against the oracle, a tier-4 set (12,951 ADOs) included."""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so
from tests.helpers import oracle_apply_batched, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


def test_apply_per_set_tiers(heom):
    """Four parameter sets (two columns each) truncated at tiers (b, f) = (2, 2), (1, 2),
    (2, 1), (0, 0) inside a (2, 2) hierarchy with bosonic and fermionic baths: each set's
    columns equal the oracle's apply of its own hierarchy on the leading ADOs, and zero
    beyond them; FP64 and FP32."""
    import torch
    prob = W.random_raw_problem(3, [("RI", 2)], [4], 2, 2, parity=1, seed=51)
    rng = np.random.default_rng(52)
    caps = [(2, 2), (1, 2), (2, 1), (0, 0)]
    probs = []
    for s in range(4):
        p = dict(prob, H=W.random_hermitian(3, rng))
        p["baths"] = [dict(b, coef=W.random_complex(len(b["coef"]), rng) * 0.3,
                           rate=rng.uniform(0.2, 2, len(b["coef"])) + 0.1j) for b in prob["baths"]]
        probs.append(p)
    g = heom.build_hierarchy(prob)
    heom.set_params(g, np.array([p["H"] for p in probs]),
                    np.array([np.concatenate([b["coef"] for b in p["baths"]]) for p in probs]),
                    np.array([np.concatenate([b["rate"] for b in p["baths"]]) for p in probs]))
    heom.set_truncation(g, [c[0] for c in caps], [c[1] for c in caps])
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, 8, seed=53)
    for s, (tb, tf) in enumerate(caps):  # inputs zero beyond each set's tiers
        ps = dict(probs[s], tier_b=tb, tier_f=tf)
        hs = hy.problem_hierarchy(ps)
        keep = np.array([h.index[a] for a in hs.ados])
        mask = np.ones(h.n_ado, bool)
        mask[keep] = False
        X[mask, ..., 2 * s:2 * s + 2] = 0
    for dt, tol in ((torch.complex128, 1e-10), (torch.complex64, 1e-5)):
        x = to_dev(X, dt)
        y = torch.empty_like(x)
        heom.apply(g, x, y)
        Y = y.cpu().numpy().astype(np.complex128)
        for s, (tb, tf) in enumerate(caps):
            ps = dict(probs[s], tier_b=tb, tier_f=tf)
            hs = hy.problem_hierarchy(ps)
            # the truncated hierarchy's ADOs, at their places in the deeper one (same relative
            # order: both are canonical)
            keep = np.array([h.index[a] for a in hs.ados])
            assert np.all(np.diff(keep) > 0)
            Ys = oracle_apply_batched(ps, hs, X[keep][..., 2 * s:2 * s + 2])
            assert rel_err(Y[keep][..., 2 * s:2 * s + 2], Ys) < tol, (s, dt)
            dropped = np.setdiff1d(np.arange(h.n_ado), keep)
            if dropped.size:
                assert np.abs(Y[dropped][..., 2 * s:2 * s + 2]).max() == 0.0
    heom.set_truncation(g)  # removed: the full hierarchy again
    with pytest.raises(heom.HeomError):
        heom.set_truncation(g, [3, 0, 0, 0], [0, 0, 0, 0])  # beyond the structure's tiers


def _c3(heom, draws):
    """Even and odd tier-4 SIAM hierarchies holding one parameter set per draw, each set
    truncated at its drawn tier (the batched-spectra workload's construction)."""
    models = [W.siam_model(U=d["U"], mu=d["mu"], kT=d["kT"], tier=4) for d in draws]
    tiers = [d["tier"] for d in draws]
    out = []
    for parity in (1, -1):
        g = heom.build_hierarchy(heom.problem_from_model(models[0], parity))
        heom.set_params_from_models(g, models, parity)
        heom.set_truncation(g, [0] * len(draws), tiers)
        out.append(g)
    return models, tiers, out[0], out[1]


def _oracle_dos(draw, om, iterative):
    """The oracle's stationary state and DOS of one drawn set at its own tier."""
    mt = W.siam_model(U=draw["U"], mu=draw["mu"], kT=draw["kT"], tier=draw["tier"])
    pe = hy.model_to_problem(mt, 1)
    h = hy.problem_hierarchy(pe)
    Me = lv.build_matrix(pe, h)
    Mo = lv.build_matrix(hy.model_to_problem(mt, -1), h)
    if iterative:
        X = so.steady_state_iterative(Me, 4)
        return X, so.dos_iterative(Mo, X, mt.fermion_baths[0][0], om), Me
    X = so.steady_state(Me, 4)
    return X, so.dos(Mo, X, mt.fermion_baths[0][0], om), Me


def test_uneven_tiers_steady_and_dos_small(heom):
    """Three SIAM sets of tiers 2, 3, 2 in one tier-3 structure: stationary states (batched,
    mixed precision) and DOS (shift-invariant) of each set against the oracle's sparse LU of
    that set's own hierarchy."""
    import torch
    draws = [dict(U=3.0, mu=0.5, kT=0.4, tier=2), dict(U=9.0, mu=1.8, kT=0.9, tier=3),
             dict(U=6.0, mu=2.5, kT=0.3, tier=2)]
    models = [W.siam_model(U=d["U"], mu=d["mu"], kT=d["kT"], tier=3) for d in draws]
    gs = []
    for parity in (1, -1):
        g = heom.build_hierarchy(heom.problem_from_model(models[0], parity))
        heom.set_params_from_models(g, models, parity)
        heom.set_truncation(g, [0, 0, 0], [d["tier"] for d in draws])
        gs.append(g)
    even, odd = gs
    x = torch.zeros((even.n_ado, 4, 4, 3), dtype=torch.complex128, device="cuda")
    st, stats = heom.steady(even, x, tol=1e-10, max_iter=4000, prec=heom.MIXED)
    assert st == heom.OK
    om = np.array([-11.0, -4.5, 0.0, 2.2, 8.0])
    A, st, stats = heom.spectrum(odd, x, models[0].fermion_baths[0][0], om, tol=1e-9,
                                 max_iter=2000, prec=heom.SHIFTED)
    assert st == heom.OK
    X = x.cpu().numpy()
    for s, d in enumerate(draws):
        n = hy.problem_hierarchy(hy.model_to_problem(W.siam_model(tier=d["tier"]))).n_ado
        if n < even.n_ado:
            assert np.abs(X[n:, ..., s]).max() == 0.0  # held at zero beyond the set's tier
        Xo, Ao, Me = _oracle_dos(d, om, iterative=False)
        assert so.steady_residual(Me, X[:n, ..., s]) < 1e-9
        assert np.abs(X[:n, ..., s] - Xo).max() < 1e-8 * np.abs(Xo).max(), s
        assert np.abs(A[s] - Ao).max() < 1e-7 * np.abs(Ao).max(), s


def test_batched_spectra_64_sets_sampled(heom):
    """The batched-spectra workload exactly as benchmarked: 64 SIAM sets (draw seed 7522;
    tiers 2, 3, 4; deepest first) x 4,096 frequencies on [-20, 20], stationary states (mixed
    precision) and
    DOS (shift-invariant) to 1e-8 in one call each. Every residual meets 1e-8; sampled
    (set, frequency) pairs match the oracle -- sparse LU for a tier-2 and a tier-3 set, the
    GMRES path for a tier-4 set (12,951 ADOs), whose LU fills in beyond reach."""
    import torch
    # deepest sets first: each ADO is then kept by a leading run of sets, and the
    # Gram-Schmidt kernels skip the columns held at zero
    draws = sorted(W.draw_siam_sets(64), key=lambda d: -d["tier"])
    models, tiers, even, odd = _c3(heom, draws)
    om = W.omega_grid(4096)
    x = torch.zeros((even.n_ado, 4, 4, 64), dtype=torch.complex128, device="cuda")
    st, sst = heom.steady(even, x, tol=1e-8, max_iter=4000, prec=heom.MIXED)
    assert st == heom.OK and max(s_["residual"] for s_ in sst) <= 1e-8
    A, st, stats = heom.spectrum(odd, x, models[0].fermion_baths[0][0], om, tol=1e-8,
                                 max_iter=2000, prec=heom.SHIFTED)
    assert st == heom.OK and A.shape == (64, 4096)
    assert max(s_["residual"] for s_ in stats) <= 1e-8
    rng = np.random.default_rng(7522)
    for tier in (2, 3, 4):
        s = int(rng.choice([i for i, t in enumerate(tiers) if t == tier]))
        idx = np.sort(rng.choice(4096, 3, replace=False))
        _, Ao, _ = _oracle_dos(draws[s], om[idx], iterative=tier == 4)
        assert np.abs(A[s, idx] - Ao).max() < 1e-7 * max(np.abs(Ao).max(), 1e-3), (tier, s)
