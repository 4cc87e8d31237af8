"""Importance-pruned hierarchies (Eq. importance) on the GPU path against the oracle.

Tables and dictionary bit-exact; apply FP64 <= 1e-10 / FP32 <= 1e-5 relative to max|y|; the
stationary state of a pruned Example 1 hierarchy against the oracle's sparse LU (residual
1e-10, tier-0 block 1e-7, current 1e-7 relative).
"""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from oracle import solvers as so
from oracle import tables as tb
from tests.helpers import oracle_apply_batched, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


def _half_pruned(parity, seed=61):
    """A hybrid random problem pruned at the median importance of its prunable ADOs."""
    prob = W.random_raw_problem(3, [("RI", 2), ("I", 1)], [4, 2], 3, 3, parity=parity, seed=seed)
    full = hy.problem_hierarchy(prob)
    bos, fer = hy.flatten_exponents(prob)
    be = [(e.coef, e.rate) for e in bos]
    fe = [(e.coef, e.rate) for e in fer]
    imp = sorted(hy.importance(be, fe, m, S) for (m, S) in full.ados if not hy.always_kept(m, S))
    return dict(prob, importance_th=imp[len(imp) // 2]), full


@pytest.mark.parametrize("parity", [1, -1])
def test_pruned_tables_and_dictionary_bit_exact(heom, parity):
    prob, full = _half_pruned(parity)
    ho = hy.problem_hierarchy(prob)
    h = heom.build_hierarchy(prob)
    assert h.n_ado == ho.n_ado < full.n_ado
    t = heom.export_tables(h)
    ref = tb.neighbour_table(prob, ho)
    assert int(t["row_ptr"][-1]) == sum(len(r) for r in ref)
    for i in range(ho.n_ado):
        a, b = t["row_ptr"][i], t["row_ptr"][i + 1]
        got = list(zip(t["nb"][a:b].tolist(), t["k"][a:b].tolist(), t["dir"][a:b].tolist(),
                       t["mult_l"][a:b].tolist(), t["mult_r"][a:b].tolist()))
        assert sorted(got) == sorted(ref[i]), i
    for i, (m, S) in enumerate(ho.ados):
        occ = list(m) + [1 if q in S else 0 for q in range(ho.K_f)]
        assert heom.ado_index(h, occ) == i
        assert heom.ado_label(h, i).tolist() == occ
    dropped = [a for a in full.ados if a not in ho.index]
    assert dropped
    for (m, S) in dropped[:50]:
        assert heom.ado_index(h, list(m) + [1 if q in S else 0 for q in range(ho.K_f)]) == -1
    assert heom.count_ados(prob["baths"], prob["tier_b"], prob["tier_f"],
                           prob["importance_th"]) == ho.n_ado


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("batch", [1, 64])
@pytest.mark.parametrize("parity", [1, -1])
def test_pruned_apply_matches_oracle(heom, prec, batch, parity):
    import torch
    prob, _ = _half_pruned(parity)
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, batch, seed=62)
    Y = oracle_apply_batched(prob, h, X)
    g = heom.build_hierarchy(prob)
    x = to_dev(X if batch > 1 else X[..., 0], torch.complex128 if prec == "fp64" else torch.complex64)
    y = torch.empty_like(x)
    heom.apply(g, x, y)
    Yg = y.cpu().numpy().astype(np.complex128)
    if batch == 1:
        Yg = Yg[..., None]
    assert rel_err(Yg, Y) < (1e-10 if prec == "fp64" else 1e-5)


def _example1(heom, n_max, th, bias=4.0):
    """Example 1 with the oracle's exponents and with the library's own."""
    m = W.siam_model(eps=-5.0, U=10.0, Gamma=1.0, W=10.0, kT=0.5, mu=bias / 2, n_poles=6,
                     tier=n_max)
    return (dict(hy.model_to_problem(m), importance_th=th),
            dict(heom.problem_from_model(m), importance_th=th))


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_pruned_example1_steady_state_and_current(heom, prec):
    """Example 1 (K_f = 56) at n_max = 2, I_th = 1e-4: 873 ADOs (Table 3)."""
    import torch
    prob, prob_g = _example1(heom, 2, 1e-4)
    h = hy.problem_hierarchy(prob)
    assert h.n_ado == 873
    M = lv.build_matrix(prob, h)
    Xo = so.steady_state(M, 4)
    g = heom.build_hierarchy(prob_g)
    assert g.n_ado == 873
    x = torch.zeros((h.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
    st, stats = heom.steady(g, x, tol=1e-10, max_iter=3000, prec=getattr(heom, prec))
    X = x.cpu().numpy()
    assert st == heom.OK and stats[0]["residual"] <= 1e-10
    assert so.steady_residual(M, X) <= 1.5e-10
    assert rel_err(X[0], Xo[0]) < 1e-7
    lead_l = [0, 1]  # baths [L up, L down, R up, R down]
    I_o = so.current(prob, h, Xo, lead_l)
    I_g = heom.current(g, x, lead_l)[0]
    assert abs(I_g - I_o) < 1e-7 * abs(I_o)


def test_example1_current_converges_with_threshold(heom):
    """Fig. importance_converge at n_max = 4: at equilibrium the current vanishes at every
    threshold; under bias (e Phi = 4) the deviation from the unpruned 396,607-ADO current
    shrinks as I_th falls and is below 1 % at I_th = 1e-7 (49,713 ADOs), where the paper
    calls the current converged."""
    import torch

    def solve(bias, th):
        g = heom.build_hierarchy(_example1(heom, 4, th, bias)[1])
        x = torch.zeros((g.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
        st, stats = heom.steady(g, x, tol=1e-10, max_iter=20000, prec=heom.MIXED)
        assert st == heom.OK
        IL, IR = heom.current(g, x, [0, 1])[0], heom.current(g, x, [2, 3])[0]
        assert abs(IL + IR) < 1e-9 * max(abs(IL), 1e-3)
        return g.n_ado, IL

    ths = [1e-5, 1e-6, 1e-7, 0.0]
    for th in ths:
        assert abs(solve(0.0, th)[1]) < 1e-10
    res = [solve(4.0, th) for th in ths]
    assert [n for n, _ in res] == [5011, 18901, 49713, 396607]
    ref = res[-1][1]
    dev = [abs(I - ref) / abs(ref) for _, I in res[:-1]]
    assert dev[0] > dev[1] > dev[2] and dev[2] < 0.01
