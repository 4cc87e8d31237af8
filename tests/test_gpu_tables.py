"""GPU-library host tables and exponents against the oracle: bit-exact integers, FP64 values."""
import numpy as np
import pytest

import workloads as W
from oracle import exponents as ex
from oracle import hierarchy as hy
from oracle import tables as tb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


@pytest.mark.parametrize("N,fermi,pade", [(2, 1, 1), (6, 1, 1), (10, 0, 1), (3, 1, 0), (4, 0, 0)])
def test_pade_constants_match_oracle(heom, N, fermi, pade):
    k, z = heom.pade_constants(N, bool(fermi), bool(pade))
    ko, zo = ex.decomposition(N, "fermi" if fermi else "bose", "pade" if pade else "matsubara")
    assert np.allclose(k, ko, rtol=1e-12, atol=0) and np.allclose(z, zo, rtol=1e-12, atol=0)


@pytest.mark.parametrize("method", ["pade", "matsubara"])
def test_exponents_match_oracle(heom, method):
    for nu in (1, -1):
        e, g = heom.exp_lorentz_fermion(2.0, 10.0, 1.0, 0.5, 2, method == "pade", nu)
        eo, go = ex.lorentz_fermion_exponents(2.0, 10.0, 1.0, 0.5, 2, method, nu)
        assert np.abs(e - eo).max() < 1e-12 * np.abs(eo).max()
        assert np.abs(g - go).max() < 1e-12 * np.abs(go).max()
    xi, chi = heom.exp_drude_lorentz(0.1, 0.5, 0.5, 2, method == "pade")
    xo, co = ex.drude_lorentz_exponents(0.1, 0.5, 0.5, 2, method)
    assert np.abs(xi - xo).max() < 1e-12 * np.abs(xo).max()
    assert np.abs(chi - co).max() < 1e-12 * np.abs(co).max()


def _compare_tables(heom, prob):
    h = heom.build_hierarchy(prob)
    ho = hy.problem_hierarchy(prob)
    assert h.n_ado == ho.n_ado
    t = heom.export_tables(h)
    ref = tb.neighbour_table(prob, ho)
    assert int(t["row_ptr"][-1]) == sum(len(r) for r in ref)
    for i in range(ho.n_ado):
        a, b = t["row_ptr"][i], t["row_ptr"][i + 1]
        got = sorted(zip(t["nb"][a:b].tolist(), t["k"][a:b].tolist(), t["dir"][a:b].tolist(),
                         t["mult_l"][a:b].tolist(), t["mult_r"][a:b].tolist()))
        assert got == sorted(ref[i]), i
    # dictionary: label <-> index for every ADO
    for i, (m, S) in enumerate(ho.ados):
        occ = list(m) + [1 if q in S else 0 for q in range(ho.K_f)]
        assert heom.ado_index(h, occ) == i
        assert heom.ado_label(h, i).tolist() == occ
    return h


@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("bos,fer,tb_,tf", [
    ([("RI", 3)], [], 4, 0),
    ([], [6, 6, 6, 6], 0, 3),
    ([("RI", 2), ("I", 1), ("R", 1)], [4, 2], 2, 2),
    ([("RI", 1)], [2], 0, 0),
])
def test_tables_bit_exact(heom, parity, bos, fer, tb_, tf):
    prob = W.random_raw_problem(2, bos, fer, tb_, tf, parity=parity, seed=5)
    _compare_tables(heom, prob)


def test_tables_paper_example1_tier2(heom):
    """Example 1 shape (K_f = 56) at tier 2: 1,597 ADOs (Table 3)."""
    prob = W.random_raw_problem(4, [], [14, 14, 14, 14], 0, 2, seed=6)
    h = _compare_tables(heom, prob)
    assert h.n_ado == 1597


def test_outside_index_is_minus_one(heom):
    prob = W.random_raw_problem(2, [("RI", 2)], [4], 2, 2, seed=7)
    h = heom.build_hierarchy(prob)
    assert heom.ado_index(h, [3, 0, 0, 0, 0, 0]) == -1
    assert heom.ado_index(h, [0, 0, 1, 1, 1, 0]) == -1


def test_invalid_inputs_raise(heom):
    prob = W.random_raw_problem(2, [], [4], 0, 2, seed=8)
    prob["baths"][0]["partner"] = np.array([0, 1, 2, 3], np.int32)
    with pytest.raises(heom.HeomError) as e:
        heom.build_hierarchy(prob)
    assert e.value.status == heom.EINVAL
    prob = W.random_raw_problem(2, [], [4], 0, 2, seed=8)
    prob["H"] = prob["H"] * np.nan
    with pytest.raises(heom.HeomError):
        heom.build_hierarchy(prob)
