"""Parity of the CUDA apply y = M x with the oracle (Eq. HEOM), element by element.

Tolerances: FP64 1e-10 relative to max|y| (the benchmark spec's bound for the plain path);
FP32 1e-5 relative: each output element sums O(K) products of unit-roundoff 6e-8 terms.
"""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv
from tests.helpers import oracle_apply_batched, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


def _run(heom, prob, X, prec):
    import torch
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    h = heom.build_hierarchy(prob)
    x = to_dev(X, dt)
    y = torch.empty_like(x)
    heom.apply(h, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("batch", [1, 3, 37, 64])
@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("bos,fer,tb_,tf", [
    ([("RI", 2), ("R", 1), ("I", 1)], [], 3, 0),
    ([], [4, 2], 0, 3),
    ([("RI", 2), ("I", 1)], [4, 2], 2, 2),
])
def test_apply_random_problems(heom, prec, batch, parity, bos, fer, tb_, tf):
    prob = W.random_raw_problem(3, bos, fer, tb_, tf, parity=parity, seed=31)
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, batch, seed=32)
    Y = oracle_apply_batched(prob, h, X)
    Xg = X if batch > 1 else X[..., 0]
    Yg = _run(heom, prob, Xg, prec)
    if batch == 1:
        Yg = Yg[..., None]
    assert rel_err(Yg, Y) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,model", [
    ("spin_boson_t4", lambda: W.spin_boson_model(tier=4)),
    ("siam_t2", lambda: W.siam_model(tier=2)),
    ("charge_cavity_d6", lambda: W.charge_cavity_model(n_fock=3, tier_b=2, tier_f=1)),
])
def test_apply_workload_models_own_exponents(heom, prec, name, model):
    """Each side generates its own exponents from the physical parameters."""
    m = model()
    prob_o = hy.model_to_problem(m)
    prob_g = heom.problem_from_model(m)
    h = hy.problem_hierarchy(prob_o)
    X = W.random_ado_vector(h.n_ado, m.d, seed=33)
    Y = lv.apply_loop(prob_o, X, h)
    Yg = _run(heom, prob_g, X, prec)
    assert rel_err(Yg, Y) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_charge_cavity_d24(heom, prec):
    """Charge-cavity at d = 24 (dense coupling operators), 790 ADOs; sampled ADOs."""
    m = W.charge_cavity_model()
    prob_o = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob_o)
    assert h.n_ado == 790
    X = W.random_ado_vector(h.n_ado, 24, seed=34)
    rng = np.random.default_rng(1)
    only = sorted(set([0, 1, h.n_ado - 1] + rng.choice(h.n_ado, 60, replace=False).tolist()))
    Y = lv.apply_loop(prob_o, X, h, only=only)
    Yg = _run(heom, heom.problem_from_model(m), X, prec)
    assert rel_err(Yg[only], Y[only]) < TOL[prec]


def test_apply_parameter_sets(heom):
    """Three parameter sets on one structure; columns 2s, 2s+1 use set s."""
    import torch
    prob = W.random_raw_problem(3, [("RI", 2)], [4], 2, 2, seed=35)
    h = hy.problem_hierarchy(prob)
    rng = np.random.default_rng(36)
    K = 2 + 4
    Hs, coefs, rates, probs = [], [], [], []
    for s in range(3):
        p = dict(prob)
        p["H"] = W.random_hermitian(3, rng)
        baths = []
        for b in prob["baths"]:
            nb = dict(b)
            nb["coef"] = W.random_complex(len(b["coef"]), rng) * 0.3
            nb["rate"] = rng.uniform(0.2, 2, len(b["coef"])) + 0.1j
            baths.append(nb)
        p["baths"] = baths
        probs.append(p)
        Hs.append(p["H"])
        coefs.append(np.concatenate([b["coef"] for b in baths]))
        rates.append(np.concatenate([b["rate"] for b in baths]))
    g = heom.build_hierarchy(prob)
    heom.set_params(g, np.array(Hs), np.array(coefs), np.array(rates))
    assert g.n_sets == 3
    X = W.random_ado_vector(h.n_ado, 3, 6, seed=37)
    x = to_dev(X, torch.complex128)
    y = torch.empty_like(x)
    heom.apply(g, x, y)
    Yg = y.cpu().numpy()
    for s in range(3):
        Y = oracle_apply_batched(probs[s], h, X[..., 2 * s:2 * s + 2])
        assert rel_err(Yg[..., 2 * s:2 * s + 2], Y) < 1e-10


def test_apply_edge_cases(heom):
    import torch
    # tier 0: a single ADO, pure system commutator minus nothing
    prob = W.random_raw_problem(3, [("RI", 2)], [4], 0, 0, seed=38)
    X = W.random_ado_vector(1, 3, seed=39)
    H = prob["H"]
    assert rel_err(_run(heom, prob, X, "fp64"), -1j * (H @ X - X @ H)) < 1e-12
    # no baths at all
    prob = dict(d=2, H=W.SX * 0.5, baths=[], tier_b=0, tier_f=0, parity=1)
    X = W.random_ado_vector(1, 2, seed=40)
    assert rel_err(_run(heom, prob, X, "fp64"), -1j * (prob["H"] @ X - X @ prob["H"])) < 1e-12
    # bad arguments are refused
    prob = W.random_raw_problem(2, [("RI", 1)], [], 1, 0, seed=41)
    g = heom.build_hierarchy(prob)
    x = torch.zeros((g.n_ado, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(heom.HeomError):
        heom.apply(g, x, x)  # in place (overlap) is refused


def test_apply_full_size_siam_batched_sampled(heom):
    """SIAM tier 3 (2,325 ADOs) x 2,000 columns in FP32 -- the batched-spectrum launch shape;
    sampled ADOs and columns against the oracle's per-ADO formula."""
    import torch
    m = W.siam_model(tier=3)
    prob_o = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob_o)
    B = 2000
    rng = np.random.default_rng(42)
    x = (torch.randn(h.n_ado, 4, 4, B, dtype=torch.complex64, device="cuda"))
    y = torch.empty_like(x)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    heom.apply(g, x, y)
    torch.cuda.synchronize()
    cols = [0, 1, 31, 32, 1999] + rng.choice(B, 5, replace=False).tolist()
    only = sorted(set([0, 1, 24, 300, h.n_ado - 1] + rng.choice(h.n_ado, 40, replace=False).tolist()))
    Xc = x[..., cols].cpu().numpy().astype(np.complex128)
    Yc = y[..., cols].cpu().numpy().astype(np.complex128)
    for j in range(len(cols)):
        Y = lv.apply_loop(prob_o, Xc[..., j], h, only=only)
        assert rel_err(Yc[only, ..., j], Y[only]) < TOL["fp32"]


def test_apply_paper_scale_example1_sampled(heom):
    """Paper Example 1 shape (K_f = 56, n_max = 4: 396,607 ADOs, Table 3), batch 1, FP64."""
    import torch
    m = W.siam_model(tier=4, Gamma=1.0, n_poles=6)
    prob_o = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob_o)
    assert h.n_ado == 396607
    x = torch.randn(h.n_ado, 4, 4, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    heom.apply(g, x, y)
    torch.cuda.synchronize()
    rng = np.random.default_rng(43)
    only = sorted(set([0, 1, 57, 1597, 29317, h.n_ado - 1] +
                      rng.choice(h.n_ado, 50, replace=False).tolist()))
    X = x.cpu().numpy()
    Y = lv.apply_loop(prob_o, X, h, only=only)
    assert rel_err(y.cpu().numpy()[only], Y[only]) < TOL["fp64"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autotune_choice_keeps_parity(heom, prec):
    """The autotuner times the per-element and the tiled kernel (1..5 ADO ranges per SM) for
    64 columns and keeps the fastest; the apply under the chosen configuration still matches
    the oracle, and a batch too narrow for the tiled kernel tunes to the per-element one."""
    import torch
    m = W.siam_model(tier=2)
    prob = hy.model_to_problem(m)
    h = hy.problem_hierarchy(prob)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    P = heom.FP32 if prec == "fp32" else heom.FP64
    res = heom.autotune(g, 64, P)
    cand = res["candidates_us"]
    valid = [c for c in cand if c > 0]
    assert cand[0] > 0 and len(valid) >= 2
    assert res["best_us"] == min(valid)
    assert res["tiled"] == (res["ctas_per_sm"] > 0)
    X = W.random_ado_vector(h.n_ado, 4, 64, seed=41)
    Y = oracle_apply_batched(prob, h, X)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    Yg = heom.apply(g, to_dev(X, dt), torch.empty_like(to_dev(X, dt))).cpu().numpy()
    assert rel_err(Yg, Y) < TOL[prec]
    narrow = heom.autotune(g, 8, P)
    assert not narrow["tiled"] and all(c < 0 for c in narrow["candidates_us"][1:])


@pytest.mark.parametrize("variant", range(6))
@pytest.mark.parametrize("batch", [18, 130, 132, 256])
def test_apply_tile_variants(heom, variant, batch):
    """Every FP32 variant of the tiled kernel (columns per lane, terms in flight) at batches
    with a ragged last chunk: 18 (one float4 per lane, lanes 9..31 idle), 130 and 132 (the
    second 128-column chunk holds 2 or 4 columns), 256 (full chunks); FP64 beside it."""
    import torch
    prob = W.random_raw_problem(3, [("RI", 2), ("I", 1)], [4, 2], 2, 2, parity=-1, seed=44)
    h = hy.problem_hierarchy(prob)
    X = W.random_ado_vector(h.n_ado, 3, batch, seed=45)
    Y = oracle_apply_batched(prob, h, X)
    g = heom.build_hierarchy(prob)
    heom.set_tile_config(g, 1 + variant % 5, variant)
    for dt, prec in ((torch.complex64, "fp32"), (torch.complex128, "fp64")):
        x = to_dev(X, dt)
        y = torch.empty_like(x)
        heom.apply(g, x, y)
        torch.cuda.synchronize()
        assert rel_err(y.cpu().numpy().astype(np.complex128), Y) < TOL[prec], (variant, batch, prec)
    with pytest.raises(heom.HeomError):
        heom.set_tile_config(g, 0, variant)
    with pytest.raises(heom.HeomError):
        heom.set_tile_config(g, 2, 6)
