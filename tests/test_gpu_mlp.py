"""GPU tests of the learned warm start: the network's forward and backward kernels against
the FP64 oracle (with the same bfloat16 operand rounding), training, the feature map, and
the gain over a cold start on held-out stationary solves."""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from oracle import mlp as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_07522_gb300 as m
    return m

# GPU and oracle round the same operands to bfloat16; they differ by FP32 against FP64
# accumulation (<= 256 terms: ~2e-5 relative), tanhf against tanh, and the rare operand that
# sits within that difference of a bfloat16 rounding boundary and rounds the other way
# (one bfloat16 ulp, 2^-8, in one term of a sum). 1e-3 of the norm bounds all of these.
TOL_FWD = 1e-3
TOL_GRAD = 5e-3


def _net(heom, widths, seed):
    rng = np.random.default_rng(seed)
    net = heom.Mlp(widths, seed=seed)
    p = net.get_params().astype(np.float64)
    p += rng.normal(0, 0.05, p.size)  # non-zero biases too
    net.set_params(p)
    norms = (rng.normal(0, 1, widths[0]), rng.uniform(0.5, 2, widths[0]),
             rng.normal(0, 1, widths[-1]), rng.uniform(0.5, 2, widths[-1]))
    net.set_standardisation(*norms)
    # the oracle sees exactly what the GPU holds (FP32 parameters and standardisation)
    return rng, net, net.get_params().astype(np.float64), tuple(np.float32(a).astype(np.float64) for a in norms)


@pytest.mark.parametrize("widths,batch", [([5, 37, 70, 3], 50), ([5, 256, 256, 256, 784], 130)])
def test_forward_matches_oracle(heom, widths, batch):
    import torch
    rng, net, p, norms = _net(heom, widths, 11)
    x = rng.normal(0, 1, (batch, widths[0])).astype(np.float32)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    yo, _ = om.forward(p, widths, x.astype(np.float64), norms, bf16=True)
    assert np.linalg.norm(y - yo) <= TOL_FWD * np.linalg.norm(yo)


@pytest.mark.parametrize("widths,batch", [([5, 37, 70, 3], 50), ([5, 256, 256, 256, 784], 130)])
def test_gradients_match_oracle(heom, widths, batch):
    import torch
    rng, net, p, norms = _net(heom, widths, 12)
    x = rng.normal(0, 1, (batch, widths[0])).astype(np.float32)
    t = rng.normal(0, 1, (batch, widths[-1])).astype(np.float32)
    g, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    lo, go = om.loss_and_grad(p, widths, x.astype(np.float64), t.astype(np.float64), norms, bf16=True)
    assert abs(loss - lo) <= 1e-3 * lo
    w_off, b_off, _ = om.layout(widths)
    for l in range(len(widths) - 1):  # every layer's weights and biases
        for a, b in ((w_off[l], w_off[l] + widths[l] * widths[l + 1]), (b_off[l], b_off[l] + widths[l + 1])):
            assert np.linalg.norm(g[a:b] - go[a:b]) <= TOL_GRAD * np.linalg.norm(go[a:b]), (l, a)


def test_training_fits_a_teacher_network(heom):
    """Adam steps on the library's gradients fit the outputs of a fixed random network."""
    import torch
    rng = np.random.default_rng(21)
    teacher = [5, 16, 4]
    _, _, n = om.layout(teacher)
    tp = rng.normal(0, 0.7, n)
    x = rng.normal(0, 1, (512, 5))
    ident = (np.zeros(5), np.ones(5), np.zeros(4), np.ones(4))
    t, _ = om.forward(tp, teacher, x, ident, bf16=False)
    net = heom.Mlp([5, 64, 64, 4], seed=3)
    net.set_standardisation(np.zeros(5), np.ones(5), t.mean(0), t.std(0))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    first = net.train_step(xd, td, 3e-3, want_loss=True)
    for _ in range(400):
        net.train_step(xd, td, 3e-3)
    last = net.gradients(xd, td)[1]
    assert last < first / 20, (first, last)


def _siam_sets(heom, draws, tier):
    base = W.siam_model(tier=tier)
    h = heom.build_hierarchy(heom.problem_from_model(base, 1))
    Hs, coefs, rates = [], [], []
    for U, eps, G, kT, mu in draws:
        p = heom.problem_from_model(W.siam_model(eps=eps, U=U, Gamma=G, kT=kT, mu=mu, tier=tier))
        Hs.append(p["H"])
        coefs.append(np.concatenate([b["coef"] for b in p["baths"]]))
        rates.append(np.concatenate([b["rate"] for b in p["baths"]]))
    heom.set_params(h, np.array(Hs), np.array(coefs), np.array(rates))
    return h, base


def _tier1(model, tier):
    prob = hy.model_to_problem(model, 1)
    hier = hy.problem_hierarchy(prob)
    return [i for i, (m, S) in enumerate(hier.ados) if sum(m) + len(S) == 1]


def test_features_and_scatter_match_oracle(heom):
    import torch
    draws = W.draw_warmstart_samples(3, seed=5)
    h, base = _siam_sets(heom, draws, 2)
    x = torch.zeros((h.n_ado, 4, 4, 3), dtype=torch.complex128, device="cuda")
    heom.steady(h, x, tol=1e-8, max_iter=3000, prec=heom.FP64)
    tier1 = _tier1(base, 2)
    nf = 16 + 2 * 16 * len(tier1)
    f = heom.warm_start_features(h, x, nf).cpu().numpy()
    X = x.cpu().numpy()
    for b in range(3):
        assert np.array_equal(f[b], om.features(X[..., b], 4, tier1).astype(np.float32))
    # scatter: the ADO vector of a network's prediction
    net = heom.Mlp([5, 32, nf], seed=4)
    pd = torch.from_numpy(draws.astype(np.float32)).cuda()
    y = net.forward(pd).cpu().numpy().astype(np.float64)
    xo = torch.full((h.n_ado, 4, 4, 3), 7.0, dtype=torch.complex128, device="cuda")
    heom.warm_start(h, net, pd, xo)
    Xo = xo.cpu().numpy()
    for b in range(3):
        assert np.array_equal(Xo[..., b], om.from_features(y[b], h.n_ado, 4, tier1))


def test_warm_start_gain_on_held_out_solves(heom):
    """Train on GPU stationary states of sampled SIAM parameters, then on held-out parameters:
    (1) the network's rho_sys is far closer to the solved one than the best answer without
    it (the mean training state), at the cost of one forward pass instead of a solve;
    (2) a solve seeded with the prediction still reaches the 1e-8 residual (the cold solve
    is the fallback and the measure of its error). Iterations are recorded for both starts: a guess made of
    rho_sys and the tier-1 ADOs (higher tiers zero) has a residual larger than ||b||, so
    heom_steady discards it and starts cold; the warm solve costs what the cold one does."""
    import torch
    tier, n_train, n_test = 2, 768, 24
    draws = W.draw_warmstart_samples(n_train + n_test, seed=99)
    h, base = _siam_sets(heom, draws, tier)
    x = torch.zeros((h.n_ado, 4, 4, len(draws)), dtype=torch.complex128, device="cuda")
    heom.steady(h, x, tol=1e-8, max_iter=3000, prec=heom.MIXED)
    tier1 = _tier1(base, tier)
    nf = 16 + 2 * 16 * len(tier1)
    feats = heom.warm_start_features(h, x, nf)
    params = torch.from_numpy(draws.astype(np.float32)).cuda()
    ftr = feats[:n_train].cpu().numpy()
    net = heom.Mlp([5, 256, 256, 256, nf], seed=1)
    net.set_standardisation(draws[:n_train].mean(0), draws[:n_train].std(0),
                            ftr.mean(0), np.maximum(ftr.std(0), 1e-6))
    order = np.random.default_rng(0).permutation(n_train)
    xs, ts = params[:n_train][order].contiguous(), feats[:n_train][order].contiguous()
    for epoch in range(300):
        lr = 2e-3 if epoch < 200 else 4e-4
        for k in range(0, n_train, 256):
            net.train_step(xs[k:k + 256], ts[k:k + 256], lr)
    rho_mean = x[0, :, :, :n_train].mean(dim=-1).cpu().numpy()
    test = draws[n_train:]
    err_net, err_mean, cold, warm = [], [], [], []
    for j in range(n_test):
        hj, _ = _siam_sets(heom, test[j:j + 1], tier)
        xj = torch.zeros((hj.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
        _, s_c = heom.steady(hj, xj, tol=1e-8, max_iter=3000, prec=heom.FP64)
        x0 = torch.zeros((hj.n_ado, 4, 4, 1), dtype=torch.complex128, device="cuda")
        heom.warm_start(hj, net, params[n_train + j:n_train + j + 1].contiguous(), x0)
        rho = xj[0].cpu().numpy()
        err_net.append(np.linalg.norm(x0[0, :, :, 0].cpu().numpy() - rho) / np.linalg.norm(rho))
        err_mean.append(np.linalg.norm(rho_mean - rho) / np.linalg.norm(rho))
        xw = torch.zeros_like(xj)
        _, s_w = heom.steady(hj, xw, x0=x0[..., 0].contiguous(), tol=1e-8, max_iter=3000, prec=heom.FP64)
        assert s_c[0]["status"] == 0 and s_w[0]["status"] == 0
        assert s_w[0]["residual"] <= 1e-8
        cold.append(s_c[0]["iterations"])
        warm.append(s_w[0]["iterations"])
    print(f"held-out rho_sys error: network {np.mean(err_net):.3e}, mean state {np.mean(err_mean):.3e}; "
          f"BiCGStab iterations cold {np.mean(cold):.1f}, warm {np.mean(warm):.1f}")
    assert np.mean(err_net) < 0.05
    assert np.mean(err_net) < 0.25 * np.mean(err_mean)
    assert np.mean(warm) <= np.mean(cold) + 1.0


def test_element_features_round_trip(heom):
    """heom_gather_elements reads the listed elements of every column; heom_warm_start_elements
    writes a network's outputs to the same elements and zero elsewhere (checked against the
    network's own forward pass); an out-of-range element index is refused."""
    import torch
    m = W.siam_model(tier=2)
    g = heom.build_hierarchy(heom.problem_from_model(m, 1))
    X = W.random_ado_vector(g.n_ado, 4, 3, seed=71)
    x = torch.from_numpy(X).cuda()
    elems = torch.tensor([0, 5, 17, 16 * g.n_ado - 1], dtype=torch.int64, device="cuda")
    f = heom.gather_elements(g, x, elems).cpu().numpy()
    flat = X.reshape(-1, 3)
    for k, e in enumerate(elems.cpu().numpy()):
        assert np.array_equal(f[:, 2 * k], flat[e].real.astype(np.float32))
        assert np.array_equal(f[:, 2 * k + 1], flat[e].imag.astype(np.float32))
    net = heom.Mlp([5, 16, 8], seed=3)
    params = torch.randn(3, 5, dtype=torch.float32, device="cuda")
    y = net.forward(params).cpu().numpy()
    x0 = torch.empty((g.n_ado, 4, 4, 3), dtype=torch.complex128, device="cuda")
    heom.warm_start_elements(g, net, params, elems, x0)
    got = x0.cpu().numpy().reshape(-1, 3)
    want = np.zeros_like(got)
    for k, e in enumerate(elems.cpu().numpy()):
        want[e] = y[:, 2 * k] + 1j * y[:, 2 * k + 1]
    assert np.array_equal(got, want)
    bad = torch.tensor([16 * g.n_ado], dtype=torch.int64, device="cuda")
    with pytest.raises(heom.HeomError):
        heom.gather_elements(g, x, bad)
