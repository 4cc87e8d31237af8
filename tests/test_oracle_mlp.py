"""Pins of the learned-warm-start oracle (oracle/mlp.py) -- CPU only.

Each pin checks the oracle against something other than itself: back-propagation against
central finite differences of the loss, bfloat16 rounding against hand-worked ties and
torch's float32 -> bfloat16 conversion, the feature map against its inverse and against the
Hermitian structure of rho_sys, and the standardisation against the formula written out.
"""
import numpy as np
import pytest

from oracle import mlp as om


def _rand_net(widths, seed):
    rng = np.random.default_rng(seed)
    _, _, n = om.layout(widths)
    params = rng.normal(0, 0.5, n)
    norms = (rng.normal(0, 1, widths[0]), rng.uniform(0.5, 2, widths[0]),
             rng.normal(0, 1, widths[-1]), rng.uniform(0.5, 2, widths[-1]))
    return rng, params, norms


def test_gradient_matches_central_differences():
    widths = [3, 5, 4, 2]
    rng, params, norms = _rand_net(widths, 1)
    x = rng.normal(0, 1, (7, 3))
    t = rng.normal(0, 1, (7, 2))
    loss, g = om.loss_and_grad(params, widths, x, t, norms, bf16=False)
    h = 1e-6
    fd = np.empty_like(params)
    for i in range(params.size):
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd[i] = (om.loss_and_grad(p1, widths, x, t, norms, bf16=False)[0]
                 - om.loss_and_grad(p2, widths, x, t, norms, bf16=False)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)
    assert loss > 0


def test_bf16_round_ties_and_torch():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to the even mantissa (1)
    assert om.bf16_round(1 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert om.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6
    assert om.bf16_round(-1.5) == -1.5
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    v = rng.normal(0, 10, 10000) * np.exp(rng.normal(0, 5, 10000))
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(om.bf16_round(v), ref)


def test_single_linear_layer_is_the_standardised_affine_map():
    widths = [4, 3]
    rng, params, norms = _rand_net(widths, 5)
    x = rng.normal(0, 1, (6, 4))
    y, _ = om.forward(params, widths, x, norms, bf16=False)
    W = params[:12].reshape(4, 3)
    b = params[12:]
    ref = (((x - norms[0]) / norms[1]) @ W + b) * norms[3] + norms[2]
    assert np.allclose(y, ref, rtol=1e-14, atol=1e-14)


def test_feature_map_round_trip_and_hermitian_rho():
    rng = np.random.default_rng(7)
    d, n_ado, tier1 = 3, 9, [1, 2, 5]
    X = rng.normal(size=(n_ado, d, d)) + 1j * rng.normal(size=(n_ado, d, d))
    X[0] = 0.5 * (X[0] + X[0].conj().T)
    f = om.features(X, d, tier1)
    assert f.size == d * d + 2 * len(tier1) * d * d
    Y = om.from_features(f, n_ado, d, tier1)
    assert np.allclose(Y[0], X[0])
    assert np.allclose(Y[tier1], X[tier1])
    others = [n for n in range(1, n_ado) if n not in tier1]
    assert not Y[others].any()
    assert np.allclose(Y[0], Y[0].conj().T)
