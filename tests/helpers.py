"""Shared helpers of the GPU parity tests (layout conversion, problem construction)."""
import numpy as np

import workloads as W
from oracle import hierarchy as hy
from oracle import liouvillian as lv


def to_dev(X, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(X)).to(device="cuda", dtype=dtype)


def oracle_apply_batched(prob, h, X):
    """M X for X of shape (N, d, d, B) through the oracle's sparse matrix (column stacking)."""
    M = lv.build_matrix(prob, h)
    N, d = X.shape[0], X.shape[1]
    B = X.shape[3]
    V = np.swapaxes(X, 1, 2).reshape(N * d * d, B)  # vec(rho_n) column stacking per column
    Y = M @ V
    return np.swapaxes(Y.reshape(N, d, d, B), 1, 2)


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def model_problem_oracle(model, parity=1):
    return hy.model_to_problem(model, parity)


CONFIG_MODELS = {
    "spin_boson_t4": lambda: W.spin_boson_model(tier=4),
    "siam_t2": lambda: W.siam_model(tier=2),
    "siam_t3": lambda: W.siam_model(tier=3),
    "charge_cavity_small": lambda: W.charge_cavity_model(n_fock=3, tier_b=2, tier_f=1),
}
