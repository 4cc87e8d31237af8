"""Oracle of the learned warm start (FP64, NumPy) -- test infrastructure only.

The paper has no learned component; this module is the plain definition of the network the
library trains to predict stationary states, so that the GPU forward and backward passes can
be checked against it:

* Layers l = 0 .. L-1: z_l = a_l W_l + b_l, a_{l+1} = tanh(z_l) for hidden layers, the output
  y = z_{L-1} linear; a_0 = (x - in_mean) / in_sd.
* Loss = mean over batch rows and outputs of (y - (t - out_mean) / out_sd)^2.
* Back-propagation by the chain rule: g_{L-1} = 2 (y - t_std) / (M n_out);
  dW_l = a_l^T g_l, db_l = sum over rows of g_l, g_{l-1} = (g_l W_l^T) (1 - a_l^2).
* Flat parameter layout: per layer W_l ([in][out], row-major) then b_l.
* With ``bf16=True`` both operands of every matrix product are first rounded to bfloat16
  (round to nearest, ties to even), as the GPU's tensor-core products do; everything else
  stays FP64.

The warm-start feature map (``features`` / ``from_features``) is the plain statement of which
numbers the network predicts: rho_sys as its d diagonal reals then Re, Im of rho[i][j] for
i < j (row-major), then the tier-1 ADOs' elements, Re and Im interleaved.

Pins (tests/test_oracle_mlp.py): gradients against central finite differences, bfloat16
rounding against torch's conversion and hand-worked ties, the feature map round trip.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    bits = x.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = ((bits + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return bits.view(np.float32).astype(np.float64)


def layout(widths):
    """Offsets (w_off, b_off) of each layer in the flat parameter array, and its length."""
    w_off, b_off, off = [], [], 0
    for l in range(len(widths) - 1):
        w_off.append(off)
        off += widths[l] * widths[l + 1]
        b_off.append(off)
        off += widths[l + 1]
    return w_off, b_off, off


def unpack(params, widths):
    w_off, b_off, _ = layout(widths)
    Ws, bs = [], []
    for l in range(len(widths) - 1):
        Ws.append(np.asarray(params[w_off[l]:w_off[l] + widths[l] * widths[l + 1]],
                             np.float64).reshape(widths[l], widths[l + 1]))
        bs.append(np.asarray(params[b_off[l]:b_off[l] + widths[l + 1]], np.float64))
    return Ws, bs


def _mm(a, b, bf16):
    if bf16:
        return bf16_round(a) @ bf16_round(b)
    return a @ b


def forward(params, widths, x, norms, bf16=True):
    """Raw outputs y [M][n_out] and the activations [a_0 .. a_L] (a_L standardised output)."""
    in_mean, in_sd, out_mean, out_sd = (np.asarray(v, np.float64) for v in norms)
    Ws, bs = unpack(params, widths)
    a = [(np.asarray(x, np.float64) - in_mean) / in_sd]
    L = len(Ws)
    for l in range(L):
        z = _mm(a[l], Ws[l], bf16) + bs[l]
        a.append(np.tanh(z) if l + 1 < L else z)
    return a[-1] * out_sd + out_mean, a


def loss_and_grad(params, widths, x, t, norms, bf16=True):
    """Loss and its gradient with respect to the flat parameters."""
    _, _, out_mean, out_sd = (np.asarray(v, np.float64) for v in norms)
    _, a = forward(params, widths, x, norms, bf16)
    Ws, _ = unpack(params, widths)
    L = len(Ws)
    tn = (np.asarray(t, np.float64) - out_mean) / out_sd
    y = a[L]
    M, n_out = y.shape
    loss = float(np.mean((y - tn) ** 2))
    g = 2.0 * (y - tn) / (M * n_out)
    w_off, b_off, n = layout(widths)
    grad = np.zeros(n)
    for l in range(L - 1, -1, -1):
        dW = _mm(a[l].T, g, bf16)
        grad[w_off[l]:w_off[l] + dW.size] = dW.ravel()
        grad[b_off[l]:b_off[l] + widths[l + 1]] = g.sum(axis=0)
        if l > 0:
            g = _mm(g, Ws[l].T, bf16) * (1.0 - a[l] ** 2)
    return loss, grad


def features(X, d: int, tier1) -> np.ndarray:
    """Warm-start features of one ADO vector X [N][d][d]."""
    rho = X[0]
    f = [rho[i, i].real for i in range(d)]
    for i in range(d):
        for j in range(i + 1, d):
            f += [rho[i, j].real, rho[i, j].imag]
    for n in tier1:
        for e in X[n].ravel():
            f += [e.real, e.imag]
    return np.array(f)


def from_features(f, n_ado: int, d: int, tier1) -> np.ndarray:
    """The ADO vector (zeros outside rho_sys and the tier-1 ADOs) that features f describe."""
    X = np.zeros((n_ado, d, d), complex)
    k = d
    for i in range(d):
        X[0, i, i] = f[i]
    for i in range(d):
        for j in range(i + 1, d):
            X[0, i, j] = f[k] + 1j * f[k + 1]
            X[0, j, i] = f[k] - 1j * f[k + 1]
            k += 2
    for n in tier1:
        vals = np.asarray(f[k:k + 2 * d * d])
        X[n] = (vals[0::2] + 1j * vals[1::2]).reshape(d, d)
        k += 2 * d * d
    return X
