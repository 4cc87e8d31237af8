"""Out-of-bounds guard for the device entry points (compute-sanitizer is closed on this machine).

Every device input sits in front of a NaN-filled tail and every output in front of a canary
tail, at ragged batch sizes that exercise the kernels' column and row tails (per-element and
tiled apply, RK4 stages, the persistent stationary solve, the shift-invariant spectrum and its
final solve). A read past the end would turn a result into NaN or change it; a write past the
end would change a canary. The results must equal those of clean buffers bit for bit.
"""
import numpy as np
import pytest

import workloads as W
from oracle import hierarchy as hy
from tests.helpers import to_dev

pytestmark = pytest.mark.gpu

PAD = 4096
CANARY = complex(7.0, -7.0)


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


def _guarded(shape, dtype, fill):
    import torch
    n = int(np.prod(shape))
    base = torch.full((n + PAD,), fill, dtype=dtype, device="cuda")
    return base, base[:n].view(shape)


def _tail_is(base, n, value):
    import torch
    return bool(torch.all(base[n:] == torch.tensor(value, dtype=base.dtype, device=base.device)))


def _tail_is_nan(base, n):
    import torch
    return bool(torch.all(torch.isnan(torch.view_as_real(base[n:]))))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("batch", [1, 3, 17, 37, 67])
def test_apply_reads_and_writes_in_bounds(heom, prec, batch):
    import torch
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    prob = W.random_raw_problem(3, [("RI", 2), ("I", 1)], [4, 2], 2, 2, seed=81)
    h = hy.problem_hierarchy(prob)
    shape = (h.n_ado, 3, 3) if batch == 1 else (h.n_ado, 3, 3, batch)
    X = W.random_ado_vector(h.n_ado, 3, None if batch == 1 else batch, seed=82)
    g = heom.build_hierarchy(prob)
    x0 = to_dev(X, dt)
    y0 = torch.empty_like(x0)
    heom.apply(g, x0, y0)
    xb, x = _guarded(shape, dt, complex("nan+nanj"))
    x.copy_(x0)
    yb, y = _guarded(shape, dt, CANARY)
    heom.apply(g, x, y)
    torch.cuda.synchronize()
    n = x.numel()
    assert torch.equal(y, y0)
    assert _tail_is(yb, n, CANARY) and _tail_is_nan(xb, n)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("batch", [1, 33])
def test_evolve_reads_and_writes_in_bounds(heom, prec, batch):
    import torch
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    m = W.spin_boson_model(tier=3)
    g = heom.build_hierarchy(heom.problem_from_model(m))
    X = np.zeros((g.n_ado, 2, 2), complex)
    X[0] = m.rho0
    if batch > 1:
        X = np.repeat(X[..., None], batch, axis=-1)
    x0 = to_dev(X, dt)
    t0 = heom.evolve(g, x0, 0.01, 50, 10)
    xb, x = _guarded(x0.shape, dt, complex("nan+nanj"))
    x.copy_(to_dev(X, dt))
    t1 = heom.evolve(g, x, 0.01, 50, 10)
    torch.cuda.synchronize()
    assert torch.equal(x, x0) and torch.equal(t1, t0)
    assert _tail_is_nan(xb, x.numel())


def test_steady_and_spectrum_read_and_write_in_bounds(heom):
    import torch
    m = W.siam_model(tier=2)
    even = heom.build_hierarchy(heom.problem_from_model(m, 1))
    odd = heom.build_hierarchy(heom.problem_from_model(m, -1))
    shape = (even.n_ado, 4, 4)
    x0 = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    heom.steady(even, x0, tol=1e-10, prec=heom.FP64)
    xb, x = _guarded(shape, torch.complex128, CANARY)
    x.zero_()
    heom.steady(even, x, tol=1e-10, prec=heom.FP64)
    torch.cuda.synchronize()
    assert torch.equal(x, x0) and _tail_is(xb, x.numel(), CANARY)
    om = np.array([-9.0, -2.5, 0.3, 6.0])
    dop = m.fermion_baths[0][0]
    A0, _, _ = heom.spectrum(odd, x0, dop, om, tol=1e-10, max_iter=2000, prec=heom.SHIFTED)
    sb, ss = _guarded(shape, torch.complex128, complex("nan+nanj"))
    ss.copy_(x0)
    A1, st, _ = heom.spectrum(odd, ss, dop, om, tol=1e-10, max_iter=2000, prec=heom.SHIFTED)
    assert st == heom.OK and np.array_equal(A0, A1)
