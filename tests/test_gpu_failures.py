"""Failure detection of the solvers, made on the host side (nothing faults, traps or hangs the
GPU): an iteration limit too small to converge returns HEOM_ENOCONV with the per-column
statistics filled instead of looping on, and invalid arguments are refused with HEOM_EINVAL
before any work is enqueued."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


@pytest.fixture(scope="module")
def siam(heom):
    m = W.siam_model(tier=2)
    return m, heom.build_hierarchy(heom.problem_from_model(m, 1)), \
        heom.build_hierarchy(heom.problem_from_model(m, -1))


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_steady_iteration_limit_returns_enoconv(heom, siam, prec):
    import torch
    m, even, _ = siam
    x = torch.zeros((even.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
    st, stats = heom.steady(even, x, tol=1e-12, max_iter=1, prec=getattr(heom, prec),
                            raise_on_error=False)
    assert st == heom.ENOCONV
    assert stats[0]["status"] == heom.ENOCONV and np.isfinite(stats[0]["residual"])
    assert stats[0]["residual"] > 1e-12
    # the same hierarchy still solves afterwards
    st, stats = heom.steady(even, x, tol=1e-10, max_iter=3000, prec=getattr(heom, prec))
    assert st == heom.OK and stats[0]["residual"] <= 1e-10


def test_spectrum_iteration_limit_returns_enoconv(heom, siam):
    import torch
    m, even, odd = siam
    x = torch.zeros((even.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
    heom.steady(even, x, tol=1e-10, prec=heom.FP64)
    om = np.array([-5.0, 0.0, 5.0])
    A, st, stats = heom.spectrum(odd, x, m.fermion_baths[0][0], om, tol=1e-12, max_iter=3,
                                 prec=heom.SHIFTED, raise_on_error=False)
    assert st == heom.ENOCONV
    assert all(s_["status"] == heom.ENOCONV for s_ in stats)
    assert all(np.isfinite(s_["residual"]) and s_["residual"] > 1e-12 for s_ in stats)


def test_solvers_refuse_invalid_arguments(heom, siam):
    import torch
    m, even, odd = siam
    x = torch.zeros((even.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
    st, _ = heom.steady(even, x, tol=0.0, prec=heom.FP64, raise_on_error=False)
    assert st == heom.EINVAL
    st, _ = heom.steady(odd, torch.zeros((odd.n_ado, 4, 4), dtype=torch.complex128, device="cuda"),
                        tol=1e-8, prec=heom.FP64, raise_on_error=False)
    assert st == heom.EINVAL  # the stationary state lives in the even sector
    _, st, _ = heom.spectrum(odd, x, m.fermion_baths[0][0], np.array([]), tol=1e-8,
                             prec=heom.SHIFTED, raise_on_error=False)
    assert st == heom.EINVAL
    _, st, _ = heom.psd(odd, x, m.fermion_baths[0][0], np.array([1.0]), raise_on_error=False)
    assert st == heom.EINVAL  # the PSD needs the even sector


def test_device_wait_timeout_returns_etimeout(heom, siam):
    """The persistent solvers' grid barriers are the library's only device-side waits. With
    the wait bound set to 300 SM cycles, ordinary skew between CTAs makes a wait run out: the
    CTA raises the shared flag, every CTA leaves the launch, and the call returns
    HEOM_ETIMEOUT with its statistics filled. Nothing hangs or faults. With the default bound
    restored the same hierarchies solve normally."""
    import torch
    m, even, odd = siam
    x = torch.zeros((even.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
    try:
        heom.set_wait_limit(300)
        st, stats = heom.steady(even, x, tol=1e-10, prec=heom.FP64, raise_on_error=False)
        assert st == heom.ETIMEOUT
        # the solve stopped at its first barrier: x is still zero, r_ss = ||M x|| / ||x|| has
        # no value and is reported as +inf
        assert stats[0]["status"] == heom.ETIMEOUT and stats[0]["residual"] > 1e-10
        A, st, stats = heom.spectrum(odd, x, m.fermion_baths[0][0], np.array([-5.0, 5.0]),
                                     tol=1e-8, prec=heom.SHIFTED, raise_on_error=False)
        assert st == heom.ETIMEOUT and all(s_["status"] == heom.ETIMEOUT for s_ in stats)
        assert np.all(np.isnan(A))
    finally:
        heom.set_wait_limit(0)
    st, stats = heom.steady(even, x, tol=1e-10, prec=heom.FP64)
    assert st == heom.OK and stats[0]["residual"] <= 1e-10
    A, st, stats = heom.spectrum(odd, x, m.fermion_baths[0][0], np.array([-5.0, 5.0]), tol=1e-8,
                                 prec=heom.SHIFTED)
    assert st == heom.OK and np.all(np.isfinite(A))


def test_entry_points_restore_the_callers_device(heom, siam):
    """Every entry point makes the hierarchy's device current for its work and gives the
    calling thread its previous current device back (checked on one GPU: the current device
    is still the caller's after apply, evolve, steady and spectrum)."""
    import torch
    m, even, odd = siam
    dev = torch.cuda.current_device()
    x = torch.zeros((even.n_ado, 4, 4), dtype=torch.complex128, device="cuda")
    heom.steady(even, x, tol=1e-8, prec=heom.FP64)
    y = torch.empty_like(x)
    heom.apply(even, x, y)
    heom.evolve(even, y, 0.01, 2)
    heom.spectrum(odd, x, m.fermion_baths[0][0], np.array([0.0]), tol=1e-8, prec=heom.SHIFTED)
    assert torch.cuda.current_device() == dev
