"""The binding refuses ADO vectors and trajectory buffers the library would index out of
bounds, before any call reaches the device. Runs without a GPU: the checks on shape, dtype,
size and contiguity come before the check that the tensor lives on a CUDA device."""
from types import SimpleNamespace

import pytest
import torch

import paper_2306_07522_gb300 as heom

H = SimpleNamespace(n_ado=7, d=3, device=None, n_sets=1)


@pytest.mark.parametrize("shape,why", [
    ((7, 3), "shape must be"),
    ((7, 3, 3, 2, 1), "shape must be"),
    ((6, 3, 3), "does not match"),
    ((7, 2, 3), "does not match"),
    ((7, 3, 2, 4), "does not match"),
    ((7, 3, 3, 0), "batch must be"),
])
def test_batch_of_refuses_wrong_shapes(shape, why):
    with pytest.raises(ValueError, match=why):
        heom._batch_of(H, torch.zeros(shape, dtype=torch.complex128))


def test_batch_of_refuses_non_contiguous_and_host_tensors():
    t = torch.zeros((7, 3, 3, 4), dtype=torch.complex128)
    with pytest.raises(ValueError, match="contiguous"):
        heom._batch_of(H, t[..., ::2])
    with pytest.raises(ValueError, match="CUDA"):
        heom._batch_of(H, t)  # the right shape on the host: still refused


def _ados(batch=2, dtype=torch.complex128):
    return torch.zeros((7, 3, 3, batch), dtype=dtype)


def test_noalloc_trajectory_buffer_is_checked():
    x = _ados()
    need = (10 // 5 + 1) * 9 * 2  # n_steps // save_every + 1 blocks of d x d x batch
    ok = torch.zeros(need, dtype=torch.complex128)
    heom._check_traj(H, x, 2, 10, 5, ok)  # accepted
    heom._check_traj(H, x, 2, 10, 0, None)  # no trajectory asked, none given
    with pytest.raises(ValueError, match="holds"):
        heom._check_traj(H, x, 2, 10, 5, ok[:-1])
    with pytest.raises(ValueError, match="dtype"):
        heom._check_traj(H, x, 2, 10, 5, torch.zeros(need, dtype=torch.complex64))
    with pytest.raises(ValueError, match="contiguous"):
        heom._check_traj(H, x, 2, 10, 5, torch.zeros(2 * need, dtype=torch.complex128)[::2])
    with pytest.raises(ValueError, match="save_every = 0"):
        heom._check_traj(H, x, 2, 10, 0, ok)
    with pytest.raises(ValueError, match="caller-owned"):
        heom._check_traj(H, x, 2, 10, 5, None)


def test_solver_inputs_are_checked():
    with pytest.raises(TypeError, match="complex128"):
        heom._need_c128(_ados(dtype=torch.complex64), "x_out")
    sets = SimpleNamespace(n_ado=7, d=3, device=None, n_sets=3)
    with pytest.raises(ValueError, match="n_sets = 3"):
        heom._check_sets(sets, torch.zeros((7, 3, 3, 2), dtype=torch.complex128))
    with pytest.raises(ValueError, match="does not match"):
        heom._check_sets(sets, torch.zeros((8, 3, 3, 3), dtype=torch.complex128))
