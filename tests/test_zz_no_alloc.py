"""heom_evolve_noalloc -- RK4 for callers that cannot let the library allocate device memory
(their memory is held by another allocator, or a cudaFree stall is not acceptable).

Called through the C ABI, twice in a row on different systems, and compared with heom_evolve
on the same inputs. The second call also checks that what the first call left in the shared
static scratch does not leak into the next result. This file is named to be collected last.
"""
import numpy as np
import pytest

import workloads as W
from oracle import solvers as so
from tests.helpers import rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_07522_gb300 as heom
    return heom


def _pair(heom, model, dt, n_steps, save_every, batch):
    import torch
    g = heom.build_hierarchy(heom.problem_from_model(model))
    X = so.initial_vector(g.n_ado, model.rho0)
    X = np.repeat(X[..., None], batch, axis=-1) * np.linspace(1.0, 0.5, batch)
    ref = to_dev(X, torch.complex128)
    ref_traj = heom.evolve(g, ref, dt, n_steps, save_every)
    x = to_dev(X, torch.complex128)
    traj = torch.empty_like(ref_traj)
    heom.evolve_noalloc(g, x, dt, n_steps, save_every, traj=traj)
    torch.cuda.synchronize()
    return (x.cpu().numpy(), ref.cpu().numpy(), traj.cpu().numpy(), ref_traj.cpu().numpy())


def test_noalloc_matches_evolve_on_two_calls_in_a_row(heom):
    # call 1: SIAM tier 2 (301 ADOs x 16 elements x 4 columns)
    x, ref, t, rt = _pair(heom, W.siam_model(tier=2), 0.005, 100, 25, 4)
    assert rel_err(x, ref) < 1e-10 and rel_err(t, rt) < 1e-10
    # call 2: spin-boson tier 4, a smaller problem that reuses the same scratch
    x, ref, t, rt = _pair(heom, W.spin_boson_model(tier=4), 0.01, 200, 50, 3)
    assert rel_err(x, ref) < 1e-10 and rel_err(t, rt) < 1e-10


def test_noalloc_call_allocates_nothing(heom):
    """After the first call on the device (which looks up the static scratch), further calls
    make no device allocation and grow no workspace: the library's allocation counters
    (every cudaMalloc of the library goes through one counted routine) stay put, and the
    hierarchy's own RK4 workspace is never taken."""
    import torch
    model = W.siam_model(tier=2)
    g = heom.build_hierarchy(heom.problem_from_model(model))
    X = so.initial_vector(g.n_ado, model.rho0)
    x = to_dev(X, torch.complex128)
    traj = torch.empty((5, 4, 4), dtype=torch.complex128, device="cuda")
    heom.evolve_noalloc(g, x, 0.01, 0)  # set-up call: n_steps = 0 does the lookup only
    torch.cuda.synchronize()
    before = heom.profile_allocs()
    heom.evolve_noalloc(g, x, 0.01, 40, 10, traj=traj)
    heom.evolve_noalloc(g, x, 0.01, 40, 10, traj=traj)
    torch.cuda.synchronize()
    assert heom.profile_allocs() == before
    ref = to_dev(X, torch.complex128)
    heom.evolve(g, ref, 0.01, 80)  # heom_evolve on the same hierarchy does take a workspace
    assert heom.profile_allocs()["workspace_takes"] == before["workspace_takes"] + 1
    assert rel_err(x.cpu().numpy(), ref.cpu().numpy()) < 1e-10


def test_noalloc_refuses_requests_beyond_its_scratch(heom):
    import torch
    g = heom.build_hierarchy(heom.problem_from_model(W.siam_model(tier=3)))
    # 2,325 ADOs x 16 x 64 columns x 16 B x 3 buffers = 114 MB > 16 MiB
    x = torch.zeros((g.n_ado, 4, 4, 64), dtype=torch.complex128, device="cuda")
    with pytest.raises(heom.HeomError) as e:
        heom.evolve_noalloc(g, x, 0.01, 1)
    assert e.value.status == heom.EINVAL
