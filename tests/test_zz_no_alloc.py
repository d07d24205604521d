"""The allocation-free entry point (eval_models_noalloc) against the regular
context path (eval_models).

Some callers cannot allocate device memory (their host owns and budgets all
of it, or they run inside another runtime's memory pool, or in a loop that
forbids allocation after start-up); eval_models_noalloc serves them from a
fixed scratch array inside the library.  Two calls in a row must both match
eval_models within the misfit tolerance of the parity tests (the second call
reuses the scratch the first one left behind).  This file is collected last
so that a stop-at-first-failure run has already run everything else.
"""
import numpy as np
import pytest

from paper_1905_12795_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MISFIT_TOL = 1e-4


def test_noalloc_matches_context_twice():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_12795_gb300 import binding as B
    nx = nz = 101
    h = 10.0
    grid = B.make_grid(nx, nz, h, h, 20, 4, 0.5, 10.0, 1500.0, 2625.0)
    rec = synth.receiver_line(nx, h, 20.0)
    shots_xz = synth.shot_line(2, (nx - 1) * h, 20.0)
    sh = B.make_shots(shots_xz, [0, 0], [nx, nx], weights=[1.0, 0.5])
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    true = synth.two_layer_model(nx, nz, h)
    dobs = torch.zeros(2 * nt * nx, device="cuda")
    ctx.forward_traces(torch.tensor(true * 1.05, dtype=torch.float32, device="cuda")[None], sh, dobs)
    models = np.stack([true, true * 0.97, synth.layered_faulted_model(nx, nz, h, h, seed=4,
                                                                       vmax=2625.0)])
    vel = torch.tensor(models, dtype=torch.float32, device="cuda")
    ref = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.eval_models(vel, sh, dobs, ref)
    for _ in range(2):
        got = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
        B.eval_models_noalloc(grid, rec, vel, sh, dobs, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.abs(g - r) <= MISFIT_TOL * np.abs(r)), (g, r)
    ctx.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_1905_12795_gb300 import binding as B
    grid = B.make_grid(461, 151, 20.0, 20.0, 40, 8, 3.0, 6.0, 1500.0, 4700.0)
    rec = synth.receiver_line(461, 20.0, 20.0)
    sh = B.make_shots([(4600.0, 20.0)], [0], [461])
    M = 64
    vel = torch.full((M, 151, 461), 2000.0, device="cuda")
    _, nt = B.time_axis(grid)
    dobs = torch.zeros(nt * 461, device="cuda")
    with pytest.raises(B.EmpsoError) as e:
        B.eval_models_noalloc(grid, rec, vel, sh, dobs,
                              torch.zeros(M, dtype=torch.float64, device="cuda"))
    assert e.value.status == 6 and "scratch" in str(e.value)


def test_noalloc_binding_checks_what_the_library_cannot_see():
    """The C entry point receives raw device pointers, so the binding checks
    the tensors' types and sizes before the call: a float32 misfit buffer
    or a short d_obs would otherwise be written or read past its end."""
    from paper_1905_12795_gb300 import binding as B
    nx = nz = 41
    grid = B.make_grid(nx, nz, 10.0, 10.0, 5, 4, 0.2, 10.0, 1500.0, 3000.0)
    rec = synth.receiver_line(nx, 10.0, 20.0)
    sh = B.make_shots([(200.0, 20.0)], [0], [nx])
    _, nt = B.time_axis(grid)
    vel = torch.full((2, nz, nx), 2000.0, device="cuda")
    dobs = torch.zeros(nt * nx, device="cuda")
    mis = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        B.eval_models_noalloc(grid, rec, vel, sh, dobs, mis.float())
    with pytest.raises(TypeError):
        B.eval_models_noalloc(grid, rec, vel.double(), sh, dobs, mis)
    with pytest.raises(TypeError):
        B.eval_models_noalloc(grid, rec, vel[:, :, :-1], sh, dobs, mis)
    with pytest.raises(ValueError):
        B.eval_models_noalloc(grid, rec, vel, sh, dobs[:-1], mis)
    B.eval_models_noalloc(grid, rec, vel, sh, dobs, mis)
    torch.cuda.synchronize()
    assert np.all(mis.cpu().numpy() > 0.0)
