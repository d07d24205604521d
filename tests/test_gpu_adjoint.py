"""The adjoint-state gradient against the definition of a gradient, and the
local FWI that uses it.

The oracle of dphi/dv is the derivative of the FP64 oracle misfit itself:
central differences (phi(v + eps d) - phi(v - eps d)) / (2 eps) along a
direction d, compared with <grad, d> from the GPU (FP32 forward and adjoint
passes over a few hundred steps: 2e-3 relative for a dense direction, 1e-2
for a single node).  One node on the model's edge checks the fold of the
damping pad (the edge extension's transpose).
"""
import numpy as np
import pytest

import oracle
from paper_1905_12795_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_12795_gb300 import binding
    binding.load()
    return binding


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("kernel", [0, 1, 3])   # forward pass: on-chip / per step / L2 cluster kernel
@pytest.mark.parametrize("order", [4, 8])
def test_gradient_matches_oracle_directional_derivatives(B, order, kernel):
    nx, nz, h, pad, T, f0, vmax = 41, 31, 10.0, 8, 0.25, 15.0, 3000.0
    og = oracle.Grid(nx, nz, h, h, pad, order, T, f0, vmax)
    v = synth.layered_faulted_model(nx, nz, h, h, seed=5, vmin=1500.0, vmax=2800.0)
    v_true = synth.layered_faulted_model(nx, nz, h, h, seed=6, vmin=1500.0, vmax=2800.0)
    shots = np.array([[105.0, 23.0], [297.0, 41.0]])
    rec = synth.receiver_line(nx, h, 27.0)[:-1] + np.array([3.7, 0.0])
    nrec = len(rec)
    rb, rc = [0, 0], [nrec, nrec]
    w = [1.0, 0.5]
    _, obs = oracle.shot_batch(og, v_true, shots, rec, rb, rc, want_traces=True)

    def phi(vel):
        p, _ = oracle.shot_batch(og, vel, shots, rec, rb, rc, dobs=obs)
        return float(np.dot(w, p[0]))

    grid = B.make_grid(nx, nz, h, h, pad, order, T, f0, 1500.0, vmax)
    ctx = B.Context([grid], rec)
    ctx.set_kernel(kernel)
    sh = B.make_shots(shots, rb, rc, weights=w)
    dobs = _dev(np.concatenate([o.ravel() for o in obs]))
    g = torch.zeros(1, nz, nx, device="cuda")
    mis = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.gradient(_dev(v[None]), sh, dobs, g, mis)
    G = g[0].cpu().numpy().astype(np.float64)
    phi0 = phi(v)
    assert mis.item() == pytest.approx(phi0, rel=1e-4)
    # the same misfit as the modelling kernels give
    m2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.set_kernel(0)
    ctx.eval_models(_dev(v[None]), sh, dobs, m2)
    assert m2.item() == pytest.approx(mis.item(), rel=1e-5)
    rng = np.random.default_rng(order)
    cases = [(rng.normal(size=(nz, nx)), 1.0, 2e-3)]
    for (j, i) in ((4, 14), (20, 0)):        # near the sources; on the left edge (pad fold)
        d = np.zeros((nz, nx))
        d[j, i] = 1.0
        cases.append((d, 5.0, 1e-2))
    for d, eps, tol in cases:
        fd = (phi(v + eps * d) - phi(v - eps * d)) / (2 * eps)
        ad = float(np.sum(G * d))
        assert abs(ad - fd) <= tol * abs(fd), (ad, fd)
    ctx.close()


@pytest.mark.parametrize("kernel", [0, 1, 3])
@pytest.mark.parametrize("order", [4, 8])
def test_gradient_field_matches_oracle_at_every_node(B, order, kernel):
    """The whole dphi/dv field against FP64 central differences of the oracle
    misfit at every physical node of a tiny grid, edge and corner nodes
    (whose sensitivity includes the folded damping pad) included."""
    nx, nz, h, pad, T, f0, vmax = 14, 11, 10.0, 4, 0.1, 25.0, 3000.0
    og = oracle.Grid(nx, nz, h, h, pad, order, T, f0, vmax)
    v = synth.layered_faulted_model(nx, nz, h, h, seed=5, vmin=1500.0, vmax=2800.0)
    v_true = synth.layered_faulted_model(nx, nz, h, h, seed=6, vmin=1500.0, vmax=2800.0)
    shots = np.array([[35.0, 23.0], [97.0, 61.0]])
    rec = synth.receiver_line(nx, h, 15.0)[:-1] + np.array([3.7, 0.0])
    nrec = len(rec)
    rb, rc = [0, 0], [nrec, nrec]
    _, obs = oracle.shot_batch(og, v_true, shots, rec, rb, rc, want_traces=True)

    def phi(vel):
        p, _ = oracle.shot_batch(og, vel, shots, rec, rb, rc, dobs=obs)
        return float(np.sum(p[0]))

    ref = np.zeros((nz, nx))
    for j in range(nz):
        for i in range(nx):
            d = np.zeros((nz, nx))
            d[j, i] = 1.0
            ref[j, i] = (phi(v + d) - phi(v - d)) / 2.0
    grid = B.make_grid(nx, nz, h, h, pad, order, T, f0, 1500.0, vmax)
    ctx = B.Context([grid], rec)
    ctx.set_kernel(kernel)
    g = torch.zeros(1, nz, nx, device="cuda")
    ctx.gradient(_dev(v[None]), B.make_shots(shots, rb, rc),
                 _dev(np.concatenate([o.ravel() for o in obs])), g)
    got = g[0].cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    assert scale > 0.0
    assert np.abs(got - ref).max() <= 1e-2 * scale
    assert np.linalg.norm(got - ref) <= 5e-3 * np.linalg.norm(ref)
    ctx.close()


@pytest.mark.parametrize("kernel", [0, 1])
def test_gradient_order16_matches_oracle(B, kernel):
    """The gradient with the 16th-order operator of the paper's local FWI
    (per-step forward and adjoint launches) against central differences of
    the oracle misfit: a dense direction and one node on the model's edge."""
    nx, nz, h, pad, T, f0, vmax = 41, 31, 10.0, 10, 0.25, 15.0, 3000.0
    og = oracle.Grid(nx, nz, h, h, pad, 16, T, f0, vmax)
    v = synth.layered_faulted_model(nx, nz, h, h, seed=5, vmin=1500.0, vmax=2800.0)
    v_true = synth.layered_faulted_model(nx, nz, h, h, seed=6, vmin=1500.0, vmax=2800.0)
    shots = np.array([[105.0, 23.0], [297.0, 41.0]])
    rec = synth.receiver_line(nx, h, 27.0)[:-1] + np.array([3.7, 0.0])
    nrec = len(rec)
    rb, rc = [0, 0], [nrec, nrec]
    _, obs = oracle.shot_batch(og, v_true, shots, rec, rb, rc, want_traces=True)

    def phi(vel):
        p, _ = oracle.shot_batch(og, vel, shots, rec, rb, rc, dobs=obs)
        return float(np.sum(p[0]))

    ctx = B.Context([B.make_grid(nx, nz, h, h, pad, 16, T, f0, 1500.0, vmax)], rec)
    ctx.set_kernel(kernel)
    g = torch.zeros(1, nz, nx, device="cuda")
    mis = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.gradient(_dev(v[None]), B.make_shots(shots, rb, rc),
                 _dev(np.concatenate([o.ravel() for o in obs])), g, mis)
    G = g[0].cpu().numpy().astype(np.float64)
    assert mis.item() == pytest.approx(phi(v), rel=1e-4)
    rng = np.random.default_rng(16)
    cases = [(rng.normal(size=(nz, nx)), 1.0, 2e-3)]
    d = np.zeros((nz, nx))
    d[20, 0] = 1.0
    cases.append((d, 5.0, 1e-2))
    for d, eps, tol in cases:
        fd = (phi(v + eps * d) - phi(v - eps * d)) / (2 * eps)
        ad = float(np.sum(G * d))
        assert abs(ad - fd) <= tol * abs(fd), (ad, fd)
    ctx.close()


def test_gradient_batch_of_models_equals_single_calls(B):
    nx, nz, h = 37, 29, 10.0
    grid = B.make_grid(nx, nz, h, h, 6, 4, 0.2, 15.0, 1500.0, 3000.0)
    rec = synth.receiver_line(nx, h, 20.0)
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    sh = B.make_shots([(120.0, 20.0), (240.0, 20.0)], [0, 0], [nx, nx])
    dobs = torch.randn(2 * nt * nx, device="cuda") * 1e-3
    vs = np.stack([synth.layered_faulted_model(nx, nz, h, h, seed=s, vmin=1500.0, vmax=2800.0)
                   for s in (1, 2, 3)])
    g3 = torch.zeros(3, nz, nx, device="cuda")
    m3 = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.gradient(_dev(vs), sh, dobs, g3, m3)
    for k in range(3):
        g1 = torch.zeros(1, nz, nx, device="cuda")
        m1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.gradient(_dev(vs[k:k + 1]), sh, dobs, g1, m1)
        assert torch.equal(g1[0], g3[k]) and m1.item() == m3[k].item()
    # the per-step forward pass agrees with the on-chip one to FP32 rounding
    ctx.set_kernel(1)
    gs = torch.zeros(3, nz, nx, device="cuda")
    ms = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.gradient(_dev(vs), sh, dobs, gs, ms)
    scale = float(g3.abs().max())
    assert float((gs - g3).abs().max()) <= 1e-4 * scale
    assert torch.allclose(ms, m3, rtol=1e-5)
    ctx.close()


def test_gradient_chains_give_identical_results(B):
    """The backward pass split into 1..8 concurrent chains of instances (5
    instances: uneven chains, and more chains than instances) computes every
    instance the same way."""
    nx, nz, h = 37, 29, 10.0
    grid = B.make_grid(nx, nz, h, h, 6, 8, 0.2, 15.0, 1500.0, 3000.0)
    rec = synth.receiver_line(nx, h, 20.0)
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    xs = [60.0, 120.0, 180.0, 240.0, 300.0]
    sh = B.make_shots([(x, 20.0) for x in xs], [0] * 5, [nx] * 5, weights=[1.0, 0.5, 2.0, 1.0, 0.25])
    dobs = torch.randn(5 * nt * nx, device="cuda") * 1e-3
    v = _dev(synth.layered_faulted_model(nx, nz, h, h, seed=4, vmin=1500.0, vmax=2800.0)[None])
    out = []
    for chains in (1, 2, 3, 4, 8):
        ctx.set_gradient_chains(chains)
        g = torch.zeros(1, nz, nx, device="cuda")
        m = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.gradient(v, sh, dobs, g, m)
        out.append((g, m.item()))
    for g, m in out[1:]:
        assert torch.equal(g, out[0][0]) and m == out[0][1]
    with pytest.raises(B.EmpsoError):
        ctx.set_gradient_chains(9)
    ctx.close()


def test_gradient_edge_cases(B):
    nx, nz, h = 37, 29, 10.0
    grid = B.make_grid(nx, nz, h, h, 6, 8, 0.2, 15.0, 1500.0, 3000.0)
    rec = synth.receiver_line(nx, h, 20.0)
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    v = _dev(synth.layered_faulted_model(nx, nz, h, h, seed=4, vmin=1500.0, vmax=2800.0)[None])
    dobs = torch.randn(nt * nx, device="cuda") * 1e-3
    g1 = torch.zeros(1, nz, nx, device="cuda")
    m1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.gradient(v, B.make_shots([(120.0, 20.0)], [0], [nx]), dobs, g1, m1)
    assert m1.item() > 0.0 and float(g1.abs().max()) > 0.0
    # a shot without receivers has no residual, no adjoint source and zero
    # misfit: adding it changes neither the gradient nor the misfit
    g2 = torch.zeros(1, nz, nx, device="cuda")
    m2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.gradient(v, B.make_shots([(120.0, 20.0), (250.0, 20.0)], [0, 0], [nx, 0]), dobs, g2, m2)
    assert torch.equal(g1, g2) and m1.item() == m2.item()
    # invalid arguments are refused before any launch
    sh = B.make_shots([(120.0, 20.0)], [0], [nx])
    with pytest.raises(B.EmpsoError) as e:
        ctx.gradient(v[:0], sh, dobs, g1)
    assert e.value.status == 1
    with pytest.raises(B.EmpsoError) as e:
        ctx.gradient(v, B.make_shots([(-5.0, 20.0)], [0], [nx]), dobs, g1)
    assert e.value.status == 1
    ctx.close()


@pytest.mark.parametrize("order", [4, 16])
def test_fwi_descends_and_improves_the_model(B, order):
    """Steepest descent with the BB step and backtracking (section "Testing
    approach", local FWI) from a smoothed model; order 16 is the paper's
    operator for it (line-search misfits on the gradient's forward pass)."""
    nx, nz, h, pad = 61, 41, 10.0, 10
    grid = B.make_grid(nx, nz, h, h, pad, order, 0.45, 12.0, 1400.0, 3000.0)
    rec = synth.receiver_line(nx, h, 20.0)
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    shots = synth.shot_line(3, (nx - 1) * h, 20.0)
    sh = B.make_shots(shots, [0] * 3, [nx] * 3)
    true = synth.layered_faulted_model(nx, nz, h, h, seed=11, vmin=1500.0, vmax=2600.0)
    dobs = torch.zeros(3 * nt * nx, device="cuda")
    ctx.forward_traces(_dev(true[None]), sh, dobs)
    # start: the true model smoothed by a 9 x 9 box (a background model)
    k = 4
    pad_t = np.pad(true, k, mode="edge")
    start = np.zeros_like(true)
    for dj in range(-k, k + 1):
        for di in range(-k, k + 1):
            start += pad_t[k + dj:k + dj + nz, k + di:k + di + nx]
    start /= (2 * k + 1) ** 2
    vel = _dev(start)
    hist = ctx.fwi(vel, sh, dobs, 8, 1400.0, 3000.0)
    assert len(hist) >= 5
    assert all(b < a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 0.5 * hist[0]
    err0 = np.linalg.norm(start - true)
    err1 = np.linalg.norm(vel.cpu().numpy() - true)
    assert err1 < err0
    assert float(vel.min()) >= 1400.0 and float(vel.max()) <= 3000.0
    ctx.close()
