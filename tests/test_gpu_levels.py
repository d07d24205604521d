"""GPU parity of the irregular level-wise control grid ("Testing approach":
two-grid strategy with a variable node spacing, fixed water layer,
depth-dependent search ranges) against the FP64 oracle.

Velocities: the taps are computed in FP64 from the same FP32 node positions
the oracle receives, the four-tap sum in FP32: 2e-6 relative.  Fitness: the
modelling bar of the other parity tests (1e-4 relative misfit).
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


def _layout(nx, nz, h, water, f0):
    lz, lc, node_x, v1d = synth.level_layout((nx - 1) * h, (nz - 1) * h, water, f0=f0)
    # the library takes FP32 positions: give the oracle exactly those values
    return (lz.astype(np.float32).astype(np.float64), lc,
            node_x.astype(np.float32).astype(np.float64), v1d)


@pytest.mark.parametrize("water", [0.0, 60.0])
def test_level_interp_matches_oracle(B, water):
    nx, nz, h = 121, 61, 10.0
    lz, lc, node_x, _ = _layout(nx, nz, h, water, 12.0)
    K = int(lc.sum())
    grid = B.make_grid(nx, nz, h, h, 5, 8, 0.2, 12.0, 1500.0, 4700.0)
    ctx = B.Context([grid], [[0.0, 0.0]])
    ctx.set_levels(0, lz, lc, node_x)
    if water:
        ctx.set_water(0, water, 1500.0)
    parts = synth.random_particles(4, K, 1000.0, 5200.0, seed=21)   # some nodes clipped
    out = torch.zeros(4, nz, nx, device="cuda")
    ctx.interp(0, _dev(parts), out)
    got = out.cpu().numpy()
    for p in range(4):
        ref = oracle.interp_levels(lz, lc, node_x, parts[p].astype(np.float32), nz, nx, h, h,
                                   water, 1500.0, 1500.0, 4700.0)
        assert np.max(np.abs(got[p] - ref) / ref) < 2e-6
        if water:
            assert np.all(got[p][: int(water / h) + 1] == 1500.0)
    ctx.close()


def test_level_bounds_match_oracle(B):
    lz, lc, _, v1d = _layout(121, 61, 10.0, 60.0, 12.0)
    lo, hi = B.level_bounds(lz, lc, float(v1d(lz[0])), float(v1d(lz[-1])), 0.25, 0.25, 0.3, 0.2)
    lo_r, hi_r = oracle.level_bounds(lz, lc, float(v1d(lz[0])), float(v1d(lz[-1])), 0.25, 0.25,
                                     0.3, 0.2)
    assert np.allclose(lo, lo_r, rtol=1e-15) and np.allclose(hi, hi_r, rtol=1e-15)
    with pytest.raises(B.EmpsoError):
        B.level_bounds(lz[::-1].copy(), lc, 1500.0, 3000.0, 0.1, 0.1, 0.1, 0.1)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_level_fitness_and_generation_match_oracle(B, kind):
    nx, nz, h, pad = 77, 35, 20.0, 12
    vmin, vmax, water = 1500.0, 4700.0, 40.0
    og = oracle.Grid(nx, nz, h, h, pad, 8, 0.8, 6.0, vmax)
    lz, lc, node_x, v1d = _layout(nx, nz, h, water, 6.0)
    K, P = int(lc.sum()), 6
    true = synth.layered_faulted_model(nx, nz, h, h, seed=1905, vmin=vmin, vmax=vmax)
    shots = synth.shot_line(3, (nx - 1) * h, 20.0)
    rec = synth.receiver_line(nx, h, 20.0)
    rb, rc = [0] * 3, [nx] * 3
    _, obs = oracle.shot_batch(og, true, shots, rec, rb, rc, want_traces=True)
    lo, hi = oracle.level_bounds(lz, lc, float(v1d(lz[0])), float(v1d(lz[-1])), 0.3, 0.3, 0.3,
                                 0.3)
    grid = B.make_grid(nx, nz, h, h, pad, 8, 0.8, 6.0, vmin, vmax)
    pso = B.EmpsoPso(P, K, 1.2, 2.9, 0.5, 0.3, 0.25, 2, 1, 31)
    ctx = B.Context([grid], rec, pso, lo, hi)
    ctx.set_kernel(kind)
    ctx.set_levels(0, lz, lc, node_x)
    ctx.set_water(0, water, 1500.0)
    x0 = torch.zeros(P, K, device="cuda")
    ctx.pso_init(x0)
    parts = x0.cpu().numpy()
    assert np.all(parts >= lo.astype(np.float32) - 1e-3) and np.all(parts <= hi.astype(np.float32) + 1e-3)
    ref = []
    for p in range(P):
        vel = oracle.interp_levels(lz, lc, node_x, parts[p], og.nz, og.nx, h, h, water, 1500.0,
                                   vmin, vmax)
        phi, _ = oracle.shot_batch(og, vel, shots, rec, rb, rc, dobs=obs)
        ref.append(float(np.sum(phi[0])))
    sh = B.make_shots(shots, rb, rc)
    dobs = _dev(np.concatenate([o.ravel() for o in obs]))
    mis = torch.zeros(P, dtype=torch.float64, device="cuda")
    ctx.eval_fitness(x0, sh, dobs, mis)
    assert ctx.last_launch()[0] == kind
    e = 0.5 * sum(np.sum(o ** 2) for o in obs)
    got = mis.cpu().numpy()
    for g, r in zip(got, ref):
        if r >= 1e-4 * e:
            assert abs(g - r) <= 1e-4 * r, (g, r)
        else:
            assert abs(g - r) <= 1e-4 * e, (g, r)
    # a captured generation on the level grid evaluates the same positions
    mis_g = torch.zeros_like(mis)
    ctx.generation(sh, dobs, mis_g)
    assert torch.equal(mis_g, mis)
    ctx.close()


def test_level_errors(B):
    grid = B.make_grid(41, 31, 10.0, 10.0, 5, 4, 0.2, 10.0, 1500.0, 4700.0)
    ctx = B.Context([grid], [[0.0, 0.0]])
    with pytest.raises(B.EmpsoError) as e:
        ctx.set_levels(0, [100.0, 50.0], [2, 2], [0.0, 400.0, 0.0, 400.0])
    assert e.value.status == 1
    with pytest.raises(B.EmpsoError) as e:
        ctx.set_levels(0, [50.0, 100.0], [2, 2], [0.0, 400.0, 400.0, 0.0])
    assert e.value.status == 1
    with pytest.raises(B.EmpsoError) as e:
        ctx.set_levels(0, [50.0, 100.0], [600, 600], np.tile(np.arange(600.0), 2))
    assert e.value.status == 6
    with pytest.raises(B.EmpsoError) as e:
        ctx.set_levels(1, [50.0], [2], [0.0, 1.0])
    assert e.value.status == 1
    ctx.close()
