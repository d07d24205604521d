"""GPU parity of the EMPSO step against the FP64 CPU oracle.

Both sides draw from Philox4x32-10 with the same counters and evaluate every
FP64 operation (including the series log/cos of the Box-Muller normals) in the
same order without fused multiply-adds, so the integer bookkeeping (global
best, sort order, elite set, generation) must agree exactly and the FP64
state bit for bit.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_12795_gb300 import binding
    binding.load()
    return binding


def _ctx(B, P, D, lo, hi, **kw):
    cfg = dict(c1=1.2, c2=2.9, lam=0.5, p_em=0.3, nm_frac=0.25, em_start=10, em_enabled=True,
               seed=12795)
    cfg.update(kw)
    pso = B.EmpsoPso(P, D, cfg["c1"], cfg["c2"], cfg["lam"], cfg["p_em"], cfg["nm_frac"],
                     cfg["em_start"], 1 if cfg["em_enabled"] else 0, cfg["seed"])
    grid = B.make_grid(11, 11, 10.0, 10.0, 0, 2, 0.05, 10.0, 1.0, 2.0, kx=2, kz=2)
    ctx = B.Context([grid], [[0.0, 0.0]], pso, lo, hi)
    sw = oracle.Swarm(P, D, lo, hi, cfg["c1"], cfg["c2"], cfg["lam"], cfg["p_em"],
                      cfg["nm_frac"], cfg["em_start"], cfg["em_enabled"], cfg["seed"])
    return ctx, sw


def _state(ctx, P, D):
    dv = "cuda"
    x = torch.zeros(P, D, dtype=torch.float64, device=dv)
    v, p = torch.zeros_like(x), torch.zeros_like(x)
    pf = torch.zeros(P, dtype=torch.float64, device=dv)
    order = torch.zeros(P, dtype=torch.int32, device=dv)
    gk = torch.zeros(2, dtype=torch.int32, device=dv)
    ctx.pso_get_state(x, v, p, pf, order, gk)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (x, v, p, pf, order, gk)]


def _same(ctx, sw, P, D):
    x, v, p, pf, order, gk = _state(ctx, P, D)
    assert gk[0] == sw.g and gk[1] == sw.k
    assert np.array_equal(order, sw.order)
    assert np.array_equal(pf, sw.pf)
    assert np.array_equal(x, sw.x)
    assert np.array_equal(v, sw.v)
    assert np.array_equal(p, sw.p)


@pytest.mark.parametrize("P,D", [(32, 32), (7, 3), (1024, 32), (300, 192)])
def test_init_bit_exact(B, P, D):
    lo, hi = np.linspace(1200, 1500, D), np.linspace(3200, 4700, D)
    ctx, sw = _ctx(B, P, D, lo, hi)
    out = torch.zeros(P, D, device="cuda")
    ctx.pso_init(out)
    _same(ctx, sw, P, D)
    assert np.array_equal(out.cpu().numpy(), sw.x.astype(np.float32))
    ctx.close()


@pytest.mark.parametrize("P,D,em_start", [(32, 32, 1), (33, 5, 1), (1024, 32, 1), (16, 8, 99), (2048, 64, 1),
                                            (1000, 7, 1)])
def test_step_from_given_state_bit_exact(B, P, D, em_start):
    rng = np.random.default_rng(P + D)
    lo, hi = -5.0, 5.0
    ctx, sw = _ctx(B, P, D, lo, hi, em_start=em_start, nm_frac=0.25)
    x = rng.uniform(-5, 5, (P, D))
    v = rng.uniform(-2, 2, (P, D))
    p = np.clip(x + rng.uniform(-1, 1, (P, D)), -5, 5)
    pf = rng.uniform(1, 10, P)
    f = rng.uniform(0, 12, P)
    f[::7] = f[0]                    # ties in the fitness: stable order decides
    f[3 % P] = np.nan                # non-finite fitness counts as +inf
    f[5 % P] = np.inf
    g0 = int(np.argmin(pf))
    k0 = 4
    sw.set_state(x, v, p, pf, g0, k0)
    dv = "cuda"
    ctx.pso_set_state(*(torch.tensor(a, device=dv) for a in (x, v, p, pf)), g0, k0)
    out = torch.zeros(P, D, device=dv)
    mis = torch.tensor(f, device=dv)
    g = ctx.pso_step(mis, out, want_gbest=True)
    sw.step(f)
    assert g == sw.g
    _same(ctx, sw, P, D)
    assert np.array_equal(out.cpu().numpy(), sw.x.astype(np.float32))
    ctx.close()


def _sphere(x):
    return np.sum(x * x, axis=1)


def _rastrigin(x):
    return 10.0 * x.shape[1] + np.sum(x * x - 10.0 * np.cos(2 * np.pi * x), axis=1)


@pytest.mark.parametrize("fn,D,gens", [(_sphere, 10, 120), (_rastrigin, 4, 120)])
def test_full_run_identical(B, fn, D, gens):
    """Whole EMPSO runs with an FP64 test function evaluated on the host for
    both swarms: every generation's global best, sort order and state agree."""
    P = 40
    ctx, sw = _ctx(B, P, D, -5.12, 5.12, em_start=12)
    ctx.pso_init()
    xs = torch.zeros(P, D, dtype=torch.float64, device="cuda")
    for _ in range(gens):
        ctx.pso_get_state(x=xs)
        fx = fn(xs.cpu().numpy())
        assert np.array_equal(xs.cpu().numpy(), sw.x)
        f_or = fn(sw.x)
        ctx.pso_step(torch.tensor(fx, device="cuda"))
        sw.step(f_or)
    _same(ctx, sw, P, D)
    assert np.min(sw.pf) < (1e-2 if fn is _sphere else 1.0)   # sanity: the run made progress
    ctx.close()


def test_uninitialised_swarm(B):
    grid = B.make_grid(11, 11, 10.0, 10.0, 0, 2, 0.05, 10.0, 1.0, 2.0, kx=2, kz=2)
    ctx = B.Context([grid], [[0.0, 0.0]])
    with pytest.raises(B.EmpsoError) as e:
        ctx.pso_init()
    assert e.value.status == 7
    with pytest.raises(B.EmpsoError) as e:
        B.Context([grid], [[0.0, 0.0]], B.EmpsoPso(4096, 4, 1.2, 2.9, 0.5, 0.3, 0.25, 10, 1, 1),
                  0.0, 1.0)
    assert e.value.status == 6
    with pytest.raises(B.EmpsoError) as e:     # phi = c1 + c2 < 4 has no real constriction
        B.Context([grid], [[0.0, 0.0]], B.EmpsoPso(4, 4, 1.0, 1.0, 0.5, 0.3, 0.25, 10, 1, 1),
                  0.0, 1.0)
    assert e.value.status == 1
    ctx.close()


def test_checkpoint_resume_bit_exact(B):
    """Checkpoint/resume: the swarm state (x, v, p, pf, g, k) is the whole
    state of a run because the random numbers are counter-based; restoring it
    into a fresh context continues the run bit for bit."""
    P, D = 24, 8
    ctx, _ = _ctx(B, P, D, -5.12, 5.12, em_start=3)
    ctx.pso_init()
    xs = torch.zeros(P, D, dtype=torch.float64, device="cuda")

    def run(c, gens):
        for _ in range(gens):
            c.pso_get_state(x=xs)
            c.pso_step(torch.tensor(_rastrigin(xs.cpu().numpy()), device="cuda"))

    run(ctx, 6)
    x, v, p, pf, order, gk = _state(ctx, P, D)
    run(ctx, 6)
    ref = _state(ctx, P, D)
    ctx2, _ = _ctx(B, P, D, -5.12, 5.12, em_start=3)
    ctx2.pso_set_state(*(torch.tensor(a, device="cuda") for a in (x, v, p, pf)), int(gk[0]),
                       int(gk[1]))
    run(ctx2, 6)
    got = _state(ctx2, P, D)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    ctx.close()
    ctx2.close()
