"""Batching machinery: one EMPSO generation captured as a CUDA graph must give
the same swarm as the eager calls, and the autotuner's choice must be used,
persisted and reloaded."""
import json
import os

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


def _problem(B, P=6, S=3, seed=12795):
    nx, nz, h, pad = 77, 35, 20.0, 12
    grid = B.make_grid(nx, nz, h, h, pad, 8, 0.8, 6.0, 1500.0, 4700.0)
    rec = synth.receiver_line(nx, h, 20.0)
    shots_xz = synth.shot_line(S, (nx - 1) * h, 20.0)
    sh = B.make_shots(shots_xz, [0] * S, [nx] * S)
    og = oracle.Grid(nx, nz, h, h, pad, 8, 0.8, 6.0, 4700.0)
    true = synth.layered_faulted_model(nx, nz, h, h, seed=1905)
    _, obs = oracle.shot_batch(og, true, shots_xz, rec, [0] * S, [nx] * S, want_traces=True)
    dobs = torch.tensor(np.concatenate([o.ravel() for o in obs]), dtype=torch.float32,
                        device="cuda")
    pso = B.EmpsoPso(P, 32, 1.2, 2.9, 0.5, 0.3, 0.34, 2, 1, seed)
    return grid, rec, sh, dobs, pso


def _state(ctx, P, D):
    x = torch.zeros(P, D, dtype=torch.float64, device="cuda")
    v, p = torch.zeros_like(x), torch.zeros_like(x)
    pf = torch.zeros(P, dtype=torch.float64, device="cuda")
    gk = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.pso_get_state(x=x, v=v, p=p, pf=pf, gk=gk)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (x, v, p, pf, gk)]


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_graph_generation_equals_eager(B, kind):
    grid, rec, sh, dobs, pso = _problem(B)
    P = pso.P
    eager = B.Context([grid], rec, pso, 1500.0, 4700.0)
    graph = B.Context([grid], rec, pso, 1500.0, 4700.0)
    for c in (eager, graph):
        c.set_kernel(kind)
    x = torch.zeros(P, 32, device="cuda")
    mis = torch.zeros(P, dtype=torch.float64, device="cuda")
    gmis = torch.zeros(P, dtype=torch.float64, device="cuda")
    eager.pso_init(x)
    graph.pso_init()
    for gen in range(4):
        eager.eval_fitness(x, sh, dobs, mis)
        eager.pso_step(mis, x)
        graph.generation(sh, dobs, gmis)
        torch.cuda.synchronize()
        assert torch.equal(mis, gmis), gen
    for a, b in zip(_state(eager, P, 32), _state(graph, P, 32)):
        assert np.array_equal(a, b)
    assert graph.last_launch()[0] == kind
    eager.close()
    graph.close()


def test_autotune_choice_is_used_and_cached(B, tmp_path):
    grid, rec, sh, dobs, pso = _problem(B, P=4, S=2)
    cache = str(tmp_path / "tune.jsonl")
    ctx = B.Context([grid], rec)
    ctx.set_tuning_cache(cache)
    x = torch.tensor(synth.random_particles(4, 32, 1500.0, 4700.0, seed=2), dtype=torch.float32,
                     device="cuda")
    mis = torch.zeros(4, dtype=torch.float64, device="cuda")
    kind, cl = ctx.autotune(x, sh, dobs, mis)
    assert kind in (1, 2) and (kind == 1) == (cl == 0)
    ref = mis.clone()
    ctx.eval_fitness(x, sh, dobs, mis)
    assert ctx.last_launch() == (kind, cl if kind == 2 else 1)
    # every candidate computes the same misfits to FP32 rounding
    assert torch.allclose(mis, ref, rtol=1e-4)
    lines = [json.loads(s) for s in open(cache)]
    assert lines and lines[-1]["kind"] == kind and lines[-1]["cluster"] == cl
    ctx.close()
    # a new context picks the cached choice for the same batch shape
    ctx2 = B.Context([grid], rec)
    ctx2.set_tuning_cache(cache)
    ctx2.eval_fitness(x, sh, dobs, mis)
    assert ctx2.last_launch() == (kind, cl if kind == 2 else 1)
    ctx2.close()
