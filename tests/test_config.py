"""The run configuration in the paper's JSON layout: the paper's own example
(tests/golden/paper_json_example.json, from its JSON example figure) is read,
converted to SI units and turned into a library context; one generation of it
runs on the GPU with a per-generation log."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
EXAMPLE = os.path.join(HERE, "golden", "paper_json_example.json")


def test_paper_example_in_si_units():
    from paper_1905_12795_gb300 import config
    cfg = config.load(EXAMPLE)
    assert (cfg.nx, cfg.nz, cfg.hx, cfg.hz, cfg.pad, cfg.order) == (369, 375, 25.0, 8.0, 40, 8)
    assert cfg.T == pytest.approx(4.0) and cfg.dt == pytest.approx(0.61e-3) and cfg.f0 == pytest.approx(3.0)
    assert cfg.shots.shape == (50, 2)
    assert cfg.shots[0, 0] == 175.0 and cfg.shots[-1, 0] == 175.0 * 50 and np.all(cfg.shots[:, 1] == 0.0)
    assert cfg.receivers.shape == (369, 2)
    assert cfg.receivers[-1, 0] == pytest.approx(368 * 25.0)
    assert cfg.water_depth == pytest.approx(32.0)
    assert (cfg.gens, cfg.c1, cfg.c2, cfg.lam) == (100, 2.0, 2.0, 0.5)
    # the paper's EMPSO settings fill what the example leaves out
    assert (cfg.npop, cfg.p_em, cfg.nm_frac, cfg.em_start) == (360, 0.3, 0.25, 10)
    # unknowns: a level grid of the same order as the paper's 176 nodes
    assert 150 <= cfg.K <= 200 and cfg.level_count[0] > cfg.level_count[-1]
    assert np.all(cfg.xmin < cfg.xmax)
    # the library's time axis for the given dt: 4 s at 0.61 ms
    from paper_1905_12795_gb300 import binding as B
    g = B.make_grid(cfg.nx, cfg.nz, cfg.hx, cfg.hz, cfg.pad, cfg.order, cfg.T, cfg.f0, cfg.vmin,
                    cfg.vmax, dt=cfg.dt)
    dt, nt = B.time_axis(g)
    assert nt == 6558 and dt == pytest.approx(0.61e-3)


def test_overrides_and_missing_keys():
    from paper_1905_12795_gb300 import config
    cfg = config.load(EXAMPLE, {"nshots": 2, "pso": {"npop": 8, "gen": 3}, "cgrid": {"scale": 1.25}})
    base = config.load(EXAMPLE)
    assert cfg.shots.shape == (2, 2) and cfg.npop == 8 and cfg.gens == 3 and cfg.c1 == 2.0
    assert cfg.K < base.K
    raw = json.load(open(EXAMPLE))
    del raw["pso"]
    with pytest.raises(KeyError):
        config.load(raw)
    # the optional surrogate group (not in the paper): defaults filled, keys checked
    sur = config.load(EXAMPLE, {"surrogate": {"keep": 0.5}}).surrogate
    assert sur["keep"] == 0.5 and sur["hidden"] == 256 and sur["train_steps"] == 6 and sur["batch"] == 1024
    assert config.load(EXAMPLE).surrogate is None
    with pytest.raises(KeyError):
        config.load(EXAMPLE, {"surrogate": {"keeep": 0.5}})
    with pytest.raises(ValueError):
        config.load(EXAMPLE, {"surrogate": {"keep": 0.0}})


@pytest.mark.gpu
def test_one_generation_from_the_paper_example(tmp_path):
    """The paper's example (4 s at 0.61 ms = 6558 steps on the 449 x 455
    padded grid), reduced to 2 shots and 4 particles, runs one EMPSO
    generation; the log holds one record and the final swarm."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_1905_12795_gb300 import config
    cfg = config.load(EXAMPLE, {"nshots": 2, "pso": {"npop": 4}})
    log = tmp_path / "run.jsonl"
    recs = config.run(cfg, str(log), gens=1)
    assert len(recs) == 1
    r = recs[0]
    assert r["evaluations"] == 4 and r["nonfinite"] == 0
    assert 0.0 < r["best_misfit"] <= r["mean_misfit"] and r["gbest_misfit"] == r["best_misfit"]
    assert r["updates_per_s"] > 1e9
    lines = log.read_text().splitlines()
    assert len(lines) == 2
    final = json.loads(lines[-1])
    assert len(final["final_swarm"]) == 4 and len(final["final_swarm"][0]) == cfg.K


@pytest.mark.gpu
def test_surrogate_generations_from_the_paper_example(tmp_path):
    """The same reduced example with the surrogate group: a warm-up
    generation models all 8 particles, the next ones the predicted-best
    quarter, and their records carry the surrogate's rank correlation."""
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_1905_12795_gb300 import config
    cfg = config.load(EXAMPLE, {"nshots": 1, "tn": 1000.0, "pso": {"npop": 8},
                                "surrogate": {"hidden": 64, "capacity": 256, "batch": 8}})
    recs = config.run(cfg, str(tmp_path / "run.jsonl"), gens=3)
    assert [r["modelled"] for r in recs] == [8, 2, 2]
    assert [r["evaluations"] for r in recs] == [8, 10, 12]
    assert recs[0]["surrogate_rank_corr"] is None
    assert all(-1.0 <= r["surrogate_rank_corr"] <= 1.0 for r in recs[1:])
    assert all(r["gbest_misfit"] <= r["best_misfit"] for r in recs)
