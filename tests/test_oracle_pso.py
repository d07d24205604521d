"""Pins for the oracle's EMPSO ("Theory": Eq. 1-3 and the elitist-mutation
figure; "Testing approach": EMPSO parameters and the box constraint).

Closed forms (Clerc's constriction constant), the invariants the method
defines (strict personal-best update, lowest-index global best, the NM worst
particles by a stable ascending sort are the ones mutated, their velocities
untouched, mutation spread 0.1 VR with probability p_em), and the known minima
of the sphere and Rastrigin functions.
"""
import numpy as np
import pytest
from scipy import stats


def test_constriction_closed_form(orc):
    # Clerc & Kennedy (2002): phi = 4.1 gives chi = 0.7298437881...
    assert orc.chi(1.2, 2.9) == pytest.approx(0.72984378812835757, rel=1e-15)
    assert orc.chi(2.05, 2.05) == pytest.approx(0.72984378812835757, rel=1e-15)
    assert orc.chi(2.0, 2.0) == 1.0
    phi = 5.0
    assert orc.chi(2.5, 2.5) == pytest.approx(2.0 / (phi - 2.0 + np.sqrt(phi * phi - 4 * phi)))


def test_init_ranges(orc):
    P, D = 64, 7
    xmin = np.linspace(1000, 2000, D)
    xmax = xmin + np.linspace(500, 3000, D)
    s = orc.Swarm(P, D, xmin, xmax, lam=0.5, seed=99)
    assert np.all(s.x > xmin) and np.all(s.x < xmax)
    vmax = 0.5 * (xmax - xmin)
    assert np.all(np.abs(s.v) < vmax)
    assert np.array_equal(s.p, s.x)
    assert np.all(np.isinf(s.pf)) and s.g == 0 and s.k == 0
    ux = (s.x - xmin) / (xmax - xmin)
    uv = (s.v / vmax + 1) / 2
    assert stats.kstest(ux.ravel(), "uniform").pvalue > 1e-3
    assert stats.kstest(uv.ravel(), "uniform").pvalue > 1e-3


def _state(P, D, rng):
    x = rng.uniform(-3, 3, (P, D))
    v = rng.uniform(-1, 1, (P, D))
    p = x + rng.uniform(-1, 1, (P, D))
    pf = rng.uniform(1, 10, P)
    return x, v, p, pf


def test_bests_and_em_set(orc):
    P, D, NM = 16, 5, 4
    rng = np.random.default_rng(5)
    s = orc.Swarm(P, D, -10.0, 10.0, em_start=1, nm_frac=0.25, seed=3)
    x, v, p, pf = _state(P, D, rng)
    pf[3] = 0.5
    f = rng.uniform(0, 12, P)
    f[7] = 0.5        # ties with pf[3]: g stays on the lower index 3... unless 7 improves pf[7]
    f[9] = np.nan     # non-finite counts as +inf
    f[10] = 11.0
    f[12] = 11.0      # equal worst keys: stable order keeps 10 before 12
    s.set_state(x, v, p, pf, 0, 4)
    s.step(f)
    assert s.k == 5 and s.em_ran
    fe = np.where(np.isfinite(f), f, np.inf)
    improved = fe < pf
    pf_new = np.where(improved, fe, pf)
    assert np.array_equal(s.pf, pf_new)
    assert np.array_equal(s.p[improved], x[improved])
    assert np.array_equal(s.p[~improved], p[~improved])
    assert s.g == int(np.argmin(pf_new))          # numpy returns the first minimum
    order = np.argsort(fe, kind="stable")
    assert np.array_equal(s.order, order)
    mutated = set(order[P - NM:].tolist())
    gpos = s.p[s.g]
    for i in range(P):
        if i in mutated:
            assert np.array_equal(s.v[i], v[i])   # velocities unchanged
            same = s.x[i] == gpos
            diff = ~same
            assert np.all(np.abs(s.x[i][diff] - gpos[diff]) > 0)
        else:
            assert not np.array_equal(s.v[i], v[i])


def test_eq1_eq2_against_drawn_uniforms(orc):
    P, D = 8, 6
    rng = np.random.default_rng(6)
    c1, c2, lam, seed = 1.2, 2.9, 0.5, 777
    s = orc.Swarm(P, D, -10.0, 10.0, c1=c1, c2=c2, lam=lam, em_enabled=False, seed=seed)
    x, v, p, pf = _state(P, D, rng)
    f = rng.uniform(0, 12, P)
    s.set_state(x, v, p, pf, 0, 0)
    s.step(f)
    chi = orc.chi(c1, c2)
    g = s.p[s.g]
    k = s.k
    for i in range(P):
        for d in range(D):
            u1 = orc.uniform(seed, k, i, d, orc.U1)
            u2 = orc.uniform(seed, k, i, d, orc.U2)
            vn = chi * (v[i, d] + c1 * u1 * (s.p[i, d] - x[i, d]) + c2 * u2 * (g[d] - x[i, d]))
            vn = np.clip(vn, -lam * 20.0, lam * 20.0)
            assert s.v[i, d] == pytest.approx(vn, rel=1e-14, abs=1e-14)
            assert s.x[i, d] == pytest.approx(np.clip(x[i, d] + vn, -10, 10), rel=1e-14, abs=1e-14)


def test_box_constraint_and_velocity_clamp(orc):
    P, D = 32, 4
    s = orc.Swarm(P, D, 0.0, 1.0, lam=0.2, em_start=2, seed=4)
    rng = np.random.default_rng(0)
    for _ in range(30):
        s.step(rng.uniform(0, 1, P))
        assert np.all(s.x >= 0.0) and np.all(s.x <= 1.0)
        assert np.all(np.abs(s.v) <= 0.2 + 1e-15)


def test_mutation_statistics(orc):
    # many mutated coordinates: a fraction p_em moves by 0.1 VR N(0,1), the
    # rest sit exactly on the global best
    P, D = 200, 50
    s = orc.Swarm(P, D, -1e3, 1e3, em_start=1, nm_frac=0.5, p_em=0.3, seed=21)
    x = np.zeros((P, D))
    s.set_state(x, np.zeros((P, D)), x, np.full(P, np.inf), 0, 0)
    f = np.arange(P, dtype=float)
    s.step(f)
    mut = s.x[P // 2:]
    g = s.p[s.g]
    moved = mut != g
    frac = moved.mean()
    assert abs(frac - 0.3) < 0.02
    z = (mut[moved] - np.broadcast_to(g, mut.shape)[moved]) / (0.1 * 2e3)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_no_em_before_start(orc):
    P, D = 20, 3
    s = orc.Swarm(P, D, -5, 5, em_start=10, seed=1)
    rng = np.random.default_rng(2)
    for gen in range(1, 12):
        s.step(rng.uniform(0, 1, P))
        assert s.em_ran == (gen >= 10)


def _run(orc, fn, P, D, lo, hi, gens, seed, em=True):
    s = orc.Swarm(P, D, lo, hi, em_enabled=em, em_start=max(1, gens // 10), seed=seed)
    for _ in range(gens):
        s.step(fn(s.x))
    f = fn(s.x)
    s.step(f)
    return float(np.min(s.pf))


def _sphere(x):
    return np.sum(x * x, axis=1)


def _rastrigin(x):
    return 10.0 * x.shape[1] + np.sum(x * x - 10.0 * np.cos(2 * np.pi * x), axis=1)


def test_sphere_minimum_reached(orc):
    assert _run(orc, _sphere, 32, 10, -5.12, 5.12, 300, 12795) < 1e-7


def test_rastrigin_minimum_reached(orc):
    best = [_run(orc, _rastrigin, 40, 2, -5.12, 5.12, 200, seed) for seed in range(5)]
    assert max(best) < 1e-8, best


def test_empso_beats_pso_on_rastrigin(orc):
    # the paper's comparison ("Results"): EMPSO reaches better fitness than the
    # standard PSO and does not stagnate; on 6-D Rastrigin the standard PSO
    # sticks in local minima (integer-like values ~1-3) while EMPSO finds 0
    em = [_run(orc, _rastrigin, 40, 6, -5.12, 5.12, 300, s) for s in range(6)]
    pso = [_run(orc, _rastrigin, 40, 6, -5.12, 5.12, 300, s, em=False) for s in range(6)]
    assert np.median(em) < 1e-4
    assert np.median(pso) > 0.5


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    out = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("="))
            out[k] = float(v)
    return out


def test_paper_run_counts(orc):
    # the paper's run: 360 particles x 100 iterations = 36,000 evaluations,
    # NM = 25 % of the swarm mutated from the 10th iteration on
    gd = _golden("empso_experiment.txt")
    P, G = int(gd["particles"]), int(gd["iterations"])
    s = orc.Swarm(P, 3, -1.0, 1.0, c1=gd["c1"], c2=gd["c2"], p_em=gd["p_em"],
                  nm_frac=gd["nm_percent"] / 100.0, em_start=int(gd["em_first_iteration"]),
                  seed=1)
    evals, em_gens, mutated = 0, 0, set()
    rng = np.random.default_rng(0)
    for gen in range(1, G + 1):
        f = rng.uniform(0, 1, P)
        evals += P
        x_before, v_before = s.x.copy(), s.v.copy()
        s.step(f)
        if s.em_ran:
            em_gens += 1
            mut = np.where(np.all(s.v == v_before, axis=1))[0]
            assert len(mut) == int(0.25 * P)
            assert set(mut.tolist()) == set(np.argsort(f, kind="stable")[P - len(mut):].tolist())
    assert evals == int(gd["model_evaluations"])
    assert em_gens == G - int(gd["em_first_iteration"]) + 1


def test_rank_keys_drive_em_only(orc):
    # surrogate pre-screen: unevaluated particles have +inf fitness (no best
    # update) and their predicted misfit as EM sort key
    P, D = 12, 4
    rng = np.random.default_rng(9)
    s = orc.Swarm(P, D, -5.0, 5.0, em_start=1, nm_frac=0.25, seed=8)
    x, v, p, pf = _state(P, D, rng)
    s.set_state(x, v, p, pf, int(np.argmin(pf)), 3)
    f = np.full(P, np.inf)
    ev = np.array([0, 3, 7])
    f[ev] = rng.uniform(0.5, 2.0, 3)
    rank = rng.uniform(0, 10, P)
    rank[ev] = f[ev]
    s.step(f, rank)
    improved = f < pf
    assert np.array_equal(s.pf, np.where(improved, f, pf))
    assert np.array_equal(s.order, np.argsort(rank, kind="stable"))
    mutated = set(np.argsort(rank, kind="stable")[P - 3:].tolist())
    for i in range(P):
        assert np.array_equal(s.v[i], v[i]) == (i in mutated)
