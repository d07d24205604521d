"""GPU parity of the modelling path against the FP64 CPU oracle.

Bar (from the method's accuracy target): traces within 1e-4 relative L2 of the
oracle; misfits within 1e-4 relative when the residual is at least 10 % of the
observed data, else within the error that traces at 1e-4 can put on them
(misfit_rule.py).  All inputs are seeded and
synthetic (layered/faulted or two-layer models, shots and receivers on a line).
"""
import numpy as np
import pytest

import oracle
from misfit_rule import misfit_bound, misfit_ok
from paper_1905_12795_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4
MISFIT_TOL = 1e-4


@pytest.fixture(scope="module")
def B():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_12795_gb300 import binding
    binding.load()
    return binding


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _check_misfit(got, ref, dobs_energy):
    for g, r, e in zip(np.atleast_1d(got), np.atleast_1d(ref), np.atleast_1d(dobs_energy)):
        assert misfit_ok(g, r, e), (g, r, e, misfit_bound(r, e))


def _geometry(nx, nz, h, S, src_z, rec_z, off_grid=False):
    Lx = (nx - 1) * h
    shots = synth.shot_line(S, Lx, src_z)
    rec = synth.receiver_line(nx, h, rec_z)
    if off_grid:
        rec = rec[:-1] + np.array([0.37 * h, 0.0])
        shots = shots + np.array([0.21 * h, 0.43 * h])
    return shots, rec


KINDS = [1, 2, 3]   # streaming, on-chip cluster and L2 cluster variants of the persistent launch


def _use(ctx, kind):
    ctx.set_kernel(kind)


def _ran(ctx, kind):
    assert ctx.last_launch()[0] == kind


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("order,nx,nz,pad,h", [
    (2, 37, 29, 7, 10.0),    # ragged: NX = 51, not a multiple of 4
    (4, 61, 45, 10, 12.5),
    (8, 70, 33, 9, 15.0),
    (8, 23, 19, 0, 10.0),    # no damping layer, rigid edges
])
def test_traces_match_oracle(B, kind, order, nx, nz, pad, h):
    vmax = 3200.0
    og = oracle.Grid(nx, nz, h, h, pad, order, 0.3, 12.0, vmax)
    vel = synth.layered_faulted_model(nx, nz, h, h, seed=order + nx, vmin=1500.0, vmax=vmax)
    shots, rec = _geometry(nx, nz, h, 3, 2.5 * h, 1.5 * h, off_grid=True)
    nrec = len(rec)
    _, ref = oracle.shot_batch(og, vel, shots, rec, [0] * 3, [nrec] * 3, want_traces=True)
    grid = B.make_grid(nx, nz, h, h, pad, order, 0.3, 12.0, 1500.0, vmax)
    ctx = B.Context([grid], rec)
    _use(ctx, kind)
    dt, nt = ctx.grid_info(0)
    assert nt == og.nt and dt == pytest.approx(og.dt, rel=1e-6)
    out = torch.zeros(3 * og.nt * nrec, device="cuda")
    ctx.forward_traces(_dev(vel[None]), B.make_shots(shots, [0] * 3, [nrec] * 3), out)
    _ran(ctx, kind)
    got = out.cpu().numpy().reshape(3, og.nt, nrec)
    for s in range(3):
        assert _rel_l2(got[s], ref[s]) < TRACE_TOL, (s, _rel_l2(got[s], ref[s]))
    ctx.close()


@pytest.mark.parametrize("rows", [4, 6, 8, 9, 11, 13])
@pytest.mark.parametrize("order,nx,nz,pad,h,C", [
    (8, 70, 61, 9, 15.0, 3),     # 79 rows on 3 CTAs: runs of unequal length
    (4, 61, 45, 10, 12.5, 5),    # 13 rows per CTA, a short last CTA
    (2, 37, 29, 7, 10.0, 2),
])
def test_on_chip_row_shapes_match_oracle(B, rows, order, nx, nz, pad, h, C):
    """Run lengths of both instantiations of the on-chip kernel against the
    oracle, with the source and receivers off the grid nodes."""
    vmax = 3200.0
    og = oracle.Grid(nx, nz, h, h, pad, order, 0.3, 12.0, vmax)
    vel = synth.layered_faulted_model(nx, nz, h, h, seed=order + nx, vmin=1500.0, vmax=vmax)
    shots, rec = _geometry(nx, nz, h, 3, 2.5 * h, 1.5 * h, off_grid=True)
    nrec = len(rec)
    _, ref = oracle.shot_batch(og, vel, shots, rec, [0] * 3, [nrec] * 3, want_traces=True)
    ctx = B.Context([B.make_grid(nx, nz, h, h, pad, order, 0.3, 12.0, 1500.0, vmax)], rec)
    ctx.set_kernel(2)
    ctx.set_cluster(C)
    ctx.set_tile_rows(rows)
    out = torch.zeros(3 * og.nt * nrec, device="cuda")
    # a slab cut into runs hands its first and last R rows to its neighbours
    # from its first and last runs: a run length that leaves a run shorter
    # than R rows is refused
    NZ, R = nz + 2 * pad, order // 2
    rows_c = -(-NZ // C)
    short = any(-(-my // rows) > 1 and my // -(-my // rows) < R for my in (rows_c, NZ - (C - 1) * rows_c))
    if short:
        with pytest.raises(B.EmpsoError):
            ctx.forward_traces(_dev(vel[None]), B.make_shots(shots, [0] * 3, [nrec] * 3), out)
        ctx.close()
        return
    ctx.forward_traces(_dev(vel[None]), B.make_shots(shots, [0] * 3, [nrec] * 3), out)
    assert ctx.last_launch() == (2, C) and ctx.last_tile_rows() == rows
    got = out.cpu().numpy().reshape(3, og.nt, nrec)
    for s in range(3):
        assert _rel_l2(got[s], ref[s]) < TRACE_TOL, (s, _rel_l2(got[s], ref[s]))
    for bad in (3, 14):
        with pytest.raises(B.EmpsoError):
            ctx.set_tile_rows(bad)
    ctx.close()


@pytest.mark.parametrize("nx,nz,pad,h", [(70, 33, 9, 15.0), (37, 29, 12, 10.0)])
def test_order16_traces_match_oracle(B, nx, nz, pad, h):
    """Order 16 in space (the local FWI's operator) runs on the plain
    streaming kernel: traces against the oracle; the cluster kernels, which
    hold radius-4 stencils, refuse it."""
    vmax = 3200.0
    og = oracle.Grid(nx, nz, h, h, pad, 16, 0.3, 12.0, vmax)
    vel = synth.layered_faulted_model(nx, nz, h, h, seed=16 + nx, vmin=1500.0, vmax=vmax)
    shots, rec = _geometry(nx, nz, h, 3, 2.5 * h, 1.5 * h, off_grid=True)
    nrec = len(rec)
    _, ref = oracle.shot_batch(og, vel, shots, rec, [0] * 3, [nrec] * 3, want_traces=True)
    ctx = B.Context([B.make_grid(nx, nz, h, h, pad, 16, 0.3, 12.0, 1500.0, vmax)], rec)
    dt, nt = ctx.grid_info(0)
    assert nt == og.nt and dt == pytest.approx(og.dt, rel=1e-6)
    out = torch.zeros(3 * og.nt * nrec, device="cuda")
    sh = B.make_shots(shots, [0] * 3, [nrec] * 3)
    ctx.forward_traces(_dev(vel[None]), sh, out)
    assert ctx.last_launch() == (1, 1) and ctx.last_kernel_name() == "wave_kernel"
    got = out.cpu().numpy().reshape(3, og.nt, nrec)
    for s in range(3):
        assert _rel_l2(got[s], ref[s]) < TRACE_TOL, (s, _rel_l2(got[s], ref[s]))
    for kind in (2, 3):
        ctx.set_kernel(kind)
        with pytest.raises(B.EmpsoError) as e:
            ctx.forward_traces(_dev(vel[None]), sh, out)
        assert e.value.status == 6
    ctx.close()


@pytest.mark.parametrize("kind", KINDS)
def test_single_forward_two_layer(B, kind):
    """Two-layer model (1500/2500 m/s, interface at 500 m) on 101 x 101 at 10 m
    with a 20-cell damping layer, order 4, 10 Hz Ricker at (500, 20) m, 101
    receivers at 20 m, 0.5 s; observed data from the model with +5 % velocity."""
    nx = nz = 101
    h = 10.0
    og = oracle.Grid(nx, nz, h, h, 20, 4, 0.5, 10.0, 2625.0)
    true = synth.two_layer_model(nx, nz, h)
    obs_model = true * 1.05
    shots = [(500.0, 20.0)]
    rec = synth.receiver_line(nx, h, 20.0)
    _, obs = oracle.shot_batch(og, obs_model, shots, rec, [0], [nx], want_traces=True)
    phi_ref, _ = oracle.shot_batch(og, true, shots, rec, [0], [nx], dobs=obs)
    _, tr_ref = oracle.shot_batch(og, true, shots, rec, [0], [nx], want_traces=True)
    grid = B.make_grid(nx, nz, h, h, 20, 4, 0.5, 10.0, 1500.0, 2625.0)
    ctx = B.Context([grid], rec)
    _use(ctx, kind)
    sh = B.make_shots(shots, [0], [nx])
    tr = torch.zeros(og.nt * nx, device="cuda")
    ctx.forward_traces(_dev(true[None]), sh, tr)
    _ran(ctx, kind)
    assert _rel_l2(tr.cpu().numpy().reshape(og.nt, nx), tr_ref[0]) < TRACE_TOL
    mis = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.eval_models(_dev(true[None]), sh, _dev(obs[0].ravel()), mis)
    _check_misfit(mis.cpu().numpy(), phi_ref[0], 0.5 * np.sum(obs[0] ** 2))
    # model == observed model: the misfit is round-off only
    ctx.eval_models(_dev(obs_model[None]), sh, _dev(obs[0].ravel()), mis)
    assert mis.item() <= MISFIT_TOL * 0.5 * np.sum(obs[0] ** 2)
    ctx.close()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kx,kz", [(8, 4), (4, 16), (3, 21)])
def test_interp_matches_oracle(B, mode, kx, kz):
    """Both tensor-product modes against the oracle, with node rows formed in
    registers per column (kz <= 16) and per point (kz = 21)."""
    nx, nz, h = 93, 41, 20.0
    grid = B.make_grid(nx, nz, h, h, 5, 8, 0.2, 6.0, 1500.0, 4700.0, kx=kx, kz=kz, mode=mode)
    ctx = B.Context([grid], [[0.0, 0.0]])
    parts = synth.random_particles(5, kx * kz, 1000.0, 5200.0, seed=9)   # some nodes outside the clip
    out = torch.zeros(5, nz, nx, device="cuda")
    ctx.interp(0, _dev(parts), out)
    got = out.cpu().numpy()
    for p in range(5):
        ref = oracle.interp_model(parts[p].reshape(kz, kx), nz, nx, mode, 1500.0, 4700.0)
        assert np.max(np.abs(got[p] - ref) / ref) < 2e-6
    ctx.close()


def _oracle_fitness(og, parts, kz, kx, mode, vmin, vmax, shots, rec, rb, rc, dobs, weights=None):
    out = []
    for p in range(len(parts)):
        vel = oracle.interp_model(parts[p].reshape(kz, kx), og.nz, og.nx, mode, vmin, vmax)
        phi, _ = oracle.shot_batch(og, vel, shots, rec, rb, rc, dobs=dobs)
        w = np.ones(len(shots)) if weights is None else np.asarray(weights)
        out.append(float(np.sum(w * phi[0])))
    return np.array(out)


@pytest.mark.parametrize("kind", KINDS)
def test_eval_fitness_particles(B, kind):
    nx, nz, h, pad = 77, 35, 20.0, 12
    vmin, vmax = 1500.0, 4700.0
    og = oracle.Grid(nx, nz, h, h, pad, 8, 0.8, 6.0, vmax)
    true = synth.layered_faulted_model(nx, nz, h, h, seed=1905, vmin=vmin, vmax=vmax)
    shots, rec = _geometry(nx, nz, h, 4, 20.0, 20.0)
    nrec = len(rec)
    rb, rc = [0] * 4, [nrec] * 4
    _, obs = oracle.shot_batch(og, true, shots, rec, rb, rc, want_traces=True)
    parts = synth.random_particles(6, 32, vmin, vmax, seed=3)
    ref = _oracle_fitness(og, parts, 4, 8, 0, vmin, vmax, shots, rec, rb, rc, obs)
    grid = B.make_grid(nx, nz, h, h, pad, 8, 0.8, 6.0, vmin, vmax)
    ctx = B.Context([grid], rec)
    _use(ctx, kind)
    mis = torch.zeros(6, dtype=torch.float64, device="cuda")
    dobs = _dev(np.concatenate([o.ravel() for o in obs]))
    ctx.eval_fitness(_dev(parts), B.make_shots(shots, rb, rc), dobs, mis)
    _ran(ctx, kind)
    e = 0.5 * sum(np.sum(o ** 2) for o in obs)
    _check_misfit(mis.cpu().numpy(), ref, [e] * 6)
    # the same call again gives the same bits (fixed reduction order)
    mis2 = torch.zeros_like(mis)
    ctx.eval_fitness(_dev(parts), B.make_shots(shots, rb, rc), dobs, mis2)
    assert torch.equal(mis, mis2)
    ctx.close()


def _uneven_problem(B):
    """Two grid classes (coarse 40 m / 3 Hz / long record, fine 20 m / 6 Hz),
    2 shots each, 5 particles, weighted misfit sum in fixed shot order."""
    vmin, vmax = 1500.0, 4700.0
    coarse = dict(nx=39, nz=17, h=40.0, pad=6, T=1.2, f0=3.0)
    fine = dict(nx=77, nz=33, h=20.0, pad=10, T=0.9, f0=6.0)
    ogs, grids, recs, shots_all, obs_all = [], [], [], [], []
    for c in (coarse, fine):
        og = oracle.Grid(c["nx"], c["nz"], c["h"], c["h"], c["pad"], 8, c["T"], c["f0"], vmax)
        ogs.append(og)
        grids.append(B.make_grid(c["nx"], c["nz"], c["h"], c["h"], c["pad"], 8, c["T"], c["f0"],
                                 vmin, vmax))
        sh, rec = _geometry(c["nx"], c["nz"], c["h"], 2, 40.0, 40.0)
        true = synth.layered_faulted_model(c["nx"], c["nz"], c["h"], c["h"], seed=7, vmin=vmin,
                                           vmax=vmax)
        _, obs = oracle.shot_batch(og, true, sh, rec, [0, 0], [len(rec)] * 2, want_traces=True)
        recs.append(rec)
        shots_all.append(sh)
        obs_all.append(obs)
    parts = synth.random_particles(5, 32, vmin, vmax, seed=11)
    w = [0.7, 0.7, 1.3, 1.3]
    ref = np.zeros(5)
    for gi in range(2):
        nrec = len(recs[gi])
        ref += _oracle_fitness(ogs[gi], parts, 4, 8, 0, vmin, vmax, shots_all[gi], recs[gi], [0, 0],
                               [nrec] * 2, obs_all[gi], weights=w[2 * gi:2 * gi + 2])
    n0 = len(recs[0])
    sh = B.make_shots(np.concatenate(shots_all), [0, 0, n0, n0], [n0, n0, len(recs[1]), len(recs[1])],
                      grid_ids=[0, 0, 1, 1], weights=w)
    dobs = _dev(np.concatenate([o.ravel() for ob in obs_all for o in ob]))
    e = sum(wi * 0.5 * np.sum(o ** 2) for wi, o in zip(w, [o for ob in obs_all for o in ob]))
    return grids, np.concatenate(recs), sh, dobs, parts, ref, e


@pytest.mark.parametrize("kind", KINDS)
def test_uneven_batch_two_grids(B, kind):
    """One launch over instances of two grid classes."""
    grids, rec, sh, dobs, parts, ref, e = _uneven_problem(B)
    ctx = B.Context(grids, rec)
    _use(ctx, kind)
    mis = torch.zeros(5, dtype=torch.float64, device="cuda")
    ctx.eval_fitness(_dev(parts), sh, dobs, mis)
    _ran(ctx, kind)
    _check_misfit(mis.cpu().numpy(), ref, [e] * 5)
    ctx.close()


def test_uneven_batch_pairs_the_small_grid(B):
    """On a cluster of 4 CTAs the coarse grid also fits 2 CTAs without needing
    more shared memory or threads than the fine one: its instances run two per
    cluster, one on each half, in the same launch as the fine ones.  The result
    matches the oracle and the unpaired launch (3 CTAs, odd: no halves)."""
    grids, rec, sh, dobs, parts, ref, e = _uneven_problem(B)
    ctx = B.Context(grids, rec)
    ctx.set_kernel(2)
    got = {}
    for C in (4, 3):
        ctx.set_cluster(C)
        mis = torch.zeros(5, dtype=torch.float64, device="cuda")
        ctx.eval_fitness(_dev(parts), sh, dobs, mis)
        assert ctx.last_launch() == (2, C)
        got[C] = mis.cpu().numpy()
        _check_misfit(got[C], ref, [e] * 5)
    ctx.set_cluster(4)
    ctx.eval_fitness(_dev(parts), sh, dobs, mis)
    assert ctx.last_paired_units() == 5          # 10 coarse instances in 5 pairs
    ctx.set_cluster(3)
    ctx.eval_fitness(_dev(parts), sh, dobs, mis)
    assert ctx.last_paired_units() == 0
    assert np.allclose(got[4], got[3], rtol=1e-5)
    ctx.close()


def test_uneven_batch_every_cluster_size(B):
    """Every cluster size that holds both grids of the uneven batch: the
    coarse grid's instances run shorter runs than the launch's (more runs per
    column, sized by the fine grid's threads) wherever the planner finds such
    runs; the misfits match the oracle at each size."""
    grids, rec, sh, dobs, parts, ref, e = _uneven_problem(B)
    ctx = B.Context(grids, rec)
    ctx.set_kernel(2)
    ran = 0
    for C in range(2, 8):
        ctx.set_cluster(C)
        mis = torch.zeros(5, dtype=torch.float64, device="cuda")
        try:
            ctx.eval_fitness(_dev(parts), sh, dobs, mis)
        except B.EmpsoError:
            continue                      # this size does not hold one of the grids
        assert ctx.last_launch() == (2, C)
        _check_misfit(mis.cpu().numpy(), ref, [e] * 5)
        ran += 1
    assert ran >= 4
    ctx.close()


def test_edge_cases(B):
    nx, nz, h = 41, 31, 10.0
    grid = B.make_grid(nx, nz, h, h, 5, 4, 0.2, 10.0, 1500.0, 3000.0)
    rec = synth.receiver_line(nx, h, 0.0)
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    # zero particles: no work, no error
    ctx.eval_fitness(torch.zeros(0, 32, device="cuda"), B.make_shots([(200.0, 0.0)], [0], [nx]),
                     torch.zeros(nt * nx, device="cuda"), torch.zeros(0, dtype=torch.float64,
                                                                       device="cuda"))
    # a shot with no receivers has zero misfit; sources on the domain corners are valid
    sh = B.make_shots([(0.0, 0.0), ((nx - 1) * h, (nz - 1) * h)], [0, 0], [0, nx])
    vel = torch.full((2, nz, nx), 2000.0, device="cuda")
    og = oracle.Grid(nx, nz, h, h, 5, 4, 0.2, 10.0, 3000.0)
    _, ref = oracle.shot_batch(og, np.full((nz, nx), 2000.0), [((nx - 1) * h, (nz - 1) * h)], rec,
                               [0], [nx], want_traces=True)
    tr = torch.zeros(2 * nt * nx, device="cuda")
    ctx.forward_traces(vel, sh, tr)
    got = tr.cpu().numpy().reshape(2, nt, nx)
    assert _rel_l2(got[1], ref[0]) < TRACE_TOL and _rel_l2(got[0], ref[0]) < TRACE_TOL
    mis = torch.zeros(2, dtype=torch.float64, device="cuda")
    ctx.eval_models(vel, sh, torch.zeros(nt * nx, device="cuda"), mis)
    assert mis[0].item() == pytest.approx(0.5 * np.sum(ref[0].astype(np.float64) ** 2), rel=1e-4)
    # invalid arguments are refused before any launch
    with pytest.raises(B.EmpsoError) as e:
        ctx.forward_traces(vel, B.make_shots([(-1.0, 0.0)], [0], [nx]), tr)
    assert e.value.status == 1
    with pytest.raises(B.EmpsoError):
        ctx.forward_traces(vel, B.make_shots([(0.0, 0.0)], [5], [nx]), tr)
    with pytest.raises(B.EmpsoError) as e:
        B.Context([B.make_grid(nx, nz, h, h, 5, 6, 0.2, 10.0, 1500.0, 3000.0)], rec)
    assert e.value.status == 6
    ctx.close()


_FULL = {}


def _full_size_reference():
    """Oracle observed data and the misfits of particles 0 and P-1 for the
    plain EMPSO workload (computed once per session: 48 full-size shots)."""
    if not _FULL:
        wl = synth.workloads()["empso-461x151-P32-S16"]
        gs = wl.grids[0]
        og = oracle.Grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmax)
        S = wl.shots_per_grid[0]
        shots = synth.shot_line(S, (gs.nx - 1) * gs.hx, wl.src_z)
        rec = synth.receiver_line(gs.nx, gs.hx, wl.rec_z)
        nrec = len(rec)
        true = synth.layered_faulted_model(gs.nx, gs.nz, gs.hx, gs.hz, seed=wl.seed_model)
        _, obs = oracle.shot_batch(og, true, shots, rec, [0] * S, [nrec] * S, want_traces=True)
        parts = synth.random_particles(wl.P, gs.kx * gs.kz, wl.xmin, wl.xmax, seed=wl.seed_pso)
        sel = [0, wl.P - 1]
        ref = _oracle_fitness(og, parts[sel], gs.kz, gs.kx, 0, gs.vmin, gs.vmax, shots, rec,
                              [0] * S, [nrec] * S, obs)
        _FULL.update(wl=wl, gs=gs, og=og, S=S, shots=shots, rec=rec, obs=np.stack(obs),
                     parts=parts, sel=sel, ref=ref)
    return _FULL


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_full_size_sampled(B, kind):
    """The 461 x 151 / 20 m / order 8 / 3 s / 6 Hz grid of the plain EMPSO
    workload with 32 particles x 16 shots in one launch (the benchmarked launch
    configuration); particles 0 and 31 are recomputed by the oracle (all 16
    shots each)."""
    F = _full_size_reference()
    wl, gs, S, rec, obs = F["wl"], F["gs"], F["S"], F["rec"], F["obs"]
    nrec = len(rec)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz)
    ctx = B.Context([grid], rec)
    _use(ctx, kind)
    sh = B.make_shots(F["shots"], [0] * S, [nrec] * S)
    dobs = _dev(obs.ravel())
    mis = torch.zeros(wl.P, dtype=torch.float64, device="cuda")
    ctx.eval_fitness(_dev(F["parts"]), sh, dobs, mis)
    # the default picks the on-chip kernel for this grid
    assert ctx.last_launch()[0] == (2 if kind == 0 else kind)
    got = mis.cpu().numpy()
    e = 0.5 * np.sum(obs.astype(np.float64) ** 2)
    _check_misfit(got[F["sel"]], F["ref"], [e] * 2)
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    ctx.close()


@pytest.mark.parametrize("kind", KINDS)
def test_nonfinite_model_gives_inf_misfit(B, kind):
    """Failure handling: a model whose wavefield blows up (a NaN velocity node)
    gets misfit +inf, the other models of the launch are unaffected, and
    pso_step never takes it as a best."""
    nx, nz, h = 41, 31, 10.0
    grid = B.make_grid(nx, nz, h, h, 5, 4, 0.2, 10.0, 1500.0, 3000.0)
    rec = synth.receiver_line(nx, h, 20.0)
    pso = B.EmpsoPso(3, 32, 1.2, 2.9, 0.5, 0.3, 0.25, 10, 1, 1)
    ctx = B.Context([grid], rec, pso, 1500.0, 3000.0)
    _use(ctx, kind)
    _, nt = ctx.grid_info(0)
    sh = B.make_shots([(200.0, 20.0)], [0], [nx])
    vel = np.full((3, nz, nx), 2000.0, dtype=np.float32)
    vel[1, 10, 10] = np.nan
    dobs = torch.zeros(nt * nx, device="cuda")
    mis = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.eval_models(_dev(vel), sh, dobs, mis)
    m = mis.cpu().numpy()
    assert np.isinf(m[1]) and m[1] > 0
    assert np.isfinite(m[0]) and m[0] == m[2]
    assert ctx.nonfinite_count() == 1
    # strict mode: the call reports it, the outputs are still written
    ctx.set_strict(True)
    mis.zero_()
    with pytest.raises(B.EmpsoError) as e:
        ctx.eval_models(_dev(vel), sh, dobs, mis)
    assert e.value.status == 4
    assert np.array_equal(mis.cpu().numpy(), m)
    assert ctx.nonfinite_count(reset=True) == 2 and ctx.nonfinite_count() == 0
    ctx.eval_models(_dev(vel[[0, 2]]), sh, dobs, torch.zeros_like(mis[:2]))   # finite: no error
    ctx.set_strict(False)
    ctx.pso_init()
    ctx.pso_step(mis)
    pf = torch.zeros(3, dtype=torch.float64, device="cuda")
    gk = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.pso_get_state(pf=pf, gk=gk)
    assert np.isinf(pf.cpu().numpy()[1]) and gk.cpu().numpy()[0] == 0
    ctx.close()


def test_grid_too_large_for_chip_runs_on_l2_cluster_kernel(B):
    """The 921 x 301 / 10 m grid with a 60-cell damping layer (the
    high-resolution workload's grid, record shortened to 0.3 s for the
    oracle) does not fit the on-chip kernel: the default picks the L2 cluster
    kernel, which matches the oracle and the streaming kernel."""
    nx, nz, h, pad = 921, 301, 10.0, 60
    vmin, vmax = 1500.0, 4700.0
    og = oracle.Grid(nx, nz, h, h, pad, 8, 0.3, 12.0, vmax)
    true = synth.layered_faulted_model(nx, nz, h, h, seed=1905, vmin=vmin, vmax=vmax)
    shots = synth.shot_line(2, (nx - 1) * h, 20.0)
    rec = synth.receiver_line(nx, h, 20.0)[::2]
    nrec = len(rec)
    _, obs = oracle.shot_batch(og, true, shots, rec, [0, 0], [nrec, nrec], want_traces=True)
    parts = synth.random_particles(2, 8 * 24, vmin, vmax, seed=4)
    ref = _oracle_fitness(og, parts, 8, 24, 0, vmin, vmax, shots, rec, [0, 0], [nrec, nrec], obs)
    grid = B.make_grid(nx, nz, h, h, pad, 8, 0.3, 12.0, vmin, vmax, kx=24, kz=8)
    ctx = B.Context([grid], rec)
    sh = B.make_shots(shots, [0, 0], [nrec, nrec])
    dobs = _dev(np.concatenate([o.ravel() for o in obs]))
    e = 0.5 * sum(np.sum(o ** 2) for o in obs)
    got = {}
    for kind in (0, 1):
        ctx.set_kernel(kind)
        mis = torch.zeros(2, dtype=torch.float64, device="cuda")
        ctx.eval_fitness(_dev(parts), sh, dobs, mis)
        if kind == 0:
            assert ctx.last_launch()[0] == 3 and ctx.last_kernel_name() == "wave_l2_kernel"
        got[kind] = mis.cpu().numpy()
        _check_misfit(got[kind], ref, [e] * 2)
    assert np.allclose(got[0], got[1], rtol=1e-5)
    assert ctx.device_error() == 0
    ctx.close()


def test_every_cluster_shape_matches_oracle(B):
    """Every cluster size and run length the planner or the autotuner may pick
    for a small grid (77 x 35 + 12 cells, order 8: slabs of 4 to 59 rows, the
    last slab shorter) gives the oracle's misfits; the L2 cluster kernel's
    sizes too."""
    nx, nz, h, pad, P, S = 77, 35, 20.0, 12, 4, 2
    grid = B.make_grid(nx, nz, h, h, pad, 8, 0.8, 6.0, 1500.0, 4700.0)
    rec = synth.receiver_line(nx, h, 20.0)
    shots = synth.shot_line(S, (nx - 1) * h, 20.0)
    og = oracle.Grid(nx, nz, h, h, pad, 8, 0.8, 6.0, 4700.0)
    true = synth.layered_faulted_model(nx, nz, h, h, seed=1905)
    _, obs = oracle.shot_batch(og, true, shots, rec, [0] * S, [nx] * S, want_traces=True)
    dobs = _dev(np.concatenate([o.ravel() for o in obs]))
    x = _dev(synth.random_particles(P, 32, 1500.0, 4700.0, seed=2))
    ctx = B.Context([grid], rec)
    vel = torch.zeros(P, nz, nx, device="cuda")
    ctx.interp(0, x, vel)
    ref = np.array([oracle.shot_batch(og, vel[m].cpu().numpy().astype(np.float64), shots, rec, [0] * S,
                                      [nx] * S, dobs=obs)[0].sum() for m in range(P)])
    sh = B.make_shots(shots, [0] * S, [nx] * S)
    mis = torch.zeros(P, dtype=torch.float64, device="cuda")
    ran = 0
    cands = [(2, C, r) for C in range(1, 17) for r in (13, 11, 9, 8, 6, 4)] + \
            [(3, C, 0) for C in (1, 2, 4, 8, 10, 12, 16)]
    for kind, C, rows in cands:
        ctx.set_kernel(kind)
        ctx.set_cluster(C)
        ctx.set_tile_rows(rows)
        try:
            ctx.eval_fitness(x, sh, dobs, mis)
        except B.EmpsoError:
            continue                     # the shape does not fit this grid
        got = mis.cpu().numpy()
        assert np.all(np.abs(got / ref - 1.0) < 1e-4), (kind, C, rows, got, ref)
        ran += 1
    assert ran >= 40
    ctx.close()


def test_run_lengths_give_identical_traces(B):
    """Every run length computes every point with the same operations (the
    13-row shape carries the z-differences from row to row, which adds the
    same rounded terms in the other order), so the traces agree bit for bit
    across run lengths and across the two instantiations."""
    nx, nz, h, pad = 70, 61, 15.0, 9
    vmax = 3200.0
    grid = B.make_grid(nx, nz, h, h, pad, 8, 0.3, 12.0, 1500.0, vmax)
    vel = synth.layered_faulted_model(nx, nz, h, h, seed=78, vmin=1500.0, vmax=vmax)
    shots, rec = _geometry(nx, nz, h, 3, 2.5 * h, 1.5 * h, off_grid=True)
    nrec = len(rec)
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    ctx.set_kernel(2)
    ctx.set_cluster(3)
    outs = {}
    for rows in (13, 11, 9, 8, 6):
        ctx.set_tile_rows(rows)
        out = torch.zeros(3 * nt * nrec, device="cuda")
        ctx.forward_traces(_dev(vel[None]), B.make_shots(shots, [0] * 3, [nrec] * 3), out)
        assert ctx.last_tile_rows() == rows
        outs[rows] = out
    for rows, out in outs.items():
        assert torch.equal(out, outs[8]), rows
    ctx.close()
