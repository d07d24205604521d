"""Parity at the benchmarked sizes: element-wise traces, near-optimal misfits
and the adjoint gradient on the full grids, against the FP64 CPU oracle.

Bar (the method's accuracy target): traces within 1e-4 relative L2 of the
oracle, per shot; misfits within 1e-4 relative when the residual is at least
10 % of the observed data, else within the error that traces at 1e-4 can put
on them (misfit_rule.py).  Inputs are
seeded and synthetic: the layered/faulted model of the plain EMPSO workload
(461 x 151 at 20 m, 40 damping cells, order 8, 6 Hz, 3 s = 1414 steps, one
receiver per horizontal node at 20 m, 16 shots on a line) and of the
high-resolution workload (921 x 301 at 10 m, 60 damping cells, 12 Hz, 4 s =
3768 steps).
"""
import numpy as np
import pytest

import oracle
from misfit_rule import misfit_bound, misfit_ok
from paper_1905_12795_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4


@pytest.fixture(scope="module")
def B():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_12795_gb300 import binding
    binding.load()
    return binding


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


_PLAIN = {}


def _plain():
    """The plain EMPSO workload's grid, geometry, true model and swarm."""
    if not _PLAIN:
        wl = synth.workloads()["empso-461x151-P32-S16"]
        gs = wl.grids[0]
        og = oracle.Grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmax)
        S = wl.shots_per_grid[0]
        shots = synth.shot_line(S, (gs.nx - 1) * gs.hx, wl.src_z)
        rec = synth.receiver_line(gs.nx, gs.hx, wl.rec_z)
        true = synth.layered_faulted_model(gs.nx, gs.nz, gs.hx, gs.hz, seed=wl.seed_model)
        parts = synth.random_particles(wl.P, gs.kx * gs.kz, wl.xmin, wl.xmax, seed=wl.seed_pso)
        _PLAIN.update(wl=wl, gs=gs, og=og, S=S, shots=shots, rec=rec, true=true, parts=parts)
    return _PLAIN


def _plain_grid(B, gs):
    return B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz)


# instances (model, shot) compared element by element: both ends of the shot
# line, for the first and the last particle of the swarm
_SAMPLE = [(0, 0), (0, 15), (31, 0), (31, 15)]
_SAMPLE_REF = {}


def _sample_reference(F):
    if not _SAMPLE_REF:
        gs, og, rec = F["gs"], F["og"], F["rec"]
        nrec = len(rec)
        for m in sorted({m for m, _ in _SAMPLE}):
            vel = oracle.interp_model(F["parts"][m].reshape(gs.kz, gs.kx), gs.nz, gs.nx, 0,
                                      gs.vmin, gs.vmax)
            ss = [s for mm, s in _SAMPLE if mm == m]
            _, tr = oracle.shot_batch(og, vel, F["shots"][ss], rec, [0] * len(ss),
                                      [nrec] * len(ss), want_traces=True)
            for s, t in zip(ss, tr):
                _SAMPLE_REF[(m, s)] = t
    return _SAMPLE_REF


@pytest.mark.parametrize("kind", [2, 3, 1])   # on-chip cluster, L2 cluster, streaming
def test_full_size_traces_elementwise(B, kind):
    """The benchmarked launch (32 particles x 16 shots = 512 instances, 1414
    steps) with traces written out: four instances at both ends of the shot
    line are compared sample by sample with the oracle."""
    F = _plain()
    gs, S, rec = F["gs"], F["S"], F["rec"]
    nrec = len(rec)
    ref = _sample_reference(F)
    ctx = B.Context([_plain_grid(B, gs)], rec)
    ctx.set_kernel(kind)
    P = F["wl"].P
    vel = torch.zeros(P, gs.nz, gs.nx, device="cuda")
    ctx.interp(0, _dev(F["parts"]), vel)
    _, nt = ctx.grid_info(0)
    assert nt == F["og"].nt == 1414
    out = torch.zeros(P * S * nt * nrec, device="cuda")
    ctx.forward_traces(vel, B.make_shots(F["shots"], [0] * S, [nrec] * S), out)
    assert ctx.last_launch()[0] == kind
    if kind == 2:
        # the planner's on-chip cluster for this batch: 9 or more CTAs hold this grid
        assert ctx.last_launch()[1] >= 9 and 4 <= ctx.last_tile_rows() <= 13
    got = out.view(P, S, nt, nrec)
    errs = {}
    for (m, s) in _SAMPLE:
        errs[(m, s)] = _rel_l2(got[m, s].cpu().numpy(), ref[(m, s)])
    assert max(errs.values()) < TRACE_TOL, errs
    assert ctx.device_error() == 0
    ctx.close()


@pytest.mark.parametrize("C,rows", [(10, 8), (10, 13), (9, 13), (9, 9), (9, 11), (12, 7)])
def test_full_size_traces_on_forced_cluster_shapes(B, C, rows):
    """The same comparison with the on-chip kernel forced onto clusters of
    C CTAs and runs of at most `rows` rows per thread (the shapes the
    benchmark's autotuner chooses among for this grid)."""
    F = _plain()
    gs, S, rec = F["gs"], F["S"], F["rec"]
    nrec = len(rec)
    ref = _sample_reference(F)
    ctx = B.Context([_plain_grid(B, gs)], rec)
    ctx.set_kernel(2)
    ctx.set_cluster(C)
    ctx.set_tile_rows(rows)
    P = F["wl"].P
    vel = torch.zeros(P, gs.nz, gs.nx, device="cuda")
    ctx.interp(0, _dev(F["parts"]), vel)
    _, nt = ctx.grid_info(0)
    out = torch.zeros(P * S * nt * nrec, device="cuda")
    ctx.forward_traces(vel, B.make_shots(F["shots"], [0] * S, [nrec] * S), out)
    assert ctx.last_launch() == (2, C) and ctx.last_tile_rows() == rows
    got = out.view(P, S, nt, nrec)
    errs = {k: _rel_l2(got[k[0], k[1]].cpu().numpy(), v) for k, v in ref.items()}
    assert max(errs.values()) < TRACE_TOL, errs
    ctx.close()


def test_full_size_near_optimal_misfits(B):
    """Near the optimum the misfit is a small difference of large traces.
    The 4 x 8 control nodes are fitted to the true model (least squares
    through the spline), the observed data are the oracle's traces of the
    fitted model, and the fitted particle and three perturbations of it
    (relative node changes 3e-4, 1e-3, 1e-2: residuals about 0.4 %, 1.4 % and
    14 % of the data) are evaluated in one launch at the full size: the
    first three are held to the error that traces at 1e-4 can put on a
    misfit, the last to 1e-4 relative."""
    F = _plain()
    gs, og, S, rec = F["gs"], F["og"], F["S"], F["rec"]
    nrec = len(rec)
    Wz = oracle.interp_matrix(gs.kz, gs.nz, 0)
    Wx = oracle.interp_matrix(gs.kx, gs.nx, 0)
    C = np.clip(np.linalg.pinv(Wz) @ F["true"] @ np.linalg.pinv(Wx).T, gs.vmin, gs.vmax)
    sign = np.random.default_rng(7).choice([-1.0, 1.0], size=C.shape)
    parts = np.stack([C.ravel()] + [(C * (1.0 + d * sign)).ravel() for d in (3e-4, 1e-3, 1e-2)])
    vfit = oracle.interp_model(C, gs.nz, gs.nx, 0, gs.vmin, gs.vmax)
    _, obs = oracle.shot_batch(og, vfit, F["shots"], rec, [0] * S, [nrec] * S, want_traces=True)
    E = 0.5 * sum(float(np.sum(o ** 2)) for o in obs)
    ref = []
    for p in parts:
        v = oracle.interp_model(p.reshape(gs.kz, gs.kx), gs.nz, gs.nx, 0, gs.vmin, gs.vmax)
        phi, _ = oracle.shot_batch(og, v, F["shots"], rec, [0] * S, [nrec] * S, dobs=obs)
        ref.append(float(phi.sum()))
    ref = np.array(ref)
    assert ref[0] == 0.0
    assert ref[1] < 1e-4 * E < ref[2] < 1e-2 * E < ref[3]
    ctx = B.Context([_plain_grid(B, gs)], rec)
    dobs = _dev(np.concatenate([o.ravel() for o in obs]))
    sh = B.make_shots(F["shots"], [0] * S, [nrec] * S)
    for kind in (2, 3):
        ctx.set_kernel(kind)
        mis = torch.zeros(len(parts), dtype=torch.float64, device="cuda")
        ctx.eval_fitness(_dev(parts), sh, dobs, mis)
        got = mis.cpu().numpy()
        for g, r in zip(got, ref):
            assert misfit_ok(g, r, E), (kind, g, r, E, misfit_bound(r, E))
    ctx.close()


def test_hires_full_record_on_l2_cluster_kernel(B):
    """The high-resolution grid at its full 4 s record (3768 steps): the L2
    cluster kernel's traces at both ends of the shot line, all 921
    receivers, against the oracle sample by sample."""
    wl = synth.workloads()["hires-921x301-P512-S64"]
    gs = wl.grids[0]
    og = oracle.Grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmax)
    assert og.nt == 3768
    shots = synth.shot_line(64, (gs.nx - 1) * gs.hx, wl.src_z)[[0, 63]]
    rec = synth.receiver_line(gs.nx, gs.hx, wl.rec_z)
    nrec = len(rec)
    true = synth.layered_faulted_model(gs.nx, gs.nz, gs.hx, gs.hz, seed=wl.seed_model)
    _, ref = oracle.shot_batch(og, true, shots, rec, [0, 0], [nrec, nrec], want_traces=True)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz)
    ctx = B.Context([grid], rec)
    ctx.set_kernel(0)
    out = torch.zeros(2 * og.nt * nrec, device="cuda")
    ctx.forward_traces(_dev(true[None]), B.make_shots(shots, [0, 0], [nrec, nrec]), out)
    assert ctx.last_launch()[0] == 3 and ctx.last_kernel_name() == "wave_l2_kernel"
    got = out.cpu().numpy().reshape(2, og.nt, nrec)
    errs = [_rel_l2(got[s], ref[s]) for s in range(2)]
    assert max(errs) < TRACE_TOL, errs
    assert ctx.device_error() == 0
    ctx.close()


def _smooth_direction(nz, nx, seed):
    """A smooth dense direction: random values on a coarse grid, bilinear up."""
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(6, 12))
    zi = np.linspace(0, 5, nz)
    xi = np.linspace(0, 11, nx)
    rows = np.array([np.interp(xi, np.arange(12), c[k]) for k in range(6)])
    return np.array([np.interp(zi, np.arange(6), rows[:, i]) for i in range(nx)]).T


@pytest.mark.parametrize("kernel", [0, 3])   # forward on the on-chip / L2 cluster kernel
def test_full_size_gradient_directional_derivative(B, kernel):
    """The adjoint gradient of the plain workload's grid (1414 steps, two
    shots at the ends of the line, the forward pass on the cluster kernels
    with the history streamed out) against FP64 central differences of the
    oracle misfit along a smooth dense direction and along one node."""
    F = _plain()
    gs, og, rec = F["gs"], F["og"], F["rec"]
    nrec = len(rec)
    shots = F["shots"][[0, 15]]
    rb, rc = [0, 0], [nrec, nrec]
    v_true = F["true"]
    v = oracle.interp_model(F["parts"][3].reshape(gs.kz, gs.kx), gs.nz, gs.nx, 0, gs.vmin, gs.vmax)
    # a start between the particle and the truth keeps the residual moderate
    v = 0.5 * (v + v_true)
    _, obs = oracle.shot_batch(og, v_true, shots, rec, rb, rc, want_traces=True)

    def phi(vel):
        p, _ = oracle.shot_batch(og, vel, shots, rec, rb, rc, dobs=obs)
        return float(p.sum())

    ctx = B.Context([_plain_grid(B, gs)], rec)
    ctx.set_kernel(kernel)
    g = torch.zeros(1, gs.nz, gs.nx, device="cuda")
    mis = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.gradient(_dev(v[None]), B.make_shots(shots, rb, rc),
                 _dev(np.concatenate([o.ravel() for o in obs])), g, mis)
    G = g[0].cpu().numpy().astype(np.float64)
    assert mis.item() == pytest.approx(phi(v), rel=1e-4)
    d = _smooth_direction(gs.nz, gs.nx, 21)
    eps = 2.0
    fd = (phi(v + eps * d) - phi(v - eps * d)) / (2 * eps)
    ad = float(np.sum(G * d))
    assert abs(ad - fd) <= 2e-3 * abs(fd), (ad, fd)
    ctx.close()


def test_gradient_one_and_two_step_adjoint_kernels_agree(B):
    """20 shots of the plain grid are more tiles than two waves of the
    two-step adjoint kernel, so their backward pass runs one step per launch;
    10 shots run two steps per launch.  Both compute every instance's steps
    with the same arithmetic, so the 20-shot gradient equals the sum of the
    two 10-shot halves' to FP32 rounding (the compiler may contract the same
    expressions differently in the two kernels, and the shot sums group
    differently), and so do the misfits (the 10-shot path is pinned to the
    oracle above)."""
    F = _plain()
    gs, rec = F["gs"], F["rec"]
    nrec = len(rec)
    ctx = B.Context([_plain_grid(B, gs)], rec)
    _, nt = ctx.grid_info(0)
    xs = np.linspace(100.0, (gs.nx - 1) * gs.hx - 100.0, 20)
    shots = np.stack([xs, np.full(20, 20.0)], axis=1)
    v = _dev(F["true"][None])
    dobs = torch.zeros(20 * nt * nrec, device="cuda")
    ctx.forward_traces(v * 1.04, B.make_shots(shots, [0] * 20, [nrec] * 20), dobs)
    d = dobs.view(20, nt * nrec)

    def grad(idx):
        g = torch.zeros(1, gs.nz, gs.nx, device="cuda")
        m = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.gradient(v, B.make_shots(shots[idx], [0] * len(idx), [nrec] * len(idx)),
                     d[idx].contiguous().view(-1), g, m)
        return g[0].double(), m.item()

    g20, m20 = grad(list(range(20)))
    ga, ma = grad(list(range(10)))
    gb, mb = grad(list(range(10, 20)))
    assert float((g20 - (ga + gb)).norm() / g20.norm()) < 1e-4
    assert m20 == pytest.approx(ma + mb, rel=1e-9)
    assert ctx.device_error() == 0
    ctx.close()


def test_hires_gradient_on_l2_cluster_kernel(B):
    """The adjoint gradient on the high-resolution grid (record shortened to
    0.5 s), forward pass on the L2 cluster kernel with the history streamed
    out, against central differences of the oracle misfit."""
    wl = synth.workloads()["hires-921x301-P512-S64"]
    gs = wl.grids[0]
    T = 0.5
    og = oracle.Grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, T, gs.f0, gs.vmax)
    shots = np.array([[4600.0, 20.0]])
    rec = synth.receiver_line(gs.nx, gs.hx, wl.rec_z)
    nrec = len(rec)
    v_true = synth.layered_faulted_model(gs.nx, gs.nz, gs.hx, gs.hz, seed=wl.seed_model)
    v = 0.97 * v_true + 0.03 * 3000.0
    _, obs = oracle.shot_batch(og, v_true, shots, rec, [0], [nrec], want_traces=True)

    def phi(vel):
        p, _ = oracle.shot_batch(og, vel, shots, rec, [0], [nrec], dobs=obs)
        return float(p.sum())

    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz)
    ctx = B.Context([grid], rec)
    ctx.set_kernel(0)
    g = torch.zeros(1, gs.nz, gs.nx, device="cuda")
    mis = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.gradient(_dev(v[None]), B.make_shots(shots, [0], [nrec]),
                 _dev(obs[0].ravel()), g, mis)
    G = g[0].cpu().numpy().astype(np.float64)
    assert mis.item() == pytest.approx(phi(v), rel=1e-4)
    d = _smooth_direction(gs.nz, gs.nx, 22)
    eps = 2.0
    fd = (phi(v + eps * d) - phi(v - eps * d)) / (2 * eps)
    ad = float(np.sum(G * d))
    assert abs(ad - fd) <= 2e-3 * abs(fd), (ad, fd)
    ctx.close()
