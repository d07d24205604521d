"""Pins for the oracle's time stepping, source/receiver handling and misfit.

* the closed-form 2-D Green's function of the wave equation convolved with the
  Ricker wavelet, with the error shrinking at 2nd order under dt refinement;
* exact conservation of the discrete energy with rigid edges and no damping,
  and its monotone decay with damping;
* source-receiver reciprocity (bilinear injection is the transpose of bilinear
  sampling) in a heterogeneous, damped model;
* a damping layer that removes most of the boundary reflection;
* the L2 misfit on hand-computed cases.
"""
import numpy as np
import pytest
from scipy.integrate import quad

from paper_1905_12795_gb300 import synth


def _green_trace(orc, v, f0, rho, ts):
    """u(rho, t) for u_tt = v^2 (lap u + delta(x) r(t)) in 2-D:
    u = (v / 2 pi) int_0^{t - rho/v} r(tau) / sqrt(v^2 (t - tau)^2 - rho^2) dtau,
    with t - tau = rho / v + s^2 removing the inverse-square-root singularity."""
    out = np.zeros(len(ts))
    for n, t in enumerate(ts):
        if t <= rho / v:
            continue
        S = np.sqrt(t - rho / v)

        def f(s):
            return 2.0 * orc.ricker(f0, t - rho / v - s * s)[0] / np.sqrt(v * (2 * rho + v * s * s))
        out[n] = v / (2 * np.pi) * quad(f, 0.0, S, limit=200)[0]
    return out


def test_green_function_and_time_order(orc):
    v, f0, h, n, T = 2000.0, 10.0, 10.0, 201, 0.5
    src, rec = (1000.0, 1000.0), (1200.0, 1000.0)
    errs = []
    base = orc.Grid(n, n, h, h, 0, 8, T, f0, v)
    for fac in (1, 2, 4):
        g = orc.Grid(n, n, h, h, 0, 8, T, f0, v, dt=base.dt / fac, nt=(base.nt - 1) * fac + 1)
        _, tr = orc.shot_batch(g, np.full((n, n), v), [src], [rec], [0], [1], want_traces=True)
        ts = (np.arange(g.nt) + 1) * g.dt        # trace sample n is the field at t_{n+1}
        ref = _green_trace(orc, v, f0, 200.0, ts)
        errs.append(np.linalg.norm(tr[0][:, 0] - ref) / np.linalg.norm(ref))
    assert errs[-1] < 1e-3
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.15), (errs, rates)


def _energy(orc, um, u0, vel, hx, hz, order, dt):
    # E^{n+1/2} = sum (1/v^2) ((u^{n+1} - u^n)/dt)^2 + sum u^{n+1} (-lap_h u^n)
    kin = np.sum((u0 - um) ** 2 / (vel ** 2 * dt * dt))
    pot = np.sum(u0 * -orc.laplacian(um, hx, hz, order))
    return kin + pot


@pytest.mark.parametrize("order", [2, 4, 8, 16])
def test_energy_conserved_without_damping(orc, order):
    NX, NZ, hx, hz = 48, 40, 10.0, 12.0
    vel = synth.layered_faulted_model(NX, NZ, hx, hz, seed=3, vmin=1500.0, vmax=3000.0)
    dt, _ = orc.time_axis(order, hx, hz, 3000.0, 1.0)
    I, J = np.meshgrid(np.arange(NX), np.arange(NZ))
    u0 = np.exp(-((I - 20.3) ** 2 + (J - 17.1) ** 2) / 8.0)
    um = u0.copy()
    zx, zz = np.zeros(NX), np.zeros(NZ)
    E = []
    for _ in range(300):
        u1 = orc.step(um, u0, vel, zx, zz, None, hx, hz, order, dt)
        um, u0 = u0, u1
        E.append(_energy(orc, um, u0, vel, hx, hz, order, dt))
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) < 1e-11 * abs(E[0])


def test_energy_decays_with_damping(orc):
    NX, NZ, hx, hz, pad = 60, 50, 10.0, 10.0, 12
    order = 8
    vel = np.full((NZ, NX), 2500.0)
    dt, _ = orc.time_axis(order, hx, hz, 2500.0, 1.0)
    etax = orc.damping_profile(NX - 2 * pad, pad, hx, 2500.0)
    etaz = orc.damping_profile(NZ - 2 * pad, pad, hz, 2500.0)
    I, J = np.meshgrid(np.arange(NX), np.arange(NZ))
    u0 = np.exp(-((I - 30.0) ** 2 + (J - 25.0) ** 2) / 6.0)
    um = u0.copy()
    E = []
    for _ in range(600):
        u1 = orc.step(um, u0, vel, etax, etaz, None, hx, hz, order, dt)
        um, u0 = u0, u1
        E.append(_energy(orc, um, u0, vel, hx, hz, order, dt))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * E[0])
    assert E[-1] < 1e-3 * E[0]


@pytest.mark.parametrize("order", [8, 16])
def test_reciprocity_heterogeneous_damped(orc, order):
    nx, nz, h = 90, 60, 10.0
    vel = synth.layered_faulted_model(nx, nz, h, h, seed=11, vmin=1500.0, vmax=3500.0)
    g = orc.Grid(nx, nz, h, h, 15, order, 0.6, 12.0, 3500.0)
    a = (213.7, 104.2)
    b = (701.3, 377.9)
    _, ta = orc.shot_batch(g, vel, [a], [b], [0], [1], want_traces=True)
    _, tb = orc.shot_batch(g, vel, [b], [a], [0], [1], want_traces=True)
    ta, tb = ta[0][:, 0], tb[0][:, 0]
    assert np.max(np.abs(ta)) > 1e-3
    assert np.max(np.abs(ta - tb)) < 1e-10 * np.max(np.abs(ta))


def test_damping_layer_absorbs(orc):
    # a shot near the right edge of a small grid, compared with the same
    # receivers on a grid large enough that no reflection returns in time
    v, h, f0, T = 2000.0, 10.0, 15.0, 0.6
    small = (81, 61)
    big = (401, 361)
    recs = np.array([[600.0 + 10 * k, 300.0] for k in range(10)])
    src = (700.0, 300.0)
    off = (160.0, 150.0)  # place the small domain inside the big one
    out = {}
    for name, (nx, nz), pad, shift in (("rigid", small, 0, (0, 0)),
                                       ("damped", small, 30, (0, 0)),
                                       ("ref", big, 0, off)):
        g = orc.Grid(nx, nz, h, h, pad, 8, T, f0, v)
        s = (src[0] + shift[0] * h, src[1] + shift[1] * h)
        r = recs + np.array([shift[0] * h, shift[1] * h])
        _, tr = orc.shot_batch(g, np.full((nz, nx), v), [s], r, [0], [len(r)], want_traces=True)
        out[name] = tr[0]
    ref = out["ref"]
    err_rigid = np.linalg.norm(out["rigid"] - ref) / np.linalg.norm(ref)
    err_damped = np.linalg.norm(out["damped"] - ref) / np.linalg.norm(ref)
    assert err_rigid > 0.5
    assert err_damped < 0.05


def test_misfit_hand_cases(orc):
    d = np.array([[1.0, 2.0], [3.0, -1.0]])
    assert orc.misfit(d, d) == 0.0
    assert orc.misfit(d, np.zeros_like(d)) == pytest.approx(0.5 * (1 + 4 + 9 + 1))
    # phi is what the shot routine accumulates against observed data
    g = orc.Grid(41, 31, 10.0, 10.0, 5, 4, 0.2, 15.0, 2000.0)
    vel = np.full((31, 41), 1800.0)
    _, tr = orc.shot_batch(g, vel, [(200.0, 50.0)], [(100.0, 40.0), (300.0, 40.0)], [0], [2],
                           want_traces=True)
    dobs = tr[0] * 1.1 + 0.01
    phi, _ = orc.shot_batch(g, vel, [(200.0, 50.0)], [(100.0, 40.0), (300.0, 40.0)], [0], [2],
                            dobs=[dobs])
    assert phi[0, 0] == pytest.approx(orc.misfit(tr[0], dobs), rel=1e-12)
