"""The reference of the GPU gradient test is a central difference of the
FP64 oracle misfit, (phi(v + eps d) - phi(v - eps d)) / (2 eps).  These
checks fix that reference itself against properties of a derivative:
- its error shrinks at second order in eps (Richardson);
- at the step sizes the GPU test uses (1 m/s for a dense direction, 5 m/s
  for a single node) its truncation error takes at most a quarter of that
  test's tolerance (2e-3 and 1e-2 relative);
- it is linear in the direction.
"""
import numpy as np
import pytest

import oracle
from paper_1905_12795_gb300 import synth


def _problem(order=8):
    nx, nz, h, pad, T, f0, vmax = 41, 31, 10.0, 8, 0.25, 15.0, 3000.0
    og = oracle.Grid(nx, nz, h, h, pad, order, T, f0, vmax)
    v = synth.layered_faulted_model(nx, nz, h, h, seed=5, vmin=1500.0, vmax=2800.0)
    v_true = synth.layered_faulted_model(nx, nz, h, h, seed=6, vmin=1500.0, vmax=2800.0)
    shots = np.array([[105.0, 23.0], [297.0, 41.0]])
    rec = synth.receiver_line(nx, h, 27.0)[:-1] + np.array([3.7, 0.0])
    rb, rc = [0, 0], [len(rec)] * 2
    w = [1.0, 0.5]
    _, obs = oracle.shot_batch(og, v_true, shots, rec, rb, rc, want_traces=True)

    def phi(vel):
        p, _ = oracle.shot_batch(og, vel, shots, rec, rb, rc, dobs=obs)
        return float(np.dot(w, p[0]))

    return v, phi


def _fd(phi, v, d, eps):
    return (phi(v + eps * d) - phi(v - eps * d)) / (2 * eps)


@pytest.mark.parametrize("kind, eps_used, gpu_tol", [("dense", 1.0, 2e-3), ("node", 5.0, 1e-2)])
def test_central_difference_converges_at_second_order(kind, eps_used, gpu_tol):
    v, phi = _problem()
    if kind == "dense":
        d = np.random.default_rng(8).normal(size=v.shape)
    else:
        d = np.zeros_like(v)
        d[4, 14] = 1.0
    e = [4 * eps_used, 2 * eps_used, eps_used]
    f = [_fd(phi, v, d, x) for x in e]
    # Richardson: f(eps) = f' + c eps^2 + O(eps^4)
    exact = f[2] + (f[2] - f[1]) / 3.0
    d1, d2 = abs(f[0] - f[1]), abs(f[1] - f[2])
    assert d2 > 0.0
    assert 2.5 < d1 / d2 < 6.0, (d1, d2)              # ratio 4 at second order
    assert abs(f[2] - exact) <= 0.25 * gpu_tol * abs(exact), (f, exact)


def test_central_difference_is_linear_in_the_direction():
    v, phi = _problem(order=4)
    rng = np.random.default_rng(3)
    d1, d2 = rng.normal(size=v.shape), rng.normal(size=v.shape)
    a = _fd(phi, v, d1, 1.0)
    b = _fd(phi, v, d2, 1.0)
    c = _fd(phi, v, d1 + 2.0 * d2, 1.0)
    assert abs(c - (a + 2.0 * b)) <= 1e-4 * (abs(a) + 2.0 * abs(b))
