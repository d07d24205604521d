"""Pins for the oracle's spatial operator, time axis and wavelet.

Each check ties the oracle to mathematics that does not come from the oracle
itself: exact differentiation of polynomials, the measured order of accuracy,
the closed-form eigenvalue of the checkerboard mode, stability at the CFL
limit, and the closed-form spectrum of the Ricker wavelet.
"""
import numpy as np
import pytest


@pytest.mark.parametrize("order", [2, 4, 8, 16])
def test_laplacian_exact_on_polynomials(orc, order):
    # a centred stencil of accuracy order 2R differentiates x^k exactly for
    # k <= 2R + 1 (away from the zero-padded edge); exactness up to degree 2R
    # alone fixes the R + 1 symmetric weights, so this pins the table
    R = order // 2
    NX, NZ, hx, hz = 40, 30, 7.0, 3.0
    # order 16: a centred domain keeps x^18 small enough for round-off to
    # stay far below its (constant) truncation error
    xc, zc = (20.3, 15.2) if order == 16 else (11.3, 5.2)
    x = (np.arange(NX) - xc) * hx
    z = (np.arange(NZ) - zc) * hz
    X, Z = np.meshgrid(x, z)
    for k in range(0, order + 2):
        u = (X / 50.0) ** k + 0.5 * (Z / 20.0) ** k
        exact = (k * (k - 1) * (X / 50.0) ** max(k - 2, 0) / 50.0 ** 2
                 + 0.5 * k * (k - 1) * (Z / 20.0) ** max(k - 2, 0) / 20.0 ** 2)
        got = orc.laplacian(u, hx, hz, order)
        inner = (slice(R, NZ - R), slice(R, NX - R))
        scale = np.max(np.abs(u[inner])) / min(hx, hz) ** 2 + 1e-300
        assert np.max(np.abs(got[inner] - exact[inner])) < 1e-10 * scale, k
    # degree 2R + 2 is not exact: the leading truncation term, proportional to
    # the (2R+2)-th derivative, is a non-zero constant
    k = order + 2
    u = (X / 50.0) ** k
    exact = k * (k - 1) * (X / 50.0) ** (k - 2) / 50.0 ** 2
    got = orc.laplacian(u, hx, hz, order)
    inner = (slice(R, NZ - R), slice(R, NX - R))
    err = np.abs(got[inner] - exact[inner])
    assert err.min() > 0.9 * err.max() > 0.0


@pytest.mark.parametrize("order", [2, 4, 8, 16])
def test_laplacian_convergence_order(orc, order):
    errs = []
    # coarse enough that round-off (~1e-16 / h^2) stays far below the error
    if order == 16:
        # wavenumbers 1.0 / 0.8 at h = 1 and 1/2: the error still falls by
        # 2^15.4 (terms beyond h^16 are not negligible at kh = 1), a stencil
        # one order lower would give 2^14 at most
        a, b, ns, span = 1.0, 0.8, (1, 2), 40
    else:
        a, b, ns, span = 2.1, 1.7, ((12, 24) if order == 8 else (24, 48)), 1
    for n in ns:
        h = 1.0 / n
        x = np.arange(-8, span * n + 8) * h
        X, Z = np.meshgrid(x, x)
        u = np.sin(a * X + 0.3) * np.cos(b * Z - 0.2)
        exact = -(a ** 2 + b ** 2) * u
        got = orc.laplacian(u, h, h, order)
        inner = (slice(8, -8), slice(8, -8))
        errs.append(np.max(np.abs(got[inner] - exact[inner])))
    rate = np.log2(errs[0] / errs[1])
    if order == 16:
        assert 15.0 < rate < 16.5, (errs, rate)
    else:
        assert abs(rate - order) < 0.3, (errs, rate)


@pytest.mark.parametrize("order", [2, 4, 8, 16])
def test_checkerboard_eigenvalue_sets_cfl(orc, order):
    # the checkerboard (-1)^(I+J) is the stencil's extreme mode: the Laplacian
    # scales it by -rho (1/hx^2 + 1/hz^2) with rho = |sum of signed weights|
    NX, NZ, hx, hz = 30, 24, 10.0, 25.0
    I, J = np.meshgrid(np.arange(NX), np.arange(NZ))
    u = (-1.0) ** (I + J)
    lap = orc.laplacian(u, hx, hz, order)
    R = order // 2
    ratio = lap[R:-R, R:-R] / u[R:-R, R:-R]
    lam = -ratio.mean()
    rho = lam / (1 / hx ** 2 + 1 / hz ** 2)
    # closed forms of the extreme eigenvalue: 4, 16/3, 6.5015873... (sum of |c_m| pattern)
    expect = {2: 4.0, 4: 16.0 / 3.0, 8: 2.0 * (205 / 144 + 8 / 5 + 1 / 5 + 8 / 315 + 1 / 560),
              16: 2.0 * (1077749 / 705600 + 16 / 9 + 14 / 45 + 112 / 1485 + 7 / 396
                         + 112 / 32175 + 2 / 3861 + 16 / 315315 + 1 / 411840)}[order]
    assert np.allclose(ratio, ratio.mean(), rtol=1e-12)
    assert rho == pytest.approx(expect, rel=1e-12)
    vmax, T = 3000.0, 0.2
    dt, nt = orc.time_axis(order, hx, hz, vmax, T, cfl=1.0)
    dtmax = 2.0 / (vmax * np.sqrt(lam))
    assert T / (nt - 1) == pytest.approx(dt)
    assert dt <= dtmax * (1 + 1e-12)
    assert (nt - 2) * dtmax < T + 1e-12


def _grow(orc, order, dt_factor, steps=400):
    NX = NZ = 32
    hx = hz = 10.0
    vmax = 3000.0
    dt, _ = orc.time_axis(order, hx, hz, vmax, 1.0, cfl=1.0)
    dt *= dt_factor
    rng = np.random.default_rng(0)
    um = rng.standard_normal((NZ, NX))
    u0 = um.copy()
    vel = np.full((NZ, NX), vmax)
    z = np.zeros(NX)
    for _ in range(steps):
        u1 = orc.step(um, u0, vel, z, np.zeros(NZ), None, hx, hz, order, dt)
        um, u0 = u0, u1
    return np.max(np.abs(u0))


@pytest.mark.parametrize("order", [4, 8, 16])
def test_cfl_limit_is_sharp(orc, order):
    assert _grow(orc, order, 0.9) < 50.0
    assert _grow(orc, order, 1.03) > 1e6


def test_ricker_closed_form(orc):
    f0 = 10.0
    dt = 1e-4
    t = np.arange(0, 2.0, dt)
    r = orc.ricker(f0, t)
    # peak of 1 at the delay 1/f0
    assert r.max() == pytest.approx(1.0, abs=1e-12)
    assert t[np.argmax(r)] == pytest.approx(1.0 / f0, abs=dt)
    # side lobes -2 e^{-3/2} at tau = +-sqrt(3/2)/(pi f0)
    assert r.min() == pytest.approx(-2.0 * np.exp(-1.5), rel=1e-6)
    # zero mean over the whole line (the wavelet is a second derivative of a
    # Gaussian); the part before t = 0 that the source never injects is tiny
    tt = np.arange(-1.0, 2.0, dt)
    assert abs(orc.ricker(f0, tt).sum() * dt) < 1e-9
    assert abs(r.sum() * dt) < 1e-5
    # continuous Fourier transform |R(f)| = (2 / sqrt(pi)) f^2 / f0^3 exp(-f^2 / f0^2),
    # peaking at f0 (evaluated over the whole line)
    spec = np.abs(np.fft.rfft(orc.ricker(f0, tt), n=1 << 18)) * dt
    freqs = np.fft.rfftfreq(1 << 18, dt)
    assert freqs[np.argmax(spec)] == pytest.approx(f0, rel=5e-3)
    sel = (freqs > 0.5) & (freqs < 40)
    model = 2.0 / np.sqrt(np.pi) * freqs[sel] ** 2 / f0 ** 3 * np.exp(-freqs[sel] ** 2 / f0 ** 2)
    assert np.allclose(spec[sel], model, rtol=1e-9)


def test_damping_profile_shape(orc):
    n, pad, h, vmax = 50, 20, 10.0, 3000.0
    eta = orc.damping_profile(n, pad, h, vmax)
    assert eta.shape == (n + 2 * pad,)
    assert np.all(eta[pad:pad + n] == 0.0)
    # symmetric, strictly increasing outward, quadratic in the depth d into the layer
    assert np.allclose(eta[:pad], eta[::-1][:pad])
    assert np.all(np.diff(eta[:pad + 1]) < 0)
    d = (pad - np.arange(pad)) * h
    q = eta[:pad] / d ** 2
    assert np.allclose(q, q[0], rtol=1e-12)
    # theoretical reflection exp(-(2/v) int_0^L eta dd) = 1e-3 at normal incidence
    L = pad * h
    integral = q[0] * L ** 3 / 3.0
    assert np.exp(-2.0 * integral / vmax) == pytest.approx(1e-3, rel=1e-9)
    assert np.all(orc.damping_profile(n, 0, h, vmax) == 0.0)
