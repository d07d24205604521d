"""Pins for the two-grid parameterisation of the oracle.

The natural cubic spline is checked against scipy's textbook implementation,
the bilinear mode against numpy.interp, and both against the defining
properties: exact reproduction of node values and of linear fields.
"""
import numpy as np
import pytest
from scipy.interpolate import CubicSpline


@pytest.mark.parametrize("K,n", [(2, 11), (4, 151), (8, 461), (24, 921), (5, 7)])
def test_spline_matrix_matches_scipy_natural(orc, K, n):
    W = orc.interp_matrix(K, n, 0)
    nodes = np.arange(K) * (n - 1) / (K - 1)
    x = np.arange(n, dtype=float)
    for k in range(K):
        e = np.zeros(K)
        e[k] = 1.0
        ref = CubicSpline(nodes, e, bc_type="natural")(x)
        assert np.allclose(W[:, k], ref, atol=1e-12)


@pytest.mark.parametrize("K,n", [(4, 151), (8, 461), (3, 10)])
def test_bilinear_matrix_matches_numpy_interp(orc, K, n):
    W = orc.interp_matrix(K, n, 1)
    nodes = np.arange(K) * (n - 1) / (K - 1)
    x = np.arange(n, dtype=float)
    rng = np.random.default_rng(1)
    y = rng.uniform(1500, 4700, K)
    assert np.allclose(W @ y, np.interp(x, nodes, y), atol=1e-9)


@pytest.mark.parametrize("mode", [0, 1])
def test_interp_model_reproduces_nodes_and_planes(orc, mode):
    Kz, Kx, nz, nx = 4, 8, 151, 421   # nodes fall on grid points: (n-1)/(K-1) is an integer
    rng = np.random.default_rng(2)
    C = rng.uniform(1500, 4700, (Kz, Kx))
    V = orc.interp_model(C, nz, nx, mode)
    jz = np.arange(Kz) * (nz - 1) // (Kz - 1)
    ix = np.arange(Kx) * (nx - 1) // (Kx - 1)
    assert np.allclose(V[np.ix_(jz, ix)], C, rtol=1e-12)
    # a bilinear plane v = a + b x + c z + d x z is reproduced exactly by both modes
    zz, xx = np.meshgrid(np.linspace(0, 1, Kz), np.linspace(0, 1, Kx), indexing="ij")
    Cp = 2000 + 800 * xx - 300 * zz + 150 * xx * zz
    Vp = orc.interp_model(Cp, nz, nx, mode)
    Z, X = np.meshgrid(np.linspace(0, 1, nz), np.linspace(0, 1, nx), indexing="ij")
    assert np.allclose(Vp, 2000 + 800 * X - 300 * Z + 150 * X * Z, rtol=1e-12)


def test_interp_model_tensor_product_and_clip(orc):
    Kz, Kx, nz, nx = 4, 8, 31, 57
    rng = np.random.default_rng(3)
    C = rng.uniform(1000, 5000, (Kz, Kx))
    V = orc.interp_model(C, nz, nx, 0)
    # brute force: spline along x for every node row, then along z for every column
    xn = np.arange(Kx) * (nx - 1) / (Kx - 1)
    zn = np.arange(Kz) * (nz - 1) / (Kz - 1)
    rows = np.stack([CubicSpline(xn, C[k], bc_type="natural")(np.arange(nx)) for k in range(Kz)])
    ref = np.stack([CubicSpline(zn, rows[:, i], bc_type="natural")(np.arange(nz))
                    for i in range(nx)], axis=1)
    assert np.allclose(V, ref, rtol=1e-12)
    Vc = orc.interp_model(C, nz, nx, 0, vmin=1500.0, vmax=4700.0)
    assert np.array_equal(Vc, np.clip(ref, 1500.0, 4700.0)) or np.allclose(
        Vc, np.clip(ref, 1500.0, 4700.0), rtol=1e-12)
    assert Vc.min() >= 1500.0 and Vc.max() <= 4700.0


# --------------------------------------------------------------------------
# irregular level-wise control grid ("Testing approach": variable node
# spacing, bilinear two-grid rule, fixed water layer, depth-dependent ranges)
# --------------------------------------------------------------------------

def _levels():
    # 4 levels, coarser with depth; nodes on grid points of a 10 m grid
    level_z = np.array([50.0, 150.0, 300.0, 500.0])
    xs = [np.array([0.0, 100.0, 250.0, 400.0, 600.0]), np.array([0.0, 200.0, 600.0]),
          np.array([100.0, 500.0]), np.array([300.0])]
    n = [len(x) for x in xs]
    rng = np.random.default_rng(7)
    C = [rng.uniform(1500, 4000, k) for k in n]
    return level_z, n, xs, C


def test_levels_along_and_between_levels_match_numpy_interp(orc):
    level_z, n, xs, C = _levels()
    nx, nz, h = 61, 61, 10.0
    V = orc.interp_levels(level_z, n, np.concatenate(xs), np.concatenate(C), nz, nx, h, h)
    x = np.arange(nx) * h
    prof = [np.interp(x, xs[l], C[l]) for l in range(4)]   # end values held outside
    for l, zl in enumerate(level_z):
        assert np.allclose(V[int(zl / h)], prof[l], rtol=1e-13)
    # between levels: linear in z at every x
    for l in range(3):
        for j in range(int(level_z[l] / h), int(level_z[l + 1] / h) + 1):
            b = (j * h - level_z[l]) / (level_z[l + 1] - level_z[l])
            assert np.allclose(V[j], (1 - b) * prof[l] + b * prof[l + 1], rtol=1e-13)
    # above the first level and below the last: held constant
    assert np.allclose(V[:5], prof[0][None, :], rtol=1e-13)
    assert np.allclose(V[50:], prof[3][None, :], rtol=1e-13)
    # node values are reproduced where nodes sit on grid points
    for l in range(4):
        for xv, cv in zip(xs[l], C[l]):
            assert V[int(level_z[l] / h), int(xv / h)] == pytest.approx(cv, rel=1e-13)


def test_levels_on_a_regular_layout_equal_tensor_bilinear(orc):
    # Kz equal levels spanning the domain, each with the same Kx uniform nodes:
    # the level-wise rule is then the tensor-product bilinear interpolation
    Kz, Kx, nz, nx, h = 4, 8, 31, 57, 10.0
    rng = np.random.default_rng(5)
    C = rng.uniform(1500, 4700, (Kz, Kx))
    level_z = np.linspace(0.0, (nz - 1) * h, Kz)
    node_x = np.tile(np.linspace(0.0, (nx - 1) * h, Kx), Kz)
    V = orc.interp_levels(level_z, [Kx] * Kz, node_x, C.ravel(), nz, nx, h, h)
    assert np.allclose(V, orc.interp_model(C, nz, nx, 1), rtol=1e-12)


def test_levels_water_layer_and_clip(orc):
    level_z, n, xs, C = _levels()
    nx, nz, h = 61, 61, 10.0
    Cc = np.concatenate(C)
    V0 = orc.interp_levels(level_z, n, np.concatenate(xs), Cc, nz, nx, h, h)
    V = orc.interp_levels(level_z, n, np.concatenate(xs), Cc, nz, nx, h, h, water_z=95.0,
                          v_water=1480.0, vmin=1600.0, vmax=3500.0)
    assert np.all(V[:10] == 1600.0)            # water 1480 clipped to vmin
    assert np.array_equal(V[10:], np.clip(V0[10:], 1600.0, 3500.0))
    Vw = orc.interp_levels(level_z, n, np.concatenate(xs), Cc, nz, nx, h, h, water_z=95.0,
                           v_water=1500.0)
    assert np.all(Vw[:10] == 1500.0) and np.array_equal(Vw[10:], V0[10:])


def test_level_bounds_straight_lines(orc):
    level_z, n, _, _ = _levels()
    lo, hi = orc.level_bounds(level_z, n, 1600.0, 3400.0, 0.2, 0.3, 0.25, 0.15)
    k = np.repeat(np.arange(4), n)
    s = (level_z - level_z[0]) / (level_z[-1] - level_z[0])
    lo_ref = np.interp(s, [0, 1], [1600.0 * 0.8, 3400.0 * 0.75])
    hi_ref = np.interp(s, [0, 1], [1600.0 * 1.3, 3400.0 * 1.15])
    assert np.allclose(lo, lo_ref[k], rtol=1e-14) and np.allclose(hi, hi_ref[k], rtol=1e-14)
    assert lo[0] == pytest.approx(1280.0) and hi[-1] == pytest.approx(3910.0)
