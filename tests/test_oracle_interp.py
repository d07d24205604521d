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
