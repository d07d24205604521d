"""Seeded synthetic inputs: velocity models, acquisition geometry, particles.

The paper's Marmousi crop and its shot file are not available, so every
workload is built from the generators below.  This module holds none of the
method's arithmetic (no interpolation, modelling or misfit); it only draws
inputs, so both the CUDA path and the CPU oracle can be fed the same arrays.

Models follow the paper's setting ("Testing approach": 1-D background with
velocity increasing with depth from 1500 m/s, a water layer on top) with
dipping layers and one normal fault added so that the search has structure to
find.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def layered_faulted_model(nx: int, nz: int, hx: float, hz: float, seed: int = 1905,
                          vmin: float = 1500.0, vmax: float = 4700.0,
                          water_depth: float = 0.0) -> np.ndarray:
    """Velocity [nz][nx] in m/s: 4-7 layers with dipping interfaces (dip <= 15
    degrees), velocity increasing with depth from `vmin` (top layer) to at
    most `vmax`, a +-5 % lateral gradient and one 60-degree normal fault with
    100-300 m throw offsetting the interfaces below its tip; with
    water_depth > 0 a 1500 m/s water layer covers depths <= water_depth."""
    rng = np.random.default_rng(seed)
    Lx, Lz = (nx - 1) * hx, (nz - 1) * hz
    nl = int(rng.integers(4, 8))
    depths = np.sort(rng.uniform(0.08, 0.92, nl - 1)) * Lz
    dips = np.tan(np.deg2rad(rng.uniform(-15.0, 15.0, nl - 1)))
    vel_layers = np.sort(rng.uniform(vmin + 300.0, vmax, nl - 1))
    vel_layers = np.concatenate([[vmin], vel_layers])
    xf = rng.uniform(0.3, 0.7) * Lx
    ztip = rng.uniform(0.1, 0.3) * Lz
    throw = rng.uniform(100.0, 300.0)
    fdip = np.tan(np.deg2rad(60.0))
    grad = rng.uniform(-0.05, 0.05)
    x = np.arange(nx) * hx
    z = np.arange(nz) * hz
    X, Z = np.meshgrid(x, z)
    # hanging wall: points right of the fault plane and below its tip are shifted up
    hanging = (X - xf) > (Z - ztip) / fdip
    Zs = np.where(hanging & (Z > ztip), Z - throw, Z)
    layer = np.zeros_like(X, dtype=np.int64)
    for b in range(nl - 1):
        zb = depths[b] + dips[b] * (X - 0.5 * Lx)
        layer += (Zs > zb).astype(np.int64)
    v = vel_layers[layer] * (1.0 + grad * (X / max(Lx, 1.0) - 0.5))
    v[layer == 0] = vmin
    v = np.clip(v, vmin, vmax)
    if water_depth > 0:
        v[z <= water_depth, :] = 1500.0
    return v


def two_layer_model(nx: int, nz: int, hz: float, v_top: float = 1500.0,
                    v_bottom: float = 2500.0, z_interface: float = 500.0) -> np.ndarray:
    """Two horizontal layers, interface at depth `z_interface` (metres)."""
    z = np.arange(nz) * hz
    v = np.where(z[:, None] < z_interface, v_top, v_bottom)
    return np.broadcast_to(v, (nz, nx)).astype(np.float64).copy()


def level_layout(Lx: float, Lz: float, water_depth: float, v_top: float = 1500.0,
                 v_bottom: float = 3500.0, f0: float = 6.0, frac: float = 0.5):
    """Irregular level-wise control grid whose spacing grows with depth, the
    structure of the paper's 176-node grid (its resolution criteria are only
    in a cited work): the prior is the 1-D model linear from v_top at z = 0 to
    v_bottom at z = Lz; the first level lies at the water bottom, each next
    level `frac` local wavelengths v(z)/f0 deeper, the last at Lz; level l
    holds nodes evenly spread over [0, Lx] at a horizontal spacing of twice
    its vertical spacing.  Returns (level_z, level_count, node_x, v1d) with
    v1d(z) the prior."""
    def v1d(z):
        return v_top + (v_bottom - v_top) * np.asarray(z, dtype=float) / Lz
    z = [max(water_depth, 0.0)]
    while True:
        dz = frac * float(v1d(z[-1])) / f0
        if z[-1] + 1.5 * dz >= Lz:
            break
        z.append(z[-1] + dz)
    z.append(Lz)
    level_z = np.array(z)
    spacing = frac * v1d(level_z) / f0
    counts = [max(2, int(np.ceil(Lx / (2.0 * d))) + 1) for d in spacing]
    node_x = np.concatenate([np.linspace(0.0, Lx, n) for n in counts])
    return level_z, np.array(counts, dtype=np.int32), node_x, v1d


def shot_line(S: int, Lx: float, z: float) -> np.ndarray:
    """S sources evenly spread over [0, Lx]: x_s = (s + 1/2) Lx / S, depth z."""
    xs = (np.arange(S) + 0.5) * Lx / S
    return np.stack([xs, np.full(S, z)], axis=1)


def receiver_line(nx: int, hx: float, z: float) -> np.ndarray:
    """One receiver per horizontal grid node at depth z (the paper's layout:
    one receiver for each sample on the horizontal axis)."""
    return np.stack([np.arange(nx) * hx, np.full(nx, z)], axis=1)


def random_particles(P: int, K: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """P particles of K control-node velocities, uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(P, K))


@dataclass
class GridSpec:
    """One modelling grid: nx x nz physical nodes, spacing hx/hz in metres,
    `pad` damping cells on each side, space order, record length T (s), Ricker
    peak frequency f0 (Hz), the velocity bound vmax (m/s) that sets the CFL
    step and the damping strength, and the Kz x Kx control-node layout of a
    particle."""
    nx: int
    nz: int
    hx: float
    hz: float
    pad: int
    order: int
    T: float
    f0: float
    vmax: float
    vmin: float = 1500.0
    kx: int = 8
    kz: int = 4
    mode: int = 0      # 0 natural cubic spline, 1 bilinear


@dataclass
class Workload:
    """A named workload: one or more grids, the shots on each grid and the
    swarm that searches it."""
    name: str
    grids: list
    shots_per_grid: list
    P: int
    gens: int
    src_z: float
    rec_z: float
    seed_model: int = 1905
    seed_pso: int = 12795
    xmin: float = 1500.0
    xmax: float = 4700.0
    extra: dict = field(default_factory=dict)


def workloads() -> dict:
    """The five workloads the framework is measured on, by name."""
    single = GridSpec(101, 101, 10.0, 10.0, 20, 4, 0.5, 10.0, 2625.0, 1500.0)
    plain = GridSpec(461, 151, 20.0, 20.0, 40, 8, 3.0, 6.0, 4700.0)
    plain_bl = GridSpec(461, 151, 20.0, 20.0, 40, 8, 3.0, 6.0, 4700.0, mode=1)
    coarse = GridSpec(231, 76, 40.0, 40.0, 20, 8, 4.0, 3.0, 4700.0)
    hires = GridSpec(921, 301, 10.0, 10.0, 60, 8, 4.0, 12.0, 4700.0, kx=24, kz=8)
    surr = GridSpec(101, 101, 10.0, 10.0, 20, 4, 0.5, 10.0, 3200.0, 1200.0)
    return {
        "single-forward-101x101": Workload("single-forward-101x101", [single], [1], 1, 1,
                                           20.0, 20.0),
        "empso-461x151-P32-S16": Workload("empso-461x151-P32-S16", [plain], [16], 32, 50,
                                          20.0, 20.0),
        "uneven-P256-S16x2": Workload("uneven-P256-S16x2", [coarse, plain], [16, 16], 256,
                                      1, 20.0, 20.0),
        "surrogate-101x101-P1024": Workload("surrogate-101x101-P1024", [surr], [1], 1024,
                                            100, 20.0, 20.0, xmin=1200.0, xmax=3200.0),
        "hires-921x301-P512-S64": Workload("hires-921x301-P512-S64", [hires], [64], 512, 1,
                                           20.0, 20.0),
        # the plain workload's grid and geometry under the paper's own
        # parameterisation: level-wise irregular control grid below a 200 m
        # water layer, bilinear, depth-dependent ranges around a linear prior
        "compare-461x151-P32-S16": Workload("compare-461x151-P32-S16", [plain_bl], [16], 32, 60,
                                            20.0, 20.0,
                                            extra=dict(water=200.0, v_prior=(1500.0, 4500.0),
                                                       ranges=(0.3, 0.6, 0.25, 0.25),
                                                       frac=0.75)),
    }
