"""Run configuration in the paper's JSON layout, and the generation loop with
its per-generation log.

The paper configures a run with one JSON file, a dictionary of dictionaries
(section "Theory", algorithm overview and its JSON example figure): modelling
keys at the top level (times in ms, the Ricker frequency in kHz, grid shape
and spacing, damping cells, space order, acquisition), a ``cgrid`` dictionary
that sets the irregular control grid (the number of unknowns) and a ``pso``
dictionary.  ``load`` accepts that layout, converts it to SI units and
returns a ``RunConfig``; ``open_context`` builds the library context from it;
``run`` runs the generations and writes one JSON record per generation (best
and mean misfit, evaluations, modelling rate) and the final swarm, the log
the paper's DEAP driver keeps ("several statistics" per generation and the
final population).

Readings of keys the paper names but does not define (each also listed with
the other readings of the paper in the design notes):

* ``shape`` / ``spacing`` are [x, z] (the example's 369 x 375 at 25 m x 8 m
  covers the 9.2 km x 3 km model).
* ``cgrid.vstart`` / ``vend``: the 1-D prior velocity at the top and the
  bottom of the model, linear in depth.  ``scale``: control levels lie a local
  wavelength v(z) / f0 divided by ``scale`` apart, with nodes along each level
  at twice that spacing (185 unknowns for the example, against the paper's
  176).  ``water_samples``: the fixed water layer is that many vertical
  samples deep.
* The search range of every node is [v(1 - lo), v(1 + hi)] around the prior,
  lo / hi given at the first and the last level (``cgrid.range_first`` /
  ``range_last``, defaults 30 % / 60 % and 25 % / 25 %) and straight lines
  between.
* ``pso``: ``lambda``, ``c1``, ``c2``, ``gen`` as printed; the swarm size,
  the elitist mutation and the seed, which the example leaves out, take the
  paper's EMPSO settings (``npop`` 360, ``p_em`` 0.3, ``nm_frac`` 0.25,
  ``em_start`` 10) unless given.
* ``shotfile``: observed traces as a ``.npy`` array [nshots][nt][nreceivers];
  when the file does not exist, synthetic observed data are modelled from the
  seeded layered/faulted model (the paper's Marmousi data are not
  available).

One group the paper does not have: an optional ``surrogate`` dictionary
(``keep`` fraction modelled per generation, ``hidden``, ``capacity``, ``lr``,
``train_steps``, ``batch``, ``recent``, ``patience``) runs the generations
with the learned pre-screen; its log records then also carry the number of
particles modelled and the surrogate's rank correlation on them.

The arithmetic of the method runs in the CUDA library; this module only
converts units and drives the library's calls.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding as B
from . import synth

PAPER_DEFAULTS = {"npop": 360, "p_em": 0.3, "nm_frac": 0.25, "em_start": 10, "seed": 12795,
                  "interp_mode": 2, "range_first": [0.3, 0.6], "range_last": [0.25, 0.25]}


@dataclass
class RunConfig:
    """Everything a run needs, in SI units."""
    nx: int
    nz: int
    hx: float
    hz: float
    pad: int
    order: int
    T: float                 # record length (s)
    dt: float                # time step (s); 0 selects the CFL rule
    f0: float                # Ricker peak frequency (Hz)
    shots: np.ndarray        # [S][2] source positions (m)
    receivers: np.ndarray    # [N][2] receiver positions (m)
    level_z: np.ndarray      # control levels (m)
    level_count: np.ndarray  # nodes per level
    node_x: np.ndarray       # node x positions (m), level by level
    xmin: np.ndarray         # per-node search range (m/s)
    xmax: np.ndarray
    water_depth: float       # fixed 1500 m/s layer above this depth (m)
    v_prior: tuple           # (vstart, vend) m/s
    npop: int
    gens: int
    c1: float
    c2: float
    lam: float
    p_em: float
    nm_frac: float
    em_start: int
    seed: int
    shotfile: str = ""
    surrogate: dict | None = None    # learned pre-screen settings (not in the paper)
    raw: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.level_count.sum())

    @property
    def vmin(self) -> float:
        return float(min(1500.0, self.xmin.min()))

    @property
    def vmax(self) -> float:
        return float(self.xmax.max())


def _merge(base: dict, over: dict) -> dict:
    out = dict(base)
    for k, v in (over or {}).items():
        out[k] = _merge(out.get(k, {}), v) if isinstance(v, dict) else v
    return out


def load(src, overrides: dict | None = None) -> RunConfig:
    """Read a run configuration in the paper's JSON layout (a path or a
    dict); `overrides` (same layout) replaces individual keys."""
    if isinstance(src, (str, os.PathLike)):
        with open(src) as f:
            raw = json.load(f)
        base_dir = os.path.dirname(os.path.abspath(src))
    else:
        raw = dict(src)
        base_dir = os.getcwd()
    raw = _merge(raw, overrides or {})
    for key in ("tn", "f0", "nshots", "shape", "spacing", "nbpml", "space_order", "nreceivers",
                "first_src_xcoor", "int_btw_shots", "src_depth", "rec_depth", "cgrid", "pso"):
        if key not in raw:
            raise KeyError(f"run configuration: missing key '{key}'")
    cg, ps = raw["cgrid"], raw["pso"]
    nx, nz = (int(v) for v in raw["shape"])
    hx, hz = (float(v) for v in raw["spacing"])
    ox, oz = (float(v) for v in raw.get("origin", [0.0, 0.0]))
    T = (float(raw["tn"]) - float(raw.get("t0", 0.0))) * 1e-3          # ms -> s
    dt = float(raw.get("dt", 0.0)) * 1e-3                              # ms -> s (0: CFL)
    f0 = float(raw["f0"]) * 1e3                                        # kHz -> Hz
    S = int(raw["nshots"])
    xs = float(raw["first_src_xcoor"]) + float(raw["int_btw_shots"]) * np.arange(S) - ox
    shots = np.stack([xs, np.full(S, float(raw["src_depth"]) - oz)], axis=1)
    N = int(raw["nreceivers"])
    Lx, Lz = (nx - 1) * hx, (nz - 1) * hz
    rx = np.linspace(0.0, Lx, N) if N > 1 else np.zeros(1)
    receivers = np.stack([rx, np.full(N, float(raw["rec_depth"]) - oz)], axis=1)
    vstart, vend = float(cg["vstart"]), float(cg["vend"])
    water = float(cg.get("water_samples", 0)) * hz
    level_z, level_count, node_x, _ = synth.level_layout(Lx, Lz, water, vstart, vend, f0,
                                                         1.0 / float(cg.get("scale", 2.0)))
    rf = cg.get("range_first", PAPER_DEFAULTS["range_first"])
    rl = cg.get("range_last", PAPER_DEFAULTS["range_last"])
    v_first = vstart + (vend - vstart) * level_z[0] / Lz
    v_last = vstart + (vend - vstart) * level_z[-1] / Lz
    xmin, xmax = B.level_bounds(level_z, level_count, v_first, v_last, rf[0], rf[1], rl[0], rl[1])
    return RunConfig(nx=nx, nz=nz, hx=hx, hz=hz, pad=int(raw["nbpml"]), order=int(raw["space_order"]),
                     T=T, dt=dt, f0=f0, shots=shots, receivers=receivers, level_z=level_z,
                     level_count=level_count, node_x=node_x, xmin=xmin, xmax=xmax, water_depth=water,
                     v_prior=(vstart, vend), npop=int(ps.get("npop", PAPER_DEFAULTS["npop"])),
                     gens=int(ps.get("gen", 100)), c1=float(ps.get("c1", 2.0)),
                     c2=float(ps.get("c2", 2.0)), lam=float(ps.get("lambda", 0.5)),
                     p_em=float(ps.get("p_em", PAPER_DEFAULTS["p_em"])),
                     nm_frac=float(ps.get("nm_frac", PAPER_DEFAULTS["nm_frac"])),
                     em_start=int(ps.get("em_start", PAPER_DEFAULTS["em_start"])),
                     seed=int(ps.get("seed", PAPER_DEFAULTS["seed"])),
                     shotfile=os.path.join(base_dir, raw["shotfile"]) if raw.get("shotfile") else "",
                     surrogate=_surrogate_settings(raw.get("surrogate")), raw=raw)


SURROGATE_DEFAULTS = {"keep": 0.25, "hidden": 256, "capacity": 50000, "lr": 1e-3, "train_steps": 6,
                      "batch": 1024, "recent": 4096, "patience": 0}


def _surrogate_settings(sur):
    if sur is None:
        return None
    bad = set(sur) - set(SURROGATE_DEFAULTS)
    if bad:
        raise KeyError(f"run configuration: unknown surrogate keys {sorted(bad)}")
    out = dict(SURROGATE_DEFAULTS)
    out.update(sur)
    if not 0.0 < float(out["keep"]) <= 1.0:
        raise ValueError("run configuration: surrogate.keep must lie in (0, 1]")
    return out


def open_context(cfg: RunConfig):
    """The library context of a run: the grid (level-grid interpolation with
    the fixed water layer), the receivers and the swarm.  Returns
    (context, shot array for the library calls)."""
    grid = B.make_grid(cfg.nx, cfg.nz, cfg.hx, cfg.hz, cfg.pad, cfg.order, cfg.T, cfg.f0,
                       cfg.vmin, cfg.vmax, dt=cfg.dt)
    pso = B.EmpsoPso(cfg.npop, cfg.K, cfg.c1, cfg.c2, cfg.lam, cfg.p_em, cfg.nm_frac,
                     cfg.em_start, 1, cfg.seed)
    ctx = B.Context([grid], cfg.receivers, pso, cfg.xmin, cfg.xmax)
    ctx.set_levels(0, cfg.level_z, cfg.level_count, cfg.node_x)
    if cfg.water_depth > 0:
        ctx.set_water(0, cfg.water_depth, 1500.0)
    N = len(cfg.receivers)
    shots = B.make_shots(cfg.shots, [0] * len(cfg.shots), [N] * len(cfg.shots))
    return ctx, shots


def observed_data(cfg: RunConfig, ctx, shots, seed_model: int = 1905):
    """Observed traces [S][nt][N] on the device: the shot file when it
    exists, else modelled from the seeded layered/faulted model."""
    import torch
    _, nt = ctx.grid_info(0)
    N, S = len(cfg.receivers), len(cfg.shots)
    if cfg.shotfile and os.path.exists(cfg.shotfile):
        d = np.load(cfg.shotfile).astype(np.float32)
        if d.shape != (S, nt, N):
            raise ValueError(f"{cfg.shotfile}: shape {d.shape}, expected {(S, nt, N)}")
        return torch.tensor(d.ravel(), device="cuda")
    true = synth.layered_faulted_model(cfg.nx, cfg.nz, cfg.hx, cfg.hz, seed=seed_model,
                                       vmin=1500.0, vmax=cfg.v_prior[1],
                                       water_depth=cfg.water_depth)
    dobs = torch.zeros(S * nt * N, device="cuda")
    ctx.forward_traces(torch.tensor(true, dtype=torch.float32, device="cuda")[None], shots, dobs)
    return dobs


def run(cfg: RunConfig, log_path: str | None = None, gens: int | None = None, dobs=None):
    """Run the EMPSO generations of `cfg` (or `gens` of them) and return the
    per-generation records; with `log_path`, write them as JSON lines and the
    final swarm (positions and personal-best misfits) as a last record."""
    import torch
    ctx, shots = open_context(cfg)
    try:
        if dobs is None:
            dobs = observed_data(cfg, ctx, shots)
        _, nt = ctx.grid_info(0)
        NX, NZ = cfg.nx + 2 * cfg.pad, cfg.nz + 2 * cfg.pad
        updates = float(cfg.npop) * len(cfg.shots) * NX * NZ * nt
        mis = torch.zeros(cfg.npop, dtype=torch.float64, device="cuda")
        ctx.set_timing(True)
        sur = cfg.surrogate
        if sur:
            ctx.surrogate_init(hidden=int(sur["hidden"]), capacity=int(sur["capacity"]), lr=float(sur["lr"]),
                               seed=cfg.seed)
            ctx.surrogate_set_overlap(True)
            ctx.surrogate_set_policy(recent=int(sur["recent"]), patience=int(sur["patience"]))
        ctx.pso_init()
        G = cfg.gens if gens is None else gens
        records = []
        log = open(log_path, "w") if log_path else None
        t_start = time.perf_counter()
        evaluations = 0
        for k in range(1, G + 1):
            rho = None
            if sur:
                n_mod = ctx.surrogate_generation(shots, dobs, float(sur["keep"]), warm=cfg.npop,
                                                 train_steps=int(sur["train_steps"]),
                                                 batch=int(sur["batch"]), misfit_out=mis)
                if n_mod < cfg.npop:
                    rho = ctx.surrogate_last_rank_corr()
            else:
                ctx.generation(shots, dobs, mis)
                n_mod = cfg.npop
            evaluations += n_mod
            m = mis.cpu().numpy()
            kernel_ms = ctx.read_timing()[1]
            fin = m[np.isfinite(m)]     # the modelled particles' misfits
            pf = torch.zeros(cfg.npop, dtype=torch.float64, device="cuda")
            gk = torch.zeros(2, dtype=torch.int32, device="cuda")
            ctx.pso_get_state(pf=pf, gk=gk)
            rec = {"generation": k, "best_misfit": float(fin.min()) if fin.size else None,
                   "mean_misfit": float(fin.mean()) if fin.size else None,
                   "gbest_misfit": float(pf[int(gk[0].item())].item()), "gbest": int(gk[0].item()),
                   "modelled": n_mod, "evaluations": evaluations,
                   "nonfinite": int(n_mod - fin.size) if not sur else None,
                   "modelling_ms": kernel_ms,
                   "updates_per_s": updates * n_mod / cfg.npop / (kernel_ms * 1e-3),
                   "surrogate_rank_corr": rho, "wall_s": time.perf_counter() - t_start}
            records.append(rec)
            if log:
                log.write(json.dumps(rec) + "\n")
                log.flush()
        if log:
            x = torch.zeros(cfg.npop, cfg.K, dtype=torch.float64, device="cuda")
            pf = torch.zeros(cfg.npop, dtype=torch.float64, device="cuda")
            ctx.pso_get_state(x=x, pf=pf)
            log.write(json.dumps({"final_swarm": x.cpu().numpy().tolist(),
                                  "personal_best_misfit": pf.cpu().numpy().tolist()}) + "\n")
            log.close()
        return records
    finally:
        ctx.close()
