"""FP64 CPU oracle for the EMPSO fitness-evaluation path (arXiv 1905.12795).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library and never imports it.

The arithmetic lives in ``empso_oracle.c`` (plain C, FP64, built with FMA
contraction off) and, for the surrogate network, in ``mlp.py`` (numpy FP64).
This module only marshals numpy arrays into those routines.

Parity status of each function (the pin that ties it to something other than
itself lives in ``tests/test_oracle_*.py``):

* ``fd_coeffs`` / ``laplacian`` - pinned: polynomial exactness, measured
  convergence order on smooth fields.
* ``step`` / ``shot`` - pinned: closed-form 2-D Green's function convolved with
  the Ricker wavelet, 2nd-order time convergence, exact discrete energy
  conservation without damping, energy decay with damping, source-receiver
  reciprocity, weak reflection from the damping layer.
* ``ricker`` - pinned: peak value/position, spectral peak at f0, zero mean.
* ``time_axis`` - pinned: stability at the computed dt, growth just above the
  CFL limit; closed-form eigenvalue of the checkerboard mode.
* ``interp_matrix`` / ``interp_model`` - pinned: node interpolation, linear
  reproduction, scipy natural ``CubicSpline``, ``numpy.interp``.
* ``interp_levels`` / ``level_bounds`` (irregular level-wise control grid,
  water layer, depth-dependent ranges) - pinned: ``numpy.interp`` along each
  level and between levels, the tensor-product bilinear mode on a regular
  layout, node reproduction, constant extension, straight-line ranges.
* ``lowpass`` (band-limited resampling with a Blackman-windowed sinc) -
  pinned: pass-band and stop-band amplitudes of sampled sinusoids, exact
  phase at the new sample times, unit DC gain, symmetry of a symmetric pulse.
* ``philox`` - pinned: published known-answer vectors of Philox4x32-10.
* ``log`` / ``cos2pi`` / ``normal`` - pinned: ``math.log`` / ``math.cos``
  within 2 ulp, normality (KS test).
* ``chi`` - pinned: Clerc's constant 0.7298437881 for phi = 4.1, and chi = 1
  at phi = 4.
* ``Swarm`` (EMPSO) - pinned: invariants of the EM rule and of Eq. 1-2,
  statistics of the mutation, sphere and Rastrigin minima reached.
* ``mlp`` (surrogate network, FP64 numpy) - pinned: central finite
  differences, closed-form first Adam step, fit of a known function.
* ``Swarm.step(f, rank)`` - EM sort keyed by ``rank`` (surrogate pre-screen)
  while bests follow f - pinned by its invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "empso_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libempso_oracle.so")
_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_l = ctypes.c_long
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)
_pl = ctypes.POINTER(ctypes.c_long)
_pu32 = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/libempso_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC",
                           "-shared", "-pthread", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _EoPso(ctypes.Structure):
    _fields_ = [("P", _i), ("D", _i), ("c1", _d), ("c2", _d), ("lam", _d),
                ("p_em", _d), ("nm_frac", _d), ("em_start", _i),
                ("em_enabled", _i), ("seed", _u64)]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.eo_fd_coeffs.argtypes = [_i, _pd]
        L.eo_fd_coeffs.restype = _i
        L.eo_ricker.argtypes = [_d, _d]
        L.eo_ricker.restype = _d
        L.eo_time_axis.argtypes = [_i, _d, _d, _d, _d, _d, _pd]
        L.eo_time_axis.restype = _i
        L.eo_damping_profile.argtypes = [_i, _i, _d, _d, _pd]
        L.eo_laplacian.argtypes = [_pd, _i, _i, _d, _d, _i, _pd]
        L.eo_step.argtypes = [_pd, _pd, _pd, _pd, _pd, _pd, _pd, _i, _i, _d, _d,
                              _i, _d, _pd]
        L.eo_shot_batch.argtypes = [_i, _i, _i, _i, _d, _d, _d, _i, _d, _d, _pd, _i,
                                    _pd, _pi, _pi, _i, _pd, _pd, _pl, _pd, _pl, _pd,
                                    _i]
        L.eo_interp_matrix.argtypes = [_i, _i, _i, _pd]
        L.eo_interp_model.argtypes = [_pd, _i, _i, _i, _i, _i, _d, _d, _pd]
        L.eo_interp_levels.argtypes = [_i, _pd, _pi, _pd, _pd, _i, _i, _d, _d, _d, _d, _d, _d,
                                       _pd]
        L.eo_level_bounds.argtypes = [_i, _pd, _pi, _d, _d, _d, _d, _d, _d, _pd, _pd]
        L.eo_lowpass.argtypes = [_pd, _i, _i, _i, _d, _pd, _i, _d, _d, _d]
        L.eo_philox.argtypes = [_pu32, _pu32, _pu32]
        L.eo_uniform.argtypes = [_u64, _u32, _u32, _u32, _u32]
        L.eo_uniform.restype = _d
        L.eo_normal.argtypes = [_u64, _u32, _u32, _u32]
        L.eo_normal.restype = _d
        L.eo_log.argtypes = [_d]
        L.eo_log.restype = _d
        L.eo_cos2pi.argtypes = [_d]
        L.eo_cos2pi.restype = _d
        L.eo_chi.argtypes = [_d, _d]
        L.eo_chi.restype = _d
        L.eo_pso_init.argtypes = [ctypes.POINTER(_EoPso), _pd, _pd, _pd, _pd, _pd, _pd,
                                  _pi, _pi]
        L.eo_pso_step.argtypes = [ctypes.POINTER(_EoPso), _pd, _pd, _pd, _pd, _pd, _pd, _pd,
                                  _pd, _pi, _pi, _pi, _pi]
        _lib = L
    return _lib


def _p(a, t=_pd):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# modelling
# --------------------------------------------------------------------------

def fd_coeffs(order: int) -> np.ndarray:
    c = np.zeros(9)
    R = lib().eo_fd_coeffs(order, _p(c))
    if R < 0:
        raise ValueError(f"unsupported space order {order}")
    return c[:R + 1].copy()


def ricker(f0: float, t) -> np.ndarray:
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.array([lib().eo_ricker(f0, float(x)) for x in t])


def time_axis(order: int, hx: float, hz: float, vmax: float, T: float,
              cfl: float = 0.9) -> tuple[float, int]:
    dt = ctypes.c_double()
    nt = lib().eo_time_axis(order, hx, hz, vmax, T, cfl, ctypes.byref(dt))
    if nt < 0:
        raise ValueError(f"unsupported space order {order}")
    return dt.value, nt


def damping_profile(n: int, pad: int, h: float, vmax: float) -> np.ndarray:
    eta = np.zeros(n + 2 * pad)
    lib().eo_damping_profile(n, pad, h, vmax, _p(eta))
    return eta


def laplacian(u, hx: float, hz: float, order: int) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    lib().eo_laplacian(_p(u), u.shape[1], u.shape[0], hx, hz, order, _p(out))
    return out


def step(um, u0, vel, etax, etaz, src, hx, hz, order, dt) -> np.ndarray:
    """u^{n+1} from u^{n-1}, u^n on an NZ x NX grid (no edge extension here:
    ``vel`` covers the whole grid)."""
    um, u0, vel, etax, etaz = map(_f64, (um, u0, vel, etax, etaz))
    NZ, NX = u0.shape
    u1 = np.empty_like(u0)
    work = np.empty_like(u0)
    s = None
    if src is not None:
        src = _f64(src)
        s = _p(src)
    lib().eo_step(_p(um), _p(u0), _p(u1), _p(vel), _p(etax), _p(etaz), s, NX, NZ,
                  hx, hz, order, dt, _p(work))
    return u1


@dataclass
class Grid:
    """A modelling grid: nx x nz physical nodes at hx, hz metres, a damping
    layer of `pad` cells on all four sides, record length T seconds, Ricker
    peak frequency f0 Hz and the velocity bound vmax used for the CFL step
    and the damping strength.  dt <= 0 selects the CFL rule."""
    nx: int
    nz: int
    hx: float
    hz: float
    pad: int
    order: int
    T: float
    f0: float
    vmax: float
    dt: float = 0.0
    nt: int = 0

    def __post_init__(self):
        if self.dt <= 0:
            self.dt, self.nt = time_axis(self.order, self.hx, self.hz, self.vmax, self.T)
        elif self.nt <= 0:
            self.nt = int(round(self.T / self.dt)) + 1


def shot_batch(grid: Grid, vel, shot_xz, rec_xz, rec_begin, rec_count, dobs=None,
               want_traces=False, nthreads: int | None = None):
    """Forward-model every (model, shot) pair on one grid.

    vel [M][nz][nx] m/s; shot_xz [S][2] m; receivers of shot s are
    rec_xz[rec_begin[s] : rec_begin[s] + rec_count[s]].  dobs: list of S arrays
    [nt][nrec_s] (or None).  Returns (phi [M][S], traces list or None)."""
    vel = _f64(vel).reshape(-1, grid.nz, grid.nx)
    M = vel.shape[0]
    shot_xz = _f64(shot_xz).reshape(-1, 2)
    S = shot_xz.shape[0]
    rec_xz = _f64(rec_xz).reshape(-1, 2)
    rb = np.ascontiguousarray(rec_begin, dtype=np.intc)
    rc = np.ascontiguousarray(rec_count, dtype=np.intc)
    sizes = [grid.nt * int(rc[s]) for s in range(S)]
    doff = np.zeros(S, dtype=np.int_)
    doff[1:] = np.cumsum(sizes)[:-1]
    dflat = None
    if dobs is not None:
        dflat = np.concatenate([_f64(d).reshape(-1) for d in dobs])
        assert dflat.size == sum(sizes)
    toff = np.zeros(M * S, dtype=np.int_)
    tsz = [sizes[q % S] for q in range(M * S)]
    toff[1:] = np.cumsum(tsz)[:-1]
    traces = np.zeros(sum(tsz)) if want_traces else None
    phi = np.zeros(M * S)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    lib().eo_shot_batch(grid.nx, grid.nz, grid.pad, grid.order, grid.hx, grid.hz,
                        grid.dt, grid.nt, grid.f0, grid.vmax, _p(vel), M, _p(shot_xz),
                        _p(rb, _pi), _p(rc, _pi), S, _p(rec_xz),
                        _p(dflat) if dflat is not None else None, _p(doff, _pl),
                        _p(traces) if traces is not None else None, _p(toff, _pl),
                        _p(phi), int(nthreads))
    tr = None
    if want_traces:
        tr = [traces[toff[q]:toff[q] + tsz[q]].reshape(grid.nt, -1) for q in range(M * S)]
    return phi.reshape(M, S), tr


def interp_matrix(K: int, n: int, mode: int = 0) -> np.ndarray:
    W = np.zeros((n, K))
    lib().eo_interp_matrix(K, n, mode, _p(W))
    return W


def interp_model(C, nz: int, nx: int, mode: int = 0, vmin: float = -np.inf,
                 vmax: float = np.inf) -> np.ndarray:
    C = _f64(C)
    Kz, Kx = C.shape
    V = np.zeros((nz, nx))
    lib().eo_interp_model(_p(C), Kz, Kx, nz, nx, mode, vmin, vmax, _p(V))
    return V


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------

INIT_X, INIT_V, U1, U2, EM_U, EM_N = range(6)


def interp_levels(level_z, level_n, node_x, C, nz: int, nx: int, hx: float, hz: float,
                  water_z: float = 0.0, v_water: float = 1500.0, vmin: float = -np.inf,
                  vmax: float = np.inf) -> np.ndarray:
    """Velocity [nz][nx] from an irregular level-wise control grid (bilinear
    two-grid rule, optional fixed water layer, clip)."""
    lz, nx_ = _f64(level_z), _f64(node_x)
    ln = np.ascontiguousarray(level_n, dtype=np.int32)
    Cc = _f64(C)
    assert Cc.size == nx_.size == ln.sum()
    V = np.zeros((nz, nx))
    lib().eo_interp_levels(len(lz), _p(lz), _p(ln, _pi), _p(nx_), _p(Cc), nz, nx, hx, hz,
                           water_z, v_water, vmin, vmax, _p(V))
    return V


def level_bounds(level_z, level_n, v_first, v_last, lo_first, hi_first, lo_last, hi_last):
    """Per-node search ranges (xmin, xmax) of an irregular level grid."""
    lz = _f64(level_z)
    ln = np.ascontiguousarray(level_n, dtype=np.int32)
    K = int(ln.sum())
    lo, hi = np.zeros(K), np.zeros(K)
    lib().eo_level_bounds(len(lz), _p(lz), _p(ln, _pi), v_first, v_last, lo_first, hi_first,
                          lo_last, hi_last, _p(lo), _p(hi))
    return lo, hi


def lowpass(traces, dt_in: float, nt_out: int, dt_out: float, fc: float, W: float) -> np.ndarray:
    """Band-limited resampling / low-pass of traces [S][nt_in][nrec] with the
    Blackman-windowed sinc (cut-off fc Hz, half-width W s) onto the time axis
    m dt_out, m < nt_out.  Returns [S][nt_out][nrec]."""
    x = _f64(traces)
    S, nt_in, nrec = x.shape
    out = np.zeros((S, nt_out, nrec))
    lib().eo_lowpass(_p(x), S, nt_in, nrec, dt_in, _p(out), nt_out, dt_out, fc, W)
    return out


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().eo_philox(_p(c, _pu32), _p(k, _pu32), _p(out, _pu32))
    return out


def uniform(seed, k, i, d, purpose) -> float:
    return lib().eo_uniform(seed, k, i, d, purpose)


def normal(seed, k, i, d) -> float:
    return lib().eo_normal(seed, k, i, d)


def log(u: float) -> float:
    return lib().eo_log(u)


def cos2pi(t: float) -> float:
    return lib().eo_cos2pi(t)


def chi(c1: float, c2: float) -> float:
    return lib().eo_chi(c1, c2)


# --------------------------------------------------------------------------
# EMPSO
# --------------------------------------------------------------------------

class Swarm:
    """EMPSO swarm state in FP64 (positions x, velocities v, personal bests p,
    their fitness pf, global-best index g, generation counter k)."""

    def __init__(self, P, D, xmin, xmax, c1=1.2, c2=2.9, lam=0.5, p_em=0.3,
                 nm_frac=0.25, em_start=10, em_enabled=True, seed=12795):
        self.cfg = _EoPso(P, D, c1, c2, lam, p_em, nm_frac, em_start,
                          1 if em_enabled else 0, seed)
        self.xmin = _f64(np.broadcast_to(xmin, (D,)))
        self.xmax = _f64(np.broadcast_to(xmax, (D,)))
        self.x = np.zeros((P, D))
        self.v = np.zeros((P, D))
        self.p = np.zeros((P, D))
        self.pf = np.zeros(P)
        self._g = ctypes.c_int(0)
        self._k = ctypes.c_int(0)
        self.order = np.arange(P, dtype=np.intc)
        self.em_ran = False
        lib().eo_pso_init(ctypes.byref(self.cfg), _p(self.xmin), _p(self.xmax),
                          _p(self.x), _p(self.v), _p(self.p), _p(self.pf),
                          ctypes.byref(self._g), ctypes.byref(self._k))

    @property
    def g(self) -> int:
        return self._g.value

    @property
    def k(self) -> int:
        return self._k.value

    def set_state(self, x, v, p, pf, g, k):
        self.x[...] = x
        self.v[...] = v
        self.p[...] = p
        self.pf[...] = pf
        self._g.value = int(g)
        self._k.value = int(k)

    def step(self, f, rank=None):
        """One generation; `rank` (optional) keys the EM sort instead of f."""
        f = _f64(f)
        rk = None
        if rank is not None:
            rank = _f64(rank)
            rk = _p(rank)
        em = ctypes.c_int(0)
        lib().eo_pso_step(ctypes.byref(self.cfg), _p(self.xmin), _p(self.xmax), _p(f), rk,
                          _p(self.x), _p(self.v), _p(self.p), _p(self.pf),
                          ctypes.byref(self._g), ctypes.byref(self._k),
                          _p(self.order, _pi), ctypes.byref(em))
        self.em_ran = bool(em.value)


def misfit(d, dobs) -> float:
    """phi = 1/2 sum (d - dobs)^2 ("Testing approach": l2 norm of the data
    residual; the 1/2 is a reading, it does not change the ranking)."""
    r = _f64(d) - _f64(dobs)
    return 0.5 * float(np.sum(r * r))

