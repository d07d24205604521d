"""Thin ctypes binding over the C ABI declared in ``include/empso.h``.

Argument marshalling only: every step of the method runs in the CUDA
library.  Device buffers are passed as ``torch.Tensor`` objects on the
current CUDA device; the current PyTorch stream is handed to the library.
If the library has not been built (``paper_1905_12795_gb300.build.build()``
or ``__graft_entry__.build()``) the first use raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_i32 = ctypes.c_int32
_f32 = ctypes.c_float
_f64 = ctypes.c_double
_vp = ctypes.c_void_p

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA_ERROR", 4: "NONFINITE",
          5: "TIMEOUT", 6: "UNSUPPORTED", 7: "NOT_INITIALIZED", 8: "IO_ERROR"}

EXPORTS = ["empso_create", "empso_destroy", "empso_grid_info", "empso_time_axis", "empso_interp", "forward_traces",
           "eval_models", "eval_fitness", "pso_init", "pso_step", "pso_get_state",
           "pso_set_state", "empso_set_kernel", "empso_set_cluster", "empso_set_tile_rows", "empso_set_gradient_chains",
           "empso_last_tile_rows", "empso_last_clusters", "empso_last_launch", "empso_device_error", "empso_set_timing", "empso_read_timing", "eval_models_noalloc",
           "empso_generation", "empso_autotune", "empso_set_tuning_cache",
           "pso_step_ranked", "surrogate_init", "surrogate_set_backend", "surrogate_set_overlap", "surrogate_set_policy", "surrogate_last_rank_corr", "surrogate_predict", "surrogate_add",
           "surrogate_train", "surrogate_params", "surrogate_grad", "surrogate_generation",
           "empso_nonfinite_count", "empso_set_strict", "empso_save", "empso_load",
           "empso_set_levels", "empso_set_water", "empso_level_bounds", "empso_last_kernel_name",
           "empso_lowpass", "empso_gradient", "empso_fwi", "empso_last_paired_units",
           "empso_status_string", "empso_last_error"]


class EmpsoGrid(ctypes.Structure):
    _fields_ = [("nx", _i32), ("nz", _i32), ("pad", _i32), ("space_order", _i32),
                ("hx", _f32), ("hz", _f32), ("t_rec", _f32), ("f0", _f32), ("dt", _f32),
                ("vmin", _f32), ("vmax", _f32), ("kx", _i32), ("kz", _i32),
                ("interp_mode", _i32)]


class EmpsoShot(ctypes.Structure):
    _fields_ = [("sx", _f32), ("sz", _f32), ("rec_begin", _i32), ("nrec", _i32),
                ("grid_id", _i32), ("weight", _f32)]


class EmpsoPso(ctypes.Structure):
    _fields_ = [("P", _i32), ("D", _i32), ("c1", _f64), ("c2", _f64), ("lam", _f64),
                ("p_em", _f64), ("nm_frac", _f64), ("em_start", _i32), ("em_enabled", _i32),
                ("seed", ctypes.c_uint64)]


class EmpsoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def level_bounds(level_z, level_count, v_first, v_last, lo_first, hi_first, lo_last, hi_last):
    """Depth-dependent search ranges (xmin, xmax) of an irregular level grid."""
    lz = np.ascontiguousarray(level_z, dtype=np.float32)
    lc = np.ascontiguousarray(level_count, dtype=np.int32)
    K = int(lc.sum())
    lo, hi = np.zeros(K), np.zeros(K)
    rc = load().empso_level_bounds(len(lz), lz.ctypes.data, lc.ctypes.data, v_first, v_last,
                                   lo_first, hi_first, lo_last, hi_last, lo.ctypes.data,
                                   hi.ctypes.data)
    if rc != 0:
        raise EmpsoError(rc, "invalid level layout or ranges")
    return lo, hi


def lib_path() -> str:
    return _build.LIB


def load():
    """Open the built library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"EMPSO CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build())")
    import torch  # noqa: F401  - load torch's CUDA runtime first so both share it
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.empso_create.argtypes = [P(EmpsoGrid), _i32, P(_f32), _i32, P(EmpsoPso), P(_f64), P(_f64),
                               P(_vp)]
    L.empso_destroy.argtypes = [_vp]
    L.empso_destroy.restype = None
    L.empso_grid_info.argtypes = [_vp, _i32, P(_f32), P(_i32)]
    L.empso_time_axis.argtypes = [P(EmpsoGrid), P(_f32), P(_i32)]
    L.empso_interp.argtypes = [_vp, _i32, _vp, _i32, _vp, _vp]
    L.forward_traces.argtypes = [_vp, _vp, _i32, P(EmpsoShot), _i32, _vp, _vp]
    L.eval_models.argtypes = [_vp, _vp, _i32, P(EmpsoShot), _i32, _vp, _vp, _vp]
    L.eval_fitness.argtypes = [_vp, _vp, _i32, P(EmpsoShot), _i32, _vp, _vp, _vp]
    L.pso_init.argtypes = [_vp, _vp, _vp]
    L.pso_step.argtypes = [_vp, _vp, _vp, P(_i32), _vp]
    L.pso_get_state.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.pso_set_state.argtypes = [_vp, _vp, _vp, _vp, _vp, _i32, _i32, _vp]
    L.empso_set_kernel.argtypes = [_vp, _i32]
    L.empso_set_cluster.argtypes = [_vp, _i32]
    L.empso_set_tile_rows.argtypes = [_vp, _i32]
    L.empso_set_gradient_chains.argtypes = [_vp, _i32]
    L.empso_last_tile_rows.argtypes = [_vp, P(_i32)]
    L.empso_last_clusters.argtypes = [_vp, P(_i32)]
    L.empso_device_error.argtypes = [_vp, P(_i32), _vp]
    L.empso_last_launch.argtypes = [_vp, P(_i32), P(_i32)]
    L.empso_set_timing.argtypes = [_vp, _i32]
    L.empso_read_timing.argtypes = [_vp, P(_f64)]
    L.empso_generation.argtypes = [_vp, P(EmpsoShot), _i32, _vp, _vp, _vp]
    L.empso_autotune.argtypes = [_vp, _vp, _i32, P(EmpsoShot), _i32, _vp, _vp, P(_i32), P(_i32), _vp]
    L.empso_set_tuning_cache.argtypes = [_vp, ctypes.c_char_p]
    L.pso_step_ranked.argtypes = [_vp, _vp, _vp, _vp, P(_i32), _vp]
    L.surrogate_init.argtypes = [_vp, _i32, _i32, _f32, ctypes.c_uint64]
    L.surrogate_set_backend.argtypes = [_vp, _i32]
    L.surrogate_set_overlap.argtypes = [_vp, _i32]
    L.surrogate_set_policy.argtypes = [_vp, _i32, _f32, _i32]
    L.surrogate_last_rank_corr.argtypes = [_vp, P(_f32), _vp]
    L.empso_nonfinite_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), _i32, _vp]
    L.empso_set_strict.argtypes = [_vp, _i32]
    L.empso_set_levels.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp]
    L.empso_last_kernel_name.argtypes = [_vp]
    L.empso_last_paired_units.argtypes = [_vp, P(_i32)]
    L.empso_last_kernel_name.restype = ctypes.c_char_p
    L.empso_set_water.argtypes = [_vp, _i32, _f32, _f32]
    L.empso_gradient.argtypes = [_vp, _vp, _i32, P(EmpsoShot), _i32, _vp, _vp, _vp, _vp]
    L.empso_fwi.argtypes = [_vp, _vp, P(EmpsoShot), _i32, _vp, _i32, _f32, _f32, P(_f64), P(_i32),
                            _vp]
    L.empso_lowpass.argtypes = [_vp, _vp, _i32, _i32, _i32, _f64, _vp, _i32, _f64, _f64, _f64, _vp]
    L.empso_level_bounds.argtypes = [_i32, _vp, _vp, _f64, _f64, _f64, _f64, _f64, _f64, _vp, _vp]
    L.empso_save.argtypes = [_vp, ctypes.c_char_p]
    L.empso_load.argtypes = [_vp, ctypes.c_char_p]
    L.surrogate_predict.argtypes = [_vp, _vp, _i32, _vp, _vp]
    L.surrogate_add.argtypes = [_vp, _vp, _vp, _i32, _vp]
    L.surrogate_train.argtypes = [_vp, _i32, _i32, _vp]
    L.surrogate_params.argtypes = [_vp, _vp, _vp, P(_i32), _vp]
    L.surrogate_grad.argtypes = [_vp, _vp, _vp, _i32, _vp, _vp, _vp]
    L.surrogate_generation.argtypes = [_vp, P(EmpsoShot), _i32, _vp, _f64, _i32, _i32, _i32, _vp,
                                       P(_i32), _vp]
    L.eval_models_noalloc.argtypes = [P(EmpsoGrid), P(_f32), _i32, _vp, _i32, P(EmpsoShot), _i32,
                                      _vp, _vp, _vp]
    L.empso_status_string.argtypes = [_i32]
    L.empso_status_string.restype = ctypes.c_char_p
    L.empso_last_error.argtypes = [_vp]
    L.empso_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("empso_destroy", "empso_status_string", "empso_last_error",
                        "empso_last_kernel_name"):
            getattr(L, name).restype = _i32
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_grid(nx, nz, hx, hz, pad, order, T, f0, vmin, vmax, kx=8, kz=4, mode=0, dt=0.0):
    return EmpsoGrid(nx, nz, pad, order, hx, hz, T, f0, dt, vmin, vmax, kx, kz, mode)


def time_axis(grid: EmpsoGrid):
    """(dt, nt) the library gives `grid`, without a context (host only)."""
    L = load()
    dt = _f32()
    nt = _i32()
    rc = L.empso_time_axis(ctypes.byref(grid), ctypes.byref(dt), ctypes.byref(nt))
    if rc != 0:
        raise EmpsoError(rc, L.empso_last_error(None).decode())
    return dt.value, nt.value


def make_shots(shot_xz, rec_begin, rec_count, grid_ids=None, weights=None):
    S = len(shot_xz)
    arr = (EmpsoShot * S)()
    for s in range(S):
        arr[s] = EmpsoShot(float(shot_xz[s][0]), float(shot_xz[s][1]), int(rec_begin[s]),
                           int(rec_count[s]), 0 if grid_ids is None else int(grid_ids[s]),
                           1.0 if weights is None else float(weights[s]))
    return arr


def eval_models_noalloc(grid: EmpsoGrid, rec_xz, vel, shots, d_obs, misfit):
    """Allocation-free misfit of gridded models (no context; fixed scratch
    inside the library).  vel, d_obs, misfit: CUDA tensors; rec_xz: host
    array [N][2]; shots: ``make_shots`` array on grid 0."""
    import torch
    L = load()
    rec = np.ascontiguousarray(np.asarray(rec_xz, dtype=np.float32).reshape(-1, 2))
    # the library sees raw pointers only: sizes and types are checked here
    if vel.dtype != torch.float32 or vel.dim() != 3 or tuple(vel.shape[1:]) != (grid.nz, grid.nx):
        raise TypeError(f"vel must be float32 [M][{grid.nz}][{grid.nx}], got "
                        f"{vel.dtype} {tuple(vel.shape)}")
    M = vel.shape[0]
    if misfit.dtype != torch.float64 or misfit.numel() < M:
        raise TypeError(f"misfit must be float64 with at least {M} elements")
    if M > 0:
        need = time_axis(grid)[1] * sum(int(sh.nrec) for sh in shots)
        if d_obs.dtype != torch.float32 or d_obs.numel() < need:
            raise ValueError(f"d_obs must be float32 with at least nt * sum(nrec) = {need} elements")
    rc = L.eval_models_noalloc(ctypes.byref(grid), rec.ctypes.data_as(ctypes.POINTER(_f32)),
                               rec.shape[0], _ptr(vel), vel.shape[0], shots, len(shots),
                               _ptr(d_obs), _ptr(misfit), _stream())
    if rc != 0:
        raise EmpsoError(rc, L.empso_last_error(None).decode())


class Context:
    """An EMPSO context: grids (``EmpsoGrid`` list), a receiver table
    ([N][2] metres) and optionally a swarm (``EmpsoPso`` + bounds)."""

    def __init__(self, grids, rec_xz, pso: EmpsoPso | None = None, xmin=None, xmax=None):
        L = load()
        self._L = L
        ng = len(grids)
        self._grids = (EmpsoGrid * ng)(*grids)
        rec = np.ascontiguousarray(np.asarray(rec_xz, dtype=np.float32).reshape(-1, 2))
        self._rec = rec
        h = ctypes.c_void_p()
        self.pso = pso
        xmn = xmx = None
        if pso is not None:
            self._xmin = np.ascontiguousarray(np.broadcast_to(xmin, (pso.D,)), dtype=np.float64)
            self._xmax = np.ascontiguousarray(np.broadcast_to(xmax, (pso.D,)), dtype=np.float64)
            xmn = self._xmin.ctypes.data_as(ctypes.POINTER(_f64))
            xmx = self._xmax.ctypes.data_as(ctypes.POINTER(_f64))
        rc = L.empso_create(self._grids, ng, rec.ctypes.data_as(ctypes.POINTER(_f32)),
                            rec.shape[0], ctypes.byref(pso) if pso is not None else None,
                            xmn, xmx, ctypes.byref(h))
        if rc != 0:
            raise EmpsoError(rc, L.empso_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.empso_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise EmpsoError(rc, self._L.empso_last_error(self._h).decode())

    def grid_info(self, gid=0):
        dt = _f32()
        nt = _i32()
        self._check(self._L.empso_grid_info(self._h, gid, ctypes.byref(dt), ctypes.byref(nt)))
        return dt.value, nt.value

    def interp(self, gid, particles, vel_out):
        self._check(self._L.empso_interp(self._h, gid, _ptr(particles), particles.shape[0],
                                         _ptr(vel_out), _stream()))

    def forward_traces(self, vel, shots, traces):
        self._check(self._L.forward_traces(self._h, _ptr(vel), vel.shape[0], shots, len(shots),
                                           _ptr(traces), _stream()))

    def eval_models(self, vel, shots, d_obs, misfit):
        self._check(self._L.eval_models(self._h, _ptr(vel), vel.shape[0], shots, len(shots),
                                        _ptr(d_obs), _ptr(misfit), _stream()))

    def eval_fitness(self, particles, shots, d_obs, misfit):
        self._check(self._L.eval_fitness(self._h, _ptr(particles), particles.shape[0], shots,
                                         len(shots), _ptr(d_obs), _ptr(misfit), _stream()))

    KERNEL_AUTO, KERNEL_STREAMING, KERNEL_RESIDENT = 0, 1, 2

    def set_kernel(self, kind: int):
        self._check(self._L.empso_set_kernel(self._h, int(kind)))

    def device_error(self):
        """Device status word of the launches since the last call (0 = none)."""
        v = _i32()
        self._check(self._L.empso_device_error(self._h, ctypes.byref(v), _stream()))
        return v.value

    def set_cluster(self, ctas: int):
        self._check(self._L.empso_set_cluster(self._h, int(ctas)))

    def set_tile_rows(self, rows: int):
        """Rows per thread of the on-chip kernel: 0 automatic, 8 or 13."""
        self._check(self._L.empso_set_tile_rows(self._h, int(rows)))

    def set_gradient_chains(self, chains: int):
        """Independent chains of instances in the gradient's backward pass (1..8; 0 automatic)."""
        self._check(self._L.empso_set_gradient_chains(self._h, int(chains)))

    def last_clusters(self) -> int:
        """Co-resident clusters (streaming kernels: CTAs) of the last launch."""
        r = _i32()
        self._check(self._L.empso_last_clusters(self._h, ctypes.byref(r)))
        return r.value

    def last_tile_rows(self) -> int:
        r = _i32()
        self._check(self._L.empso_last_tile_rows(self._h, ctypes.byref(r)))
        return r.value

    def last_launch(self):
        """(kernel kind, CTAs per instance) of the last modelling launch."""
        k, c = _i32(), _i32()
        self._check(self._L.empso_last_launch(self._h, ctypes.byref(k), ctypes.byref(c)))
        return k.value, c.value

    def set_levels(self, grid_id, level_z, level_count, node_x):
        """Irregular level-wise control grid on grid `grid_id` (interp mode 2)."""
        lz = np.ascontiguousarray(level_z, dtype=np.float32)
        lc = np.ascontiguousarray(level_count, dtype=np.int32)
        nx = np.ascontiguousarray(node_x, dtype=np.float32)
        self._check(self._L.empso_set_levels(self._h, int(grid_id), len(lz), lz.ctypes.data,
                                             lc.ctypes.data, nx.ctypes.data))

    def set_water(self, grid_id, water_depth, v_water=1500.0):
        self._check(self._L.empso_set_water(self._h, int(grid_id), float(water_depth),
                                            float(v_water)))

    def lowpass(self, traces, dt_in, out, dt_out, f_cut, half_width):
        """Band-limited resampling of traces [S][nt_in][nrec] onto out [S][nt_out][nrec]."""
        S, nt_in, nrec = traces.shape
        So, nt_out, nro = out.shape
        assert So == S and nro == nrec
        self._check(self._L.empso_lowpass(self._h, _ptr(traces), S, nt_in, nrec, float(dt_in),
                                          _ptr(out), nt_out, float(dt_out), float(f_cut),
                                          float(half_width), _stream()))

    def gradient(self, vel, shots, d_obs, grad, misfit=None):
        """Misfit (optional device [M] doubles) and dphi/dv [M][nz][nx] of gridded models."""
        self._check(self._L.empso_gradient(self._h, _ptr(vel), vel.shape[0], shots, len(shots),
                                           _ptr(d_obs), _ptr(misfit), _ptr(grad), _stream()))

    def fwi(self, vel, shots, d_obs, iters, vmin, vmax):
        """Steepest-descent FWI of vel [nz][nx] in place; returns the misfit history."""
        hist = (_f64 * (iters + 1))()
        done = _i32()
        self._check(self._L.empso_fwi(self._h, _ptr(vel), shots, len(shots), _ptr(d_obs), int(iters),
                                      float(vmin), float(vmax), hist, ctypes.byref(done), _stream()))
        return list(hist)[:done.value + 1]

    def nonfinite_count(self, reset=False):
        """Non-finite misfits (returned as +inf) since creation or the last reset."""
        n = ctypes.c_int64()
        self._check(self._L.empso_nonfinite_count(self._h, ctypes.byref(n), 1 if reset else 0,
                                                  _stream()))
        return n.value

    def set_strict(self, enable=True):
        """Evaluation calls raise EmpsoError(NONFINITE) when they produce a non-finite misfit."""
        self._check(self._L.empso_set_strict(self._h, 1 if enable else 0))

    def save(self, path):
        """Checkpoint the swarm (and surrogate) state to a file."""
        self._check(self._L.empso_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Restore a checkpoint written by save() into a context of the same shape."""
        self._check(self._L.empso_load(self._h, os.fsencode(path)))

    def last_paired_units(self):
        """Work units of the last on-chip launch that ran two instances (one per half cluster)."""
        n = _i32()
        self._check(self._L.empso_last_paired_units(self._h, ctypes.byref(n)))
        return n.value

    def last_kernel_name(self):
        """Device-function name of the last modelling launch's kernel."""
        return self._L.empso_last_kernel_name(self._h).decode()

    def set_timing(self, enable=True):
        self._check(self._L.empso_set_timing(self._h, 1 if enable else 0))

    def read_timing(self):
        """(fields_ms, modelling_ms, reduction_ms) of the last timed call."""
        ms = (_f64 * 3)()
        self._check(self._L.empso_read_timing(self._h, ms))
        return tuple(ms)

    def generation(self, shots, d_obs, misfit_out=None):
        """One EMPSO generation (fitness + step), captured as a CUDA graph on
        the first call for these shots/buffers and replayed afterwards."""
        self._check(self._L.empso_generation(self._h, shots, len(shots), _ptr(d_obs),
                                             _ptr(misfit_out), _stream()))

    def autotune(self, particles, shots, d_obs, misfit):
        """Time every kernel / cluster size on this batch; keep the fastest.
        Returns (kind, cluster)."""
        k, c = _i32(), _i32()
        self._check(self._L.empso_autotune(self._h, _ptr(particles), particles.shape[0], shots,
                                           len(shots), _ptr(d_obs), _ptr(misfit), ctypes.byref(k),
                                           ctypes.byref(c), _stream()))
        return k.value, c.value

    def set_tuning_cache(self, path):
        self._check(self._L.empso_set_tuning_cache(self._h, (path or "").encode()))

    def pso_step_ranked(self, misfit, rank, particles_out=None):
        self._check(self._L.pso_step_ranked(self._h, _ptr(misfit), _ptr(rank), _ptr(particles_out),
                                            None, _stream()))

    # surrogate pre-screening
    def surrogate_init(self, hidden=256, capacity=50000, lr=1e-3, seed=1):
        self._check(self._L.surrogate_init(self._h, hidden, capacity, lr, seed))

    def surrogate_set_policy(self, recent=0, min_rank_corr=0.0, patience=0):
        """Recency share of the minibatches, the rank-correlation fallback and
        the stagnation fallback (whole swarm after `patience` screened
        generations in a row without a new best)."""
        self._check(self._L.surrogate_set_policy(self._h, int(recent), float(min_rank_corr), int(patience)))

    def surrogate_last_rank_corr(self) -> float:
        r = _f32()
        self._check(self._L.surrogate_last_rank_corr(self._h, ctypes.byref(r), _stream()))
        return r.value

    def surrogate_set_overlap(self, enable=True):
        """Train pre-screening generations beside their modelling (one generation of lag)."""
        self._check(self._L.surrogate_set_overlap(self._h, 1 if enable else 0))

    def surrogate_set_backend(self, kind):
        """1: tcgen05 tensor cores (default), 0: mma.sync."""
        self._check(self._L.surrogate_set_backend(self._h, int(kind)))

    def surrogate_predict(self, particles, logphi):
        self._check(self._L.surrogate_predict(self._h, _ptr(particles), particles.shape[0],
                                              _ptr(logphi), _stream()))

    def surrogate_add(self, particles, misfit):
        self._check(self._L.surrogate_add(self._h, _ptr(particles), _ptr(misfit),
                                          particles.shape[0], _stream()))

    def surrogate_train(self, steps, batch):
        self._check(self._L.surrogate_train(self._h, steps, batch, _stream()))

    def surrogate_n_params(self):
        n = _i32()
        self._check(self._L.surrogate_params(self._h, None, None, ctypes.byref(n), _stream()))
        return n.value

    def surrogate_get(self, out):
        self._check(self._L.surrogate_params(self._h, _ptr(out), None, None, _stream()))

    def surrogate_set(self, params):
        self._check(self._L.surrogate_params(self._h, None, _ptr(params), None, _stream()))

    def surrogate_grad(self, particles, target, grad, loss=None):
        self._check(self._L.surrogate_grad(self._h, _ptr(particles), _ptr(target),
                                           particles.shape[0], _ptr(grad), _ptr(loss), _stream()))

    def surrogate_generation(self, shots, d_obs, keep_frac=0.25, warm=None, train_steps=20,
                             batch=256, misfit_out=None):
        """One surrogate-assisted generation; returns how many particles were modelled."""
        n = _i32()
        warm = self.pso.P if warm is None else warm
        self._check(self._L.surrogate_generation(self._h, shots, len(shots), _ptr(d_obs), keep_frac,
                                                 warm, train_steps, batch, _ptr(misfit_out),
                                                 ctypes.byref(n), _stream()))
        return n.value

    def pso_init(self, particles_out=None):
        self._check(self._L.pso_init(self._h, _ptr(particles_out), _stream()))

    def pso_step(self, misfit, particles_out=None, want_gbest=False):
        g = _i32(-1)
        self._check(self._L.pso_step(self._h, _ptr(misfit), _ptr(particles_out),
                                     ctypes.byref(g) if want_gbest else None, _stream()))
        return g.value if want_gbest else None

    def pso_get_state(self, x=None, v=None, p=None, pf=None, order=None, gk=None):
        self._check(self._L.pso_get_state(self._h, _ptr(x), _ptr(v), _ptr(p), _ptr(pf),
                                          _ptr(order), _ptr(gk), _stream()))

    def pso_set_state(self, x, v, p, pf, g, k):
        self._check(self._L.pso_set_state(self._h, _ptr(x), _ptr(v), _ptr(p), _ptr(pf), int(g),
                                          int(k), _stream()))
