"""The parity bar of a GPU misfit against the oracle's, in one place.

The method's accuracy target is 1e-4 relative L2 on traces and misfits.  A
misfit phi = 1/2 |r|^2 (r = d - d_obs) is a function of the traces, so the
error that traces within 1e-4 relative L2 can put on it is, to both orders,
|dphi| <= 1e-4 |r| |d| + 1/2 (1e-4 |d|)^2, with |d| <= |r| + |d_obs|.  For a
residual of at least 10 % of the observed data that bound is looser than
1e-4 relative on phi itself, so there the relative bar applies as written;
below it (near the optimum, where phi is a small difference of large traces
and 1e-4 relative on phi would ask the traces for ~1e-7) the bar is the bound
the trace bar implies.
"""
import math

TOL = 1e-4


def misfit_bound(ref: float, E: float) -> float:
    """Largest allowed |phi_gpu - phi_ref| for an oracle misfit `ref` and
    observed-data energy E = 1/2 |d_obs|^2."""
    if ref >= 1e-2 * E:                  # |r| >= 10 % |d_obs|
        return TOL * ref
    r = math.sqrt(2.0 * max(ref, 0.0))
    d = r + math.sqrt(2.0 * E)
    return TOL * r * d + 0.5 * (TOL * d) ** 2


def misfit_ok(got: float, ref: float, E: float) -> bool:
    return abs(got - ref) <= misfit_bound(ref, E)
