"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/empso.h declares; the binding's structures match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "empso.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s*([A-Za-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_12795_gb300 import build
    path = build.build()
    import torch  # noqa: F401  (CUDA runtime first, as the binding does)
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("empso_create", "eval_fitness", "pso_init", "pso_step", "forward_traces"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    from paper_1905_12795_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared_functions()


def test_struct_layouts():
    from paper_1905_12795_gb300 import binding as B
    # sizes follow the C layout of empso.h (natural alignment, no packing)
    assert ctypes.sizeof(B.EmpsoGrid) == 14 * 4
    assert ctypes.sizeof(B.EmpsoShot) == 6 * 4
    assert ctypes.sizeof(B.EmpsoPso) == 8 + 5 * 8 + 8 + 8


def test_status_strings(lib):
    lib.empso_status_string.restype = ctypes.c_char_p
    assert lib.empso_status_string(0) == b"ok"
    assert lib.empso_status_string(6) == b"unsupported"


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1905_12795_gb300 import binding as B
    grid = B.make_grid(41, 31, 10.0, 10.0, 5, 4, 0.2, 10.0, 1500.0, 3000.0)
    with pytest.raises(B.EmpsoError) as e:
        B.Context([grid], [[0.0, 0.0]])
    assert e.value.status == 3


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_1905_12795_gb300 import binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "lib_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        B.load()


def test_host_functions_through_the_binding(lib):
    """The two entry points that touch no device run here: the depth-dependent
    ranges equal the oracle's, and the kernel-name query is safe on NULL."""
    import numpy as np
    from paper_1905_12795_gb300 import binding as B
    import oracle
    level_z = np.array([50.0, 150.0, 300.0, 500.0])
    counts = [5, 3, 2, 1]
    lo, hi = B.level_bounds(level_z, counts, 1600.0, 3400.0, 0.2, 0.3, 0.25, 0.15)
    lo_r, hi_r = oracle.level_bounds(level_z, counts, 1600.0, 3400.0, 0.2, 0.3, 0.25, 0.15)
    assert np.allclose(lo, lo_r, rtol=1e-15) and np.allclose(hi, hi_r, rtol=1e-15)
    with pytest.raises(B.EmpsoError):
        B.level_bounds(level_z, [5, 0, 2, 1], 1600.0, 3400.0, 0.2, 0.3, 0.25, 0.15)
    assert B.load().empso_last_kernel_name(None) == b""
    lib.empso_status_string.restype = ctypes.c_char_p
    assert lib.empso_status_string(8) == b"file error"


@pytest.mark.parametrize("order,nx,nz,h,T,vmax", [(2, 37, 29, 10.0, 0.3, 3200.0),
                                                   (4, 101, 101, 10.0, 0.5, 2625.0),
                                                   (8, 461, 151, 20.0, 3.0, 4700.0),
                                                   (8, 921, 301, 10.0, 4.0, 4700.0),
                                                   (16, 301, 121, 10.0, 2.0, 4700.0)])
def test_context_free_time_axis_matches_oracle(lib, order, nx, nz, h, T, vmax):
    """Host logic only (no device work): the library's CFL time axis for a
    grid equals the oracle's, and invalid grids are refused with the codes
    empso_create uses."""
    import oracle
    from paper_1905_12795_gb300 import binding as B
    g = B.make_grid(nx, nz, h, h, 10, order, T, 6.0, 1500.0, vmax)
    dt, nt = B.time_axis(g)
    dt_o, nt_o = oracle.time_axis(order, h, h, vmax, T)
    assert nt == nt_o and dt == pytest.approx(dt_o, rel=1e-6)
    with pytest.raises(B.EmpsoError) as e:
        B.time_axis(B.make_grid(nx, nz, h, h, 10, 6, T, 6.0, 1500.0, vmax))
    assert e.value.status == 6
    with pytest.raises(B.EmpsoError) as e:
        B.time_axis(B.make_grid(nx, nz, h, h, 10, order, T, 6.0, 2000.0, 1900.0))
    assert e.value.status == 1


def test_misfit_rule_is_the_trace_bar_propagated():
    """The misfit parity bar (tests/misfit_rule.py) against its definition:
    traces perturbed by exactly 1e-4 of their norm, in the worst direction
    (along the residual), change the misfit by at most the bound, and the
    bound is 1e-4 relative once the residual reaches 10 % of the data."""
    import numpy as np
    from misfit_rule import misfit_bound
    rng = np.random.default_rng(3)
    dobs = rng.normal(size=5000)
    E = 0.5 * float(dobs @ dobs)
    for frac in (0.0, 1e-3, 1e-2, 0.05, 0.099, 0.2, 1.0, 3.0):
        r = rng.normal(size=5000)
        r *= frac * np.linalg.norm(dobs) / max(np.linalg.norm(r), 1e-300)
        d = dobs + r
        phi = 0.5 * float(r @ r)
        u = r / np.linalg.norm(r) if frac > 0 else d / np.linalg.norm(d)
        dd = d + 1e-4 * np.linalg.norm(d) * u
        phi2 = 0.5 * float((dd - dobs) @ (dd - dobs))
        if phi < 1e-2 * E:
            assert abs(phi2 - phi) <= misfit_bound(phi, E) * (1 + 1e-9)
        else:
            assert misfit_bound(phi, E) == pytest.approx(1e-4 * phi)
