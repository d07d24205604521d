"""GPU parity of the observed-data low-pass / resampling against the FP64
oracle.  The taps are FP32 (arguments formed in FP64) and each output sums a
few thousand FP32 products: 2e-5 of the trace's largest value."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_12795_gb300 import binding
    binding.load()
    return binding


def _ctx(B):
    grid = B.make_grid(11, 11, 10.0, 10.0, 0, 2, 0.05, 10.0, 1500.0, 2000.0)
    return B.Context([grid], [[0.0, 0.0]])


@pytest.mark.parametrize("S,nt_in,nrec,dt_in,nt_out,dt_out,fc,W", [
    (3, 701, 37, 1e-3, 333, 2.1e-3, 6.0, 0.3),     # resample to a coarser axis, ragged sizes
    (2, 500, 300, 2e-3, 500, 2e-3, 6.0, 0.25),     # plain low-pass, 2 receiver passes
    (1, 1200, 5, 6.25e-4, 1, 1e-3, 4.6, 0.2),      # a single output sample
    (2, 64, 33, 4e-3, 97, 2.5e-3, 10.0, 0.6),      # window longer than the record
])
def test_lowpass_matches_oracle(B, S, nt_in, nrec, dt_in, nt_out, dt_out, fc, W):
    rng = np.random.default_rng(nt_in + nrec)
    x = rng.normal(size=(S, nt_in, nrec)).astype(np.float32)
    ref = oracle.lowpass(x.astype(np.float64), dt_in, nt_out, dt_out, fc, W)
    ctx = _ctx(B)
    out = torch.full((S, nt_out, nrec), np.nan, device="cuda")
    ctx.lowpass(torch.tensor(x, device="cuda"), dt_in, out, dt_out, fc, W)
    got = out.cpu().numpy()
    for s in range(S):
        scale = max(np.max(np.abs(ref[s])), 1e-30)
        assert np.max(np.abs(got[s] - ref[s])) < 2e-5 * scale
    ctx.close()


def test_lowpass_errors(B):
    ctx = _ctx(B)
    x = torch.zeros(1, 100, 4, device="cuda")
    with pytest.raises(B.EmpsoError) as e:
        ctx.lowpass(x, 1e-3, x, 1e-3, 6.0, 0.1)           # in place
    assert e.value.status == 1
    with pytest.raises(B.EmpsoError) as e:
        ctx.lowpass(x, 1e-3, torch.zeros(1, 10, 4, device="cuda"), 1e-3, -1.0, 0.1)
    assert e.value.status == 1
    with pytest.raises(B.EmpsoError) as e:
        ctx.lowpass(x, 1e-5, torch.zeros(1, 10, 4, device="cuda"), 1e-3, 6.0, 5.0)
    assert e.value.status == 6                            # window beyond shared memory
    ctx.close()
