"""Checkpoint and resume through empso_save / empso_load.

A run interrupted after G1 generations, saved, and resumed in a fresh context
must continue bit for bit as the uninterrupted run: the swarm state is FP64
and every random number is a Philox counter of (seed, generation, particle,
dimension), so nothing else carries over.  With the surrogate the network
parameters, Adam moments and step, replay buffer and sampling counter are
restored too.  Invalid files and mismatched contexts are host-side errors.
"""
import os

import numpy as np
import pytest

from paper_1905_12795_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_12795_gb300 import binding
    binding.load()
    return binding


NX, NZ, H = 41, 31, 10.0


def _problem(B, P=48, seed=9, surrogate=False):
    grid = B.make_grid(NX, NZ, H, H, 5, 4, 0.25, 12.0, 1500.0, 3500.0)
    rec = synth.receiver_line(NX, H, 20.0)
    pso = B.EmpsoPso(P, 32, 1.2, 2.9, 0.5, 0.3, 0.25, 2, 1, seed)
    ctx = B.Context([grid], rec, pso, 1500.0, 3500.0)
    if surrogate:
        ctx.surrogate_init(hidden=64, capacity=256, lr=1e-3, seed=seed)
    sh = B.make_shots(synth.shot_line(2, (NX - 1) * H, 20.0), [0, 0], [NX, NX])
    _, nt = ctx.grid_info(0)
    # observed data of a two-layer model through this library: both runs of a
    # comparison see the same buffer, nothing is compared with the oracle here
    true = torch.tensor(synth.two_layer_model(NX, NZ, H, 1500.0, 2800.0, 150.0),
                        dtype=torch.float32, device="cuda").reshape(1, NZ, NX).contiguous()
    dobs = torch.zeros(2 * nt * NX, device="cuda")
    ctx.forward_traces(true, sh, dobs)
    return ctx, sh, dobs


def _state(ctx, P, D=32):
    x = torch.zeros(P, D, dtype=torch.float64, device="cuda")
    v, p = torch.zeros_like(x), torch.zeros_like(x)
    pf = torch.zeros(P, dtype=torch.float64, device="cuda")
    order = torch.zeros(P, dtype=torch.int32, device="cuda")
    gk = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.pso_get_state(x, v, p, pf, order, gk)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (x, v, p, pf, order, gk)]


def _equal_states(a, b):
    for u, w in zip(a, b):
        assert np.array_equal(u, w)


def test_resume_plain_generations_bit_exact(B, tmp_path):
    P, G1, G2 = 48, 3, 4
    path = str(tmp_path / "swarm.ck")
    a, sh, dobs = _problem(B, P)
    a.pso_init()
    mis = torch.zeros(P, dtype=torch.float64, device="cuda")
    for _ in range(G1):
        a.generation(sh, dobs, mis)
    a.save(path)
    assert os.path.exists(path) and not os.path.exists(path + ".tmp")
    for _ in range(G2):
        a.generation(sh, dobs, mis)
    ref, ref_mis = _state(a, P), mis.cpu().numpy()
    a.close()

    b, sh, dobs = _problem(B, P)
    b.load(path)
    assert _state(b, P)[5][1] == G1
    mis_b = torch.zeros(P, dtype=torch.float64, device="cuda")
    for _ in range(G2):
        b.generation(sh, dobs, mis_b)
    _equal_states(_state(b, P), ref)
    assert np.array_equal(mis_b.cpu().numpy(), ref_mis)
    b.close()


@pytest.mark.parametrize("overlap", [False, True])
def test_resume_surrogate_generations_bit_exact(B, tmp_path, overlap):
    """Also with training beside the modelling (second stream): the result
    does not depend on how the two streams interleave."""
    P = 48
    path = str(tmp_path / "sur.ck")
    kw = dict(keep_frac=0.25, warm=P, train_steps=8, batch=32)
    a, sh, dobs = _problem(B, P, seed=4, surrogate=True)
    a.surrogate_set_overlap(overlap)
    a.pso_init()
    mis = torch.zeros(P, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a.surrogate_generation(sh, dobs, misfit_out=mis, **kw)
    a.save(path)
    for _ in range(3):
        a.surrogate_generation(sh, dobs, misfit_out=mis, **kw)
    ref = _state(a, P)
    npar = a.surrogate_n_params()
    wa = torch.zeros(npar, device="cuda")
    a.surrogate_get(wa)
    a.close()

    b, sh, dobs = _problem(B, P, seed=4, surrogate=True)
    b.surrogate_set_overlap(overlap)
    b.load(path)
    for _ in range(3):
        b.surrogate_generation(sh, dobs, misfit_out=mis, **kw)
    _equal_states(_state(b, P), ref)
    wb = torch.zeros(npar, device="cuda")
    b.surrogate_get(wb)
    assert torch.equal(wa, wb)
    b.close()


def test_checkpoint_errors(B, tmp_path):
    P = 16
    path = str(tmp_path / "s.ck")
    a, _, _ = _problem(B, P)
    a.pso_init()
    a.save(path)
    before = _state(a, P)
    with pytest.raises(B.EmpsoError) as e:
        a.load(str(tmp_path / "missing.ck"))
    assert e.value.status == 8
    # one flipped byte: checksum
    raw = bytearray(open(path, "rb").read())
    raw[40] ^= 0x10
    bad = str(tmp_path / "bad.ck")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(B.EmpsoError) as e:
        a.load(bad)
    assert e.value.status == 8
    # truncated
    open(bad, "wb").write(bytes(raw[:100]))
    with pytest.raises(B.EmpsoError) as e:
        a.load(bad)
    assert e.value.status == 8
    _equal_states(_state(a, P), before)   # unchanged by the failed loads
    # another swarm size or seed
    c, _, _ = _problem(B, P + 1)
    with pytest.raises(B.EmpsoError) as e:
        c.load(path)
    assert e.value.status == 1
    c.close()
    d, _, _ = _problem(B, P, seed=10)
    with pytest.raises(B.EmpsoError) as e:
        d.load(path)
    assert e.value.status == 1
    d.close()
    # a surrogate checkpoint needs an initialised surrogate
    s, _, _ = _problem(B, P, surrogate=True)
    s.pso_init()
    s.save(path)
    s.close()
    with pytest.raises(B.EmpsoError) as e:
        a.load(path)
    assert e.value.status == 7
    a.close()
