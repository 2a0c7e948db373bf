"""The asynchronous state copies (cgks_set_state_async, cgks_get_state_async,
cgks_sync): two contexts on two streams, driven from one host thread with
one context's copies enqueued while the other steps, give bit for bit the
results of the waiting calls, in both forms, from page-locked host memory
and from device memory; buffers of the wrong size or type are refused."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_08965_gb300 as p
    p.lib()
    return p


KW = dict(dim=3, n=(12, 10, 8), lo=(0, 0, 0), hi=(2 * math.pi,) * 3, mu=1 / 1600, prandtl=0.72, tau_mode=2)


def tgv(x, y, z):
    return synth.taylor_green_3d(x, y, z)


@pytest.mark.parametrize("precision", [0, 1])
def test_async_copies_interleaved(cg, precision):
    import torch
    m = cg.Mesh(precision=precision, **KW)
    m.init(tgv)
    inputs = []
    for _ in range(4):
        inputs.append(m.get_state()[0].copy())
        m.step(1)
    want = []
    for s in inputs:
        m.set_state(s, 0.0)
        m.step(1)
        want.append(m.get_state()[0].copy())
    m.close()

    pins = [torch.from_numpy(s).pin_memory() for s in inputs]
    outs = [torch.empty(s.shape, dtype=torch.float64, pin_memory=True) for s in inputs]
    lanes = [cg.Mesh(precision=precision, stream=torch.cuda.Stream(), **KW) for _ in range(2)]
    lanes[0].set_state_async(pins[0])
    lanes[1].set_state_async(pins[1])
    for i in range(4):
        ln = lanes[i % 2]
        ln.step(1)
        ln.get_state_async(outs[i])
        if i + 2 < 4:
            ln.set_state_async(pins[i + 2])
    for ln in lanes:
        ln.sync()
    for i in range(4):
        assert np.array_equal(outs[i].numpy(), want[i]), i

    # device buffers, and the time the asynchronous set gives
    d_in = torch.from_numpy(inputs[3]).cuda()
    d_out = torch.empty_like(d_in)
    lanes[0].set_state_async(d_in, 0.25)
    t, dt = lanes[0].step(1)
    lanes[0].get_state_async(d_out)
    lanes[0].sync()
    assert np.array_equal(d_out.cpu().numpy(), want[3]) and t == 0.25 + dt
    for ln in lanes:
        ln.close()


def test_async_copies_refuse_bad_buffers(cg):
    import torch
    m = cg.Mesh(**KW)
    n = m.nf * m.nv * m.ncell
    with pytest.raises(ValueError):
        m.set_state_async(np.zeros(n - 1))
    with pytest.raises(ValueError):
        m.set_state_async(np.zeros(n, dtype=np.float32))
    with pytest.raises(ValueError):
        m.get_state_async(torch.empty(n + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        m.get_state_async(np.zeros((2, n))[:, 0])   # not contiguous
    m.close()
