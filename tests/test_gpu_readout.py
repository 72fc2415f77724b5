"""Asynchronous host read-out (lbmd_read_beads_async): the block it delivers
into page-locked memory equals the synchronous read-outs, also when it is
double-buffered behind the following steps."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0710_1272_gb300 as lb
    return torch, lb


def _block(torch, lb, N):
    return torch.empty(lb.bead_block_bytes(N), dtype=torch.uint8, pin_memory=True)


@pytest.mark.parametrize("streaming", ["pull", "aa"])
def test_async_readout_equals_synchronous(streaming):
    torch, lb = _gpu()
    p = si.small_translocation(0)
    pos0 = si.saw_chain(p, 0)
    sim = lb.Simulation(dict(p, streaming=streaming), init_pos=pos0)
    N = p["n_beads"]
    blk = _block(torch, lb, N)
    sim.step(7)
    lb.lbmd_read_beads_async(sim.ctx, blk.data_ptr(), blk.numel())
    sim.stream.synchronize()
    status, r, v = lb.decode_bead_block(blk.numpy(), N)
    rs, vs = sim.beads()
    np.testing.assert_array_equal(r, rs)
    np.testing.assert_array_equal(v, vs)
    assert status == sim.status()


def test_async_readout_double_buffered_behind_steps():
    """Step k+1 is enqueued before the host waits for the read-out of step k:
    every block still holds its own step's state."""
    torch, lb = _gpu()
    p = si.small_translocation(1)
    pos0 = si.saw_chain(p, 1)
    sim = lb.Simulation(p, init_pos=pos0)
    ref = lb.Simulation(p, init_pos=pos0)
    N = p["n_beads"]
    blocks = [_block(torch, lb, N) for _ in range(2)]
    events = [torch.cuda.Event(), torch.cuda.Event()]
    seen = []

    def take(k):
        events[k % 2].synchronize()
        seen.append(lb.decode_bead_block(blocks[k % 2].numpy().copy(), N))

    for k in range(6):
        lb.lbmd_step(sim.ctx, 1)
        lb.lbmd_read_beads_async(sim.ctx, blocks[k % 2].data_ptr(), blocks[k % 2].numel())
        events[k % 2].record(sim.stream)
        if k > 0:
            take(k - 1)
    take(5)
    for k, (status, pos, vel) in enumerate(seen):
        ref.step(1)
        assert status["step"] == k + 1
        rr, vr = ref.beads()
        np.testing.assert_array_equal(pos, rr)
        np.testing.assert_array_equal(vel, vr)


def test_async_readout_checks_size_and_works_without_beads():
    torch, lb = _gpu()
    sim = lb.Simulation(dict(nx=32, ny=16, nz=16))
    blk = _block(torch, lb, 0)
    sim.step(3)
    with pytest.raises(lb.LbmdError):
        lb.lbmd_read_beads_async(sim.ctx, blk.data_ptr(), 16)
    lb.lbmd_read_beads_async(sim.ctx, blk.data_ptr(), blk.numel())
    sim.stream.synchronize()
    assert lb.decode_bead_block(blk.numpy(), 0)[0]["step"] == 3


def test_async_readout_into_pageable_memory():
    """Memory the device cannot address takes the staging buffer and a copy;
    the block is the same as the one written straight into pinned memory."""
    torch, lb = _gpu()
    p = si.small_translocation(2)
    sim = lb.Simulation(p, init_pos=si.saw_chain(p, 2))
    sim.step(7)
    N = p["n_beads"]
    pageable = np.zeros(lb.bead_block_bytes(N), dtype=np.uint8)
    pinned = _block(torch, lb, N)
    lb.lbmd_read_beads_async(sim.ctx, pageable.ctypes.data, pageable.nbytes)
    lb.lbmd_read_beads_async(sim.ctx, pinned.data_ptr(), pinned.numel())
    sim.stream.synchronize()
    np.testing.assert_array_equal(pageable, pinned.numpy())
    status, pos, vel = lb.decode_bead_block(pageable, N)
    r, v = sim.beads()
    assert status["step"] == 7
    np.testing.assert_array_equal(pos, r)
    np.testing.assert_array_equal(vel, v)


@pytest.mark.parametrize("pinned", [True, False])
def test_step_read_async_equals_step_then_read(pinned):
    """lbmd_step_read_async (one graph of the step and its read-out, or the
    two separate calls for memory the device cannot address) delivers, block
    for block, what lbmd_step(1) + lbmd_read_beads_async deliver, also
    double-buffered behind the following steps and across both buffers."""
    torch, lb = _gpu()
    p = si.small_translocation(3)
    pos0 = si.saw_chain(p, 3)
    a = lb.Simulation(p, init_pos=pos0)
    b = lb.Simulation(p, init_pos=pos0)
    N = p["n_beads"]
    if pinned:
        blocks = [_block(torch, lb, N) for _ in range(2)]
        view = [blk.numpy() for blk in blocks]
        ptr = [blk.data_ptr() for blk in blocks]
    else:
        view = [np.zeros(lb.bead_block_bytes(N), dtype=np.uint8) for _ in range(2)]
        ptr = [v.ctypes.data for v in view]
    ref = _block(torch, lb, N)
    events = [torch.cuda.Event(), torch.cuda.Event()]
    for k in range(7):
        lb.lbmd_step_read_async(a.ctx, ptr[k % 2], len(view[k % 2]))
        events[k % 2].record(a.stream)
        lb.lbmd_step(b.ctx, 1)
        lb.lbmd_read_beads_async(b.ctx, ref.data_ptr(), ref.numel())
        b.stream.synchronize()
        events[k % 2].synchronize()
        np.testing.assert_array_equal(view[k % 2], ref.numpy())
        assert lb.decode_bead_block(view[k % 2], N)[0]["step"] == k + 1
    # the graphs of both buffers and the plain path interleave
    a.step(3)
    b.step(3)
    np.testing.assert_array_equal(a.populations(), b.populations())
    with pytest.raises(lb.LbmdError):
        lb.lbmd_step_read_async(a.ctx, ptr[0], 16)
