"""Run-to-run determinism of the coupled step.

The only concurrent additions of the step are those of the bead spread
(stage 3, Eq. 10: several beads hand impulse to the same node).  They are
summed per node in 64-bit fixed point at an owner chosen by atomicMin, and
the owner adds the source to the populations once, so the order in which the
GPU happens to run the atomics does not reach the result: two contexts built
from the same parameters and stepped the same way hold the same bits.  The
cases run at the benchmark's eps = 1, where the bead dynamics are chaotic and
a single differing ulp grows to a visible difference within a few hundred
steps.
"""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _lb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0710_1272_gb300 as lb
    return lb


def _same(a, b):
    np.testing.assert_array_equal(a.populations(), b.populations())
    ra, va = a.beads()
    rb, vb = b.beads()
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(va, vb)
    ua, ja = a.bead_aux()
    ub, jb = b.bead_aux()
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(ja, jb)
    assert a.status() == b.status()


@pytest.mark.parametrize("streaming", ["pull", "aa"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_two_contexts_1000_steps_bit_identical(streaming, storage):
    lb = _lb()
    p = si.small_translocation(3)
    pos = si.saw_chain(p, 3)
    q = dict(p, streaming=streaming, storage=storage)
    a = lb.Simulation(q, init_pos=pos)
    b = lb.Simulation(q, init_pos=pos)
    # graph replays of several lengths on one side, single steps on the other
    for n in (1, 16, 2, 181, 800):
        a.step(n)
        for _ in range(n):
            b.step(1)
        _same(a, b)
    assert a.status()["step"] == 1000


def test_in_place_and_pull_bit_identical_with_beads():
    """With the order-independent spread, in-place streaming equals the
    two-buffer path bit for bit with a coupled chain as well."""
    lb = _lb()
    p = si.small_translocation(4)
    pos = si.saw_chain(p, 4)
    for storage in ("f32", "f16"):
        a = lb.Simulation(dict(p, storage=storage, streaming="aa"), init_pos=pos)
        b = lb.Simulation(dict(p, storage=storage), init_pos=pos)
        for n in (1, 1, 16, 3, 300):
            a.step(n)
            b.step(n)
            _same(a, b)


def test_benchmark_box_bit_identical():
    """The 256 x 128 x 128, N = 400 benchmark workload in its launch
    configuration (graph replay), 100 steps twice."""
    lb = _lb()
    p = si.paper_translocation(0)
    pos = si.saw_chain(p, 0)
    a = lb.Simulation(p, init_pos=pos)
    a.step(100)
    fa = a.populations()
    ra = a.beads()
    sa = a.status()
    a.close()
    b = lb.Simulation(p, init_pos=pos)
    b.step(100)
    np.testing.assert_array_equal(fa, b.populations())
    np.testing.assert_array_equal(ra[0], b.beads()[0])
    np.testing.assert_array_equal(ra[1], b.beads()[1])
    assert sa == b.status()


def test_benchmark_box_records_and_apply_conversion_agree():
    """The FP32 benchmark box converts the spread sums in k_spread_finalize
    (its stream-collide sets the step); an ensemble converts them in its apply
    kernel.  Both convert the same fixed-point sums once per node: the same
    box as a one-member ensemble holds the single box's bits."""
    lb = _lb()
    p = si.paper_translocation(0)
    pos = si.saw_chain(p, 0)
    a = lb.Simulation(p, init_pos=pos)
    a.step(40)
    fa = a.populations()
    ra, va = a.beads()
    a.close()
    ens = lb.Ensemble([p], [pos])
    ens.step(40)
    np.testing.assert_array_equal(ens.populations(0), fa)
    re, ve = ens.beads(0)
    np.testing.assert_array_equal(re, ra)
    np.testing.assert_array_equal(ve, va)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_ensemble_1000_steps_bit_identical(storage):
    lb = _lb()
    specs = [
        dict(nx=32, ny=16, nz=16, wall_x=16, pore_d=3, n_beads=20, seed=21),
        dict(nx=48, ny=20, nz=13, wall_x=24, pore_d=5, n_beads=37, seed=22),
        dict(nx=40, ny=17, nz=17, wall_x=20, pore_d=5, n_beads=5, seed=23, tau=0.8),
        dict(nx=64, ny=24, nz=24, wall_x=32, pore_d=5, n_beads=70, seed=24, f_drive=0.05),
        dict(nx=36, ny=16, nz=16, wall_x=18, pore_d=3, n_beads=1, seed=25),
    ]
    members, starts = [], []
    for sp in specs:
        m = dict(si.BASE)
        m.update(sp, storage=storage)
        members.append(m)
        starts.append(si.saw_chain(m, m["seed"]))
    a = lb.Ensemble(members, starts)
    b = lb.Ensemble(members, starts)
    a.step(1000)
    for n in (1, 15, 984):
        b.step(n)
    ra, rb = a.results(), b.results()
    for key in ra:
        np.testing.assert_array_equal(ra[key], rb[key])
    for k in range(len(members)):
        np.testing.assert_array_equal(a.populations(k), b.populations(k))
        np.testing.assert_array_equal(a.beads(k)[0], b.beads(k)[0])
        np.testing.assert_array_equal(a.beads(k)[1], b.beads(k)[1])
