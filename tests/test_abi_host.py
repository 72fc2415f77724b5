"""CPU-only checks of the C ABI: the library loads, exports every function
that include/lbmd.h declares, sizes workspaces and rejects bad parameters
without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_0710_1272_gb300 as lb
import seeded_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbmd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = lb.load()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert L.lbmd_version() >> 16 == 1


def _ws(p, **kw):
    cp, keep = lb.make_params(p, **kw)
    return lb.lbmd_workspace_size(cp)


def test_workspace_covers_two_population_buffers():
    for storage, es in (("f32", 4), ("f16", 2), ("bf16", 2)):
        p = dict(si.paper_translocation(0), storage=storage)
        pos = np.zeros((400, 3)) + 130.0
        n = _ws(p, init_pos=pos)
        V = 256 * 128 * 128
        # two population buffers, the 4-byte link mask and the 4-byte spread
        # owner of every node, plus at most 80 MiB of geometry, bead buffers,
        # impulse sums and staging
        base = 2 * 19 * V * es + 4 * V + 4 * V
        assert base <= n <= base + 80 * 2 ** 20


def test_inplace_streaming_keeps_one_population_buffer():
    pos = np.zeros((400, 3)) + 130.0
    for storage, es in (("f32", 4), ("f16", 2)):
        p = dict(si.paper_translocation(0), storage=storage)
        pull = _ws(p, init_pos=pos)
        aa = _ws(dict(p, streaming="aa"), init_pos=pos)
        Vp = 256 * 128 * 128  # already a multiple of 64
        assert pull - aa == 19 * Vp * es


def test_unknown_streaming_rejected():
    p = si.small_translocation(0, n_beads=4)
    pos = si.saw_chain(p, 0)
    cp, keep = lb.make_params(p, init_pos=pos)
    cp.streaming = 7
    with pytest.raises(lb.LbmdError) as e:
        lb.lbmd_workspace_size(cp)
    assert e.value.code == lb.lbmd.LBMD_EINVAL and "streaming" in str(e.value)


@pytest.mark.parametrize("bad,msg", [
    (dict(tau=0.5), "tau"),
    (dict(nx=0), "box"),
    (dict(wall_x=99), "wall_x"),
    (dict(pore_d=40), "pore_d"),
    (dict(n_beads=1025), "n_beads"),
    (dict(storage="f64"), None),
    (dict(md_substeps=0), "md_substeps"),
    (dict(n_beads=0, hydrodynamics=0), "solvent_free"),
])
def test_invalid_parameters_rejected(bad, msg):
    p = dict(si.small_translocation(0, n_beads=4))
    p.update(bad)
    pos = np.tile([[18.0, 7.0, 7.0]], (max(int(p.get("n_beads", 4)), 1), 1))
    if msg is None:
        with pytest.raises(KeyError):
            _ws(p, init_pos=pos[: p["n_beads"]])
        return
    with pytest.raises(lb.LbmdError) as e:
        _ws(p, init_pos=pos[: min(p["n_beads"], 1025)])
    assert e.value.code == lb.lbmd.LBMD_EINVAL
    assert msg in str(e.value)


def test_missing_bead_positions_take_the_seeded_start():
    """init_pos == NULL is valid: the library draws its own start at create."""
    p = si.small_translocation(0, n_beads=4)
    assert _ws(p) == _ws(p, init_pos=si.saw_chain(p, 0))


def test_non_chain_topology_unsupported():
    p = si.small_translocation(0, n_beads=4)
    pos = si.saw_chain(p, 0)
    bonds = (np.array([0, 1, 0]), np.array([1, 2, 3]), np.full(3, 1.2))
    with pytest.raises(lb.LbmdError) as e:
        _ws(p, init_pos=pos, bonds=bonds)
    assert e.value.code == lb.lbmd.LBMD_EUNSUPPORTED
    ok = (np.array([0, 1, 2]), np.array([1, 2, 3]), np.array([1.2, 1.1, 1.3]))
    assert _ws(p, init_pos=pos, bonds=ok) > 0


def test_null_context_is_an_error():
    L = lb.load()
    assert L.lbmd_step(None, 1) == lb.lbmd.LBMD_EINVAL
    assert L.lbmd_destroy(None) == 0
    assert L.lbmd_strerror(-3) == b"CUDA error"


def _ens_ws(members, starts):
    arr = (lb.lbmd.lbmd_params * len(members))()
    keep = []
    for k, (p, pos) in enumerate(zip(members, starts)):
        cp, kk = lb.make_params(p, init_pos=pos)
        arr[k] = cp
        keep.append(kk)
    return lb.lbmd.lbmd_ensemble_workspace_size(arr)


def test_ensemble_workspace_holds_every_member():
    members, starts = si.ragged_ensemble(6, seed=3)
    n = _ens_ws(members, starts)
    singles = sum(_ws(p, init_pos=pos) for p, pos in zip(members, starts))
    pops = sum(2 * 19 * p["nx"] * p["ny"] * p["nz"] * 4 for p in members)
    # every member's buffers, but one shared read-out staging area
    assert pops < n < singles + 8 * 2 ** 20


@pytest.mark.parametrize("change,code", [
    (lambda m: m[1].update(storage="f16"), lb.lbmd.LBMD_EUNSUPPORTED),
    (lambda m: m[2].update(forcing="guo"), lb.lbmd.LBMD_EUNSUPPORTED),
    (lambda m: m[0].update(tau=0.4), lb.lbmd.LBMD_EINVAL),
    (lambda m: m[1].update(streaming="aa"), lb.lbmd.LBMD_EUNSUPPORTED),
])
def test_ensemble_rejects_mixed_or_bad_members(change, code):
    members, starts = si.ragged_ensemble(3, seed=4)
    change(members)
    with pytest.raises(lb.LbmdError) as e:
        _ens_ws(members, starts)
    assert e.value.code == code


def test_ensemble_rejects_empty_and_beadless():
    L = lb.load()
    n = ctypes.c_size_t()
    assert L.lbmd_ensemble_workspace_size(None, 0, ctypes.byref(n)) == lb.lbmd.LBMD_EINVAL
    p = dict(si.periodic_solvent(16))
    cp, keep = lb.make_params(p)
    arr = (lb.lbmd.lbmd_params * 1)(cp)
    assert L.lbmd_ensemble_workspace_size(arr, 1, ctypes.byref(n)) == lb.lbmd.LBMD_EINVAL
    assert L.lbmd_ensemble_workspace_size(arr, 0, ctypes.byref(n)) == lb.lbmd.LBMD_EINVAL
