"""GPU parity of the ensemble path (many realisations in one set of launches):
every realisation must take exactly the steps the FP64 oracle takes for its
own parameters, within the tolerances of the single-box parity tests
(populations 1e-5 relative after one step, beads 1e-4 over 100 steps), and
must stop at its own translocation step or at the step cap.

The members are ragged on purpose: different boxes (x extents that are not a
multiple of the 32-node tile, odd y and z), chain lengths in different MD
block-size groups, pore sizes, seeds and bead parameters.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu

GPU_ONLY = ("storage", "init_tg_amp", "diag_every", "diag_capacity")
PAPER_EPS = 2e-3


def _lb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0710_1272_gb300 as lb
    return lb


def rel_err(fg, fo):
    m = fo != 0
    assert np.all(fg[~m] == 0)
    return float(np.max(np.abs(fg[m].astype(np.float64) - fo[m]) / np.abs(fo[m])))


def ragged_members(storage="f32", eps=PAPER_EPS):
    specs = [
        dict(nx=32, ny=16, nz=16, wall_x=16, pore_d=3, n_beads=20, seed=11),
        dict(nx=48, ny=20, nz=13, wall_x=24, pore_d=5, n_beads=37, seed=12, gamma=0.2),
        dict(nx=40, ny=17, nz=17, wall_x=20, pore_d=3, n_beads=5, seed=13, tau=0.8),
        dict(nx=64, ny=24, nz=24, wall_x=32, pore_d=5, n_beads=70, seed=14, f_drive=0.05),
        dict(nx=36, ny=16, nz=16, wall_x=18, pore_d=3, n_beads=1, seed=15),
    ]
    members, starts = [], []
    for sp in specs:
        p = dict(si.BASE)
        p.update(sp)
        p["lj_eps"] = eps
        starts.append(si.saw_chain(p, p["seed"]))
        p["storage"] = storage
        members.append(p)
    return members, starts


def oracle_of(p, pos):
    return oracle.OracleSim({k: v for k, v in p.items() if k not in GPU_ONLY}, init_pos=pos)


def advance_like_member(sim, n, running=0):
    """Step a reference (oracle or single-box context) n steps, one at a time,
    stopping as an ensemble member does once its state leaves RUNNING."""
    for _ in range(n):
        if sim.status()["state"] != running:
            break
        sim.step(1)


def test_ensemble_members_match_oracle_one_step():
    lb = _lb()
    members, starts = ragged_members()
    ens = lb.Ensemble(members, starts)
    ens.step(1)
    for k, (p, pos) in enumerate(zip(members, starts)):
        orc = oracle_of(p, pos)
        orc.step(1)
        assert rel_err(ens.populations(k), orc.populations()) < 1e-5, k
        assert np.abs(ens.beads(k)[0] - orc.beads()[0]).max() < 1e-6, k


def test_ensemble_bead_trajectories_100_steps():
    lb = _lb()
    members, starts = ragged_members()
    ens = lb.Ensemble(members, starts)
    orcs = [oracle_of(p, pos) for p, pos in zip(members, starts)]
    for _ in range(10):
        ens.step(10)
        for k, orc in enumerate(orcs):
            advance_like_member(orc, 10, oracle.RUNNING)
            assert np.abs(ens.beads(k)[0] - orc.beads()[0]).max() < 1e-4, k
    res = ens.results()
    # the single bead starts in the pore mouth and crosses within 100 steps
    assert res["state"][4] == lb.TRANSLOCATED and res["steps"][4] < 100
    for k, orc in enumerate(orcs):
        st = orc.status()
        assert res["steps"][k] == st["step"], k
        assert res["n_trans"][k] == st["n_trans"] and res["state"][k] == st["state"], k
        assert res["t_transloc"][k] == st["t_transloc"], k


def same_state(ens, k, sim):
    """Ensemble member k and a single-box context hold the same bits."""
    assert np.array_equal(ens.populations(k), sim.populations()), k
    rg, vg = ens.beads(k)
    rs, vs = sim.beads()
    assert np.array_equal(rg, rs) and np.array_equal(vg, vs), k


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_ensemble_matches_single_box_path(storage):
    """Ensemble realisations against lbmd_step on the same parameters: the same
    collision, MD body and fixed-point spread, so the same bits in every
    storage type."""
    lb = _lb()
    members, starts = ragged_members(storage)
    ens = lb.Ensemble(members, starts)
    ens.step(25)
    for k, (p, pos) in enumerate(zip(members, starts)):
        sim = lb.Simulation(p, init_pos=pos)
        advance_like_member(sim, 25, lb.RUNNING)
        same_state(ens, k, sim)


def test_ensemble_runs_each_member_to_its_translocation():
    """Paper-like small boxes translocate in a few hundred steps.  Each member
    stops at its own completion step, which matches the oracle's within two
    steps (contractive dynamics at eps = 2e-3); a member that has stopped keeps
    its state while the others run on."""
    lb = _lb()
    members, starts = [], []
    for seed in range(4):
        p = si.small_translocation(seed)
        p["lj_eps"] = PAPER_EPS
        members.append(p)
        starts.append(si.saw_chain(p, seed))
    ens = lb.Ensemble(members, starts)
    ens.run(1200, check_every=64)
    res = ens.results()
    assert ens.live() == 0
    for k, (p, pos) in enumerate(zip(members, starts)):
        orc = oracle_of(p, pos)
        while orc.status()["state"] == oracle.RUNNING and orc.status()["step"] < 1200:
            orc.step(50)
        so = orc.status()
        assert so["state"] == oracle.TRANSLOCATED
        assert res["state"][k] == lb.TRANSLOCATED
        assert abs(int(res["t_transloc"][k]) - so["t_transloc"]) <= 2
        # stopped exactly at its completion step
        assert res["steps"][k] == res["t_transloc"][k]


def test_ensemble_step_cap_and_resume():
    """run() stops every member at the cap; a higher cap resumes them, also
    when the member's step parity differs from the ensemble's."""
    lb = _lb()
    members, starts = ragged_members()
    ens = lb.Ensemble(members, starts)
    ens.run(20, check_every=16)
    res = ens.results()
    running = res["state"] == lb.RUNNING
    assert np.all(res["steps"][running] == 20)
    ens.run(37, check_every=16)
    ens.run(50, check_every=16)
    res = ens.results()
    for k, (p, pos) in enumerate(zip(members, starts)):
        if res["state"][k] != lb.RUNNING:
            continue
        assert res["steps"][k] == 50
        sim = lb.Simulation(p, init_pos=pos)
        advance_like_member(sim, 50, lb.RUNNING)
        same_state(ens, k, sim)


def test_ensemble_autotune_leaves_the_state_unchanged():
    lb = _lb()
    members, starts = ragged_members()
    a = lb.Ensemble(members, starts)
    b = lb.Ensemble(members, starts)
    a.step(5)
    ms = a.autotune(trials=2)
    assert ms > 0
    t = a.tuning()
    assert t["rows"] in (4, 8, 16) and t["warps"] in (32, 48) and 1 <= t["claim"] <= 8
    assert t["cells_per_thread"] in (1, 2, lb.ENS_XPAIR)
    a.step(6)
    b.step(11)
    for k in range(len(members)):
        assert np.array_equal(a.populations(k), b.populations(k)), k
        assert np.array_equal(a.beads(k)[0], b.beads(k)[0]), k


@pytest.mark.parametrize("rows,warps,claim,cpt", [(4, 32, 1, 1), (16, 48, 8, 1), (8, 32, 3, 1),
                                                  (4, 32, 2, 2), (8, 32, 5, 2)])
def test_ensemble_tile_shapes_agree(rows, warps, claim, cpt):
    """Every launch shape updates every node once; two cells per thread leave a
    single-plane tile on the boxes with odd nz (13 and 17)."""
    lb = _lb()
    members, starts = ragged_members()
    a = lb.Ensemble(members, starts)
    b = lb.Ensemble(members, starts)
    a.set_tuning(rows, warps, claim, cpt)
    a.step(7)
    b.step(7)
    for k in range(len(members)):
        assert np.array_equal(a.populations(k), b.populations(k)), k


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("rows,claim", [(4, 2), (8, 5)])
def test_ensemble_xpair_tiles_agree(storage, rows, claim):
    """16-bit storage with two x-adjacent nodes per thread (tiles of 64 x rows
    nodes, pairs of one 32-bit word): the same bits as one node per thread,
    with a chain and without."""
    lb = _lb()
    members, starts = ragged_members(storage)
    a = lb.Ensemble(members, starts)
    b = lb.Ensemble(members, starts)
    a.set_tuning(rows, 32, claim, lb.ENS_XPAIR)
    assert a.tuning()["cells_per_thread"] == lb.ENS_XPAIR
    a.step(9)
    b.step(9)
    for k in range(len(members)):
        assert np.array_equal(a.populations(k), b.populations(k)), k
        assert np.array_equal(a.beads(k)[0], b.beads(k)[0]), k


def test_ensemble_xpair_needs_16_bit_storage():
    lb = _lb()
    members, starts = ragged_members("f32")
    ens = lb.Ensemble(members, starts)
    with pytest.raises(lb.LbmdError):
        ens.set_tuning(8, 32, 2, lb.ENS_XPAIR)


def test_ensemble_long_chain_matches_single_box():
    """A 600-bead chain (the 1024-thread MD block) beside a 20-bead one: the
    ensemble's spread sum kernel over both chains and the apply's conversion
    give the same bits as the single boxes."""
    lb = _lb()
    members = [si.ragged_member(600, 5, seed=61, lj_eps=PAPER_EPS),
               si.ragged_member(20, 3, seed=62, lj_eps=PAPER_EPS)]
    starts = [si.saw_chain(m, m["seed"]) for m in members]
    ens = lb.Ensemble(members, starts)
    ens.step(6)
    for k, (m, pos) in enumerate(zip(members, starts)):
        sim = lb.Simulation(m, init_pos=pos)
        advance_like_member(sim, 6, lb.RUNNING)
        same_state(ens, k, sim)


def test_ensemble_kernel_timing():
    lb = _lb()
    members, starts = ragged_members()
    ens = lb.Ensemble(members, starts)
    ens.set_kernel_timing(True)
    ens.step(3)
    kt = ens.kernel_times()
    assert kt["steps"] == 3 and 0 < kt["lb_ms"] <= kt["step_ms"]
    ens.set_kernel_timing(False)
    ens.step(2)
    assert ens.results()["steps"].min() == 5  # nobody translocates in 5 steps


def test_translocation_time_statistics_against_oracle_ensemble():
    """Bead parameters of the benchmark (eps = 1): the dynamics are chaotic, so
    single realisations of the GPU and of the oracle drift apart; the mean
    translocation time of an ensemble must still agree.  24 seeds of the
    N = 20 chain in its 32x16x16 box with a 5x5 pore: the mean t_transloc of
    the GPU ensemble with FP32, FP16 and BF16 storage lies within the 95%
    confidence interval (1.96 s / sqrt(n)) of the oracle ensemble's mean."""
    lb = _lb()
    members, starts = [], []
    for s in range(24):
        p = si.ragged_member(20, 5, seed=1000 + s)
        members.append(p)
        starts.append(si.saw_chain(p, p["seed"]))
    t_orc = []
    for p, pos in zip(members, starts):
        orc = oracle_of(p, pos)
        while orc.status()["state"] == oracle.RUNNING and orc.status()["step"] < 1500:
            orc.step(25)
        st = orc.status()
        assert st["state"] == oracle.TRANSLOCATED
        t_orc.append(st["t_transloc"])
    t_orc = np.array(t_orc, dtype=np.float64)
    half = 1.96 * t_orc.std(ddof=1) / np.sqrt(t_orc.size)
    for storage in ("f32", "f16", "bf16"):
        ens = lb.Ensemble([dict(m, storage=storage) for m in members], starts)
        ens.run(1500, check_every=128)
        r = ens.results()
        assert np.all(r["state"] == lb.TRANSLOCATED), storage
        mean = float(r["t_transloc"].mean())
        print(f"{storage}: GPU mean {mean:.1f}, oracle mean {t_orc.mean():.1f} +- {half:.1f}")
        assert abs(mean - t_orc.mean()) <= half, (storage, mean, t_orc.mean(), half)


def test_solvent_free_ensemble_matches_oracle():
    """Without a solvent the ensemble runs the MD groups and the bookkeeping
    only; each realisation translocates at the oracle's step (eps = 2e-3,
    within two steps) and stops there."""
    lb = _lb()
    members, starts = [], []
    for n, d, seed in ((20, 3, 31), (20, 5, 32), (50, 5, 33), (37, 3, 34)):
        p = si.ragged_member(n, d, seed=seed, lj_eps=PAPER_EPS, hydrodynamics=0)
        members.append(p)
        starts.append(si.saw_chain(p, p["seed"]))
    ens = lb.Ensemble(members, starts)
    assert ens.autotune(1) == 0.0
    ens.run(6000, check_every=128)
    r = ens.results()
    for k, (p, pos) in enumerate(zip(members, starts)):
        orc = oracle_of(p, pos)
        while orc.status()["state"] == oracle.RUNNING and orc.status()["step"] < 6000:
            orc.step(25)
        so = orc.status()
        assert so["state"] == oracle.TRANSLOCATED, k
        assert r["state"][k] == lb.TRANSLOCATED, k
        assert abs(int(r["t_transloc"][k]) - so["t_transloc"]) <= 2, (k, r["t_transloc"][k], so)
        assert r["steps"][k] == r["t_transloc"][k]


def test_ensemble_diagnostics_match_single_box():
    """Per-realisation diagnostic records of the ensemble equal those of the
    single-box path (same kernel body, same bits), and stop with the
    realisation."""
    lb = _lb()
    members, starts = ragged_members()
    members = [dict(m, diag_every=4, diag_capacity=50) for m in members]
    ens = lb.Ensemble(members, starts)
    ens.step(40)
    res = ens.results()
    for k, (p, pos) in enumerate(zip(members, starts)):
        d = ens.diagnostics(k)
        assert list(d["step"]) == list(range(4, res["steps"][k] + 1, 4)), k
        sim = lb.Simulation(p, init_pos=pos)
        advance_like_member(sim, 40, lb.RUNNING)
        ds = sim.diagnostics()
        assert list(ds["step"]) == list(d["step"])
        for key in ("r_u", "r_t", "r_e", "s_h", "s_e", "kinetic", "n_trans"):
            assert np.array_equal(d[key], ds[key]), (k, key)


def test_many_small_realisations():
    """1024 realisations (every MD group size from 1 to 64 beads, boxes of
    8192 nodes): sampled members equal the single-box path after 20 steps."""
    lb = _lb()
    members, starts = [], []
    for k in range(1024):
        p = dict(si.BASE)
        p.update(nx=32, ny=16, nz=16, wall_x=16, pore_d=3 if k % 2 else 5, n_beads=1 + (k * 7) % 40,
                 seed=9000 + k, lj_eps=PAPER_EPS)
        members.append(p)
        starts.append(si.saw_chain(p, p["seed"]))
    ens = lb.Ensemble(members, starts)
    ens.step(20)
    res = ens.results()
    assert np.all(res["steps"][res["state"] == lb.RUNNING] == 20)
    for k in (0, 1, 511, 777, 1023):
        sim = lb.Simulation(members[k], init_pos=starts[k])
        advance_like_member(sim, 20, lb.RUNNING)
        same_state(ens, k, sim)


def test_ensemble_forcing_and_coupling_variants():
    """Options that only the single-box tests covered, now per realisation in
    an ensemble: Guo forcing with a body force (shared), NGP coupling, bending
    stiffness and y-walls (per realisation); every member against the oracle
    after 5 steps (populations 2e-5, beads 1e-5)."""
    lb = _lb()
    specs = [
        dict(nx=32, ny=16, nz=16, wall_x=16, pore_d=3, n_beads=12, seed=51, coupling="ngp"),
        dict(nx=40, ny=18, nz=16, wall_x=20, pore_d=5, n_beads=20, seed=52, kappa_phi=0.5),
        dict(nx=36, ny=17, nz=12, wall_x=18, pore_d=3, n_beads=9, seed=53, y_walls=1),
    ]
    members, starts = [], []
    for sp in specs:
        p = dict(si.BASE)
        p.update(sp, lj_eps=PAPER_EPS, forcing="guo", body_force=(2e-5, 1e-6, 0.0))
        members.append(p)
        starts.append(si.saw_chain(p, p["seed"]))
    ens = lb.Ensemble(members, starts)
    ens.step(5)
    for k, (p, pos) in enumerate(zip(members, starts)):
        orc = oracle_of(p, pos)
        orc.step(5)
        assert rel_err(ens.populations(k), orc.populations()) < 2e-5, k
        assert np.abs(ens.beads(k)[0] - orc.beads()[0]).max() < 1e-5, k


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16", 6e-4)])
def test_bench_ensemble_full_size_sampled_against_oracle(storage, tol):
    """The benchmark's ensemble at full size and in its launch configuration
    (512 ragged realisations, 120.6 M nodes, autotuned stream-collide): after
    two steps, sampled realisations of every chain length -- the N = 400 ones
    in 144 x 80 x 80 boxes included -- against the oracle (FP32 1e-5, FP16 the
    storage bound of the single-box tests)."""
    lb = _lb()
    members, starts = si.ragged_ensemble(512, seed=0)
    ens = lb.Ensemble([dict(m, storage=storage) for m in members], starts)
    ens.autotune(2)
    ens.step(2)
    seen = set()
    for k, m in enumerate(members):
        key = (m["n_beads"], m["pore_d"])
        if key in seen or m["n_beads"] not in (20, 100, 400):
            continue
        seen.add(key)
        orc = oracle_of(m, starts[k])
        orc.step(2)
        assert rel_err(ens.populations(k), orc.populations()) < tol, (k, key)
        assert np.abs(ens.beads(k)[0] - orc.beads()[0]).max() < 1e-5, (k, key)
    assert len(seen) >= 5
