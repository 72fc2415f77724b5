"""Precision report of the 16-bit population storage against the FP64 oracle,
and the with/without-solvent comparison of Sec. III.

FP16 and BF16 storage keep the deviations h = f - w_p rho0 in 16 bits; the
collision and the bead dynamics stay in FP32.  This script measures what that
costs, next to the FP32 path, and prints a markdown report:

 1. Density, velocity and bead positions after 100 LB steps on the
    256x128x128 translocation box with a 400-bead chain, against the oracle
    (same seed, same initial state), for eps = 1 and eps = 2e-3.
 2. Mean translocation time over 32 seeds (ragged-ensemble realisations with
    N = 20 and N = 50 and a 5x5 pore, eps = 1): GPU ensembles per storage
    against the oracle ensemble's mean and 95% confidence interval.  The
    oracle cannot afford the 256x128x128 box over ~10^4 steps and 32 seeds,
    so this uses the small boxes of the ragged ensemble.
 3. The time-versus-length exponent alpha (mean t ~ N^alpha) at eps = 2e-3
    over N in {50, 100, 200, 400}, 32 seeds per N, from GPU ensembles per
    storage, and against the FP64 oracle's runs of the same seeds
    (tests/golden/oracle_transloc_eps2e-3.txt): per-N means within the
    oracle's 95 % interval, per-seed differences and the exponents.
 4. The same exponent with and without the solvent (Sec. III compares the
    two), and the cost of a step with and without it at constant volume.
 5. The chain diagnostics of Sec. III over ensembles at two friction values:
    R_T(t=1) / R_U(t=0), the effective radius over the event, the sign of
    the fluid's work rate, the mean work rates and the kinetic energy.

  python tests/precision_report.py [section ...]   # needs a CUDA device; default: all
  ALPHA_DUMP=runs.json python tests/precision_report.py 3   # also saves the GPU runs
  python tests/precision_report.py alpha-from runs.json      # section 3 again, no GPU

The oracle ensembles run in a spawn-started process pool (one realisation
per worker, one thread each) created before the first GPU call.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402

STORAGES = ("f32", "f16", "bf16")
GPU_ONLY = ("storage", "init_tg_amp")


def _oracle_run(args):
    """One oracle realisation run to translocation (or the cap): t_transloc."""
    p, pos, cap = args
    import oracle

    oracle.set_threads(1)
    orc = oracle.OracleSim({k: v for k, v in p.items() if k not in GPU_ONLY}, init_pos=pos)
    while True:
        st = orc.status()
        if st["state"] != oracle.RUNNING or st["step"] >= cap:
            return st["t_transloc"] if st["state"] == oracle.TRANSLOCATED else -1
        orc.step(25)


def ci95(t):
    t = np.asarray(t, dtype=np.float64)
    return t.mean(), 1.96 * t.std(ddof=1) / np.sqrt(t.size)


def alpha_fit(ns, means):
    x, y = np.log(np.asarray(ns, float)), np.log(np.asarray(means, float))
    return float(np.polyfit(x, y, 1)[0])


def section_fields(lb, oracle):
    print("## 1. Fields and beads after 100 steps, 256x128x128, N = 400\n")
    print("| eps | storage | max abs err rho | rms err rho | max abs err u | rms err u "
          "| max abs err bead r | max |u| |")
    print("|---|---|---|---|---|---|---|---|")
    for eps in (1.0, 2e-3):
        p = si.paper_translocation(0)
        p["lj_eps"] = eps
        pos = si.saw_chain(p, 0)
        orc = oracle.OracleSim({k: v for k, v in p.items() if k not in GPU_ONLY}, init_pos=pos)
        orc.step(100)
        rho_o, u_o = orc.fields()
        r_o = orc.beads()[0]
        del orc
        for st in STORAGES:
            sim = lb.Simulation(dict(p, storage=st), init_pos=pos)
            sim.step(100)
            rho, u = sim.fields()
            r = sim.beads()[0]
            del sim
            dr = np.abs(rho - rho_o)
            du = np.abs(u - u_o)
            print(f"| {eps:g} | {st} | {dr.max():.2e} | {np.sqrt((dr ** 2).mean()):.2e} | "
                  f"{du.max():.2e} | {np.sqrt((du ** 2).mean()):.2e} | "
                  f"{np.abs(r - r_o).max():.2e} | {np.abs(u_o).max():.2e} |")
    print()


def section_transloc(lb, pool):
    print("## 2. Mean translocation time, 32 seeds, eps = 1, 5x5 pore\n")
    print("| N | box | oracle mean +- 95% | storage | GPU mean | |GPU - oracle| / half-width "
          "| translocated |")
    print("|---|---|---|---|---|---|---|")
    for n in (20, 50):
        members, starts = [], []
        for s in range(32):
            p = si.ragged_member(n, 5, seed=2000 + 100 * n + s)
            members.append(p)
            starts.append(si.saw_chain(p, p["seed"]))
        t_o = pool.map(_oracle_run, [(p, pos, 8000) for p, pos in zip(members, starts)])
        t_o = np.array(t_o)
        assert np.all(t_o > 0), "an oracle realisation did not translocate"
        mo, ho = ci95(t_o)
        box = f"{members[0]['nx']}x{members[0]['ny']}x{members[0]['nz']}"
        for st in STORAGES:
            ens = lb.Ensemble([dict(m, storage=st) for m in members], starts)
            ens.run(8000, check_every=256)
            r = ens.results()
            del ens
            ok = r["state"] == lb.TRANSLOCATED
            mg = r["t_transloc"][ok].mean()
            print(f"| {n} | {box} | {mo:.1f} +- {ho:.1f} | {st} | {mg:.1f} | "
                  f"{abs(mg - mo) / ho:.2f} | {ok.sum()}/32 |")
    print()


ALPHA_NS = (50, 100, 200, 400)
ALPHA_SEEDS = 32
ORACLE_FILE = os.path.join(ROOT, "tests", "golden", "oracle_transloc_eps2e-3.txt")


def alpha_members():
    """The realisations of the exponent runs: ragged-ensemble boxes, 5x5 pore,
    eps = 2e-3, seeds 3000 + 1000 N + s (the seeds of the oracle runs in
    tests/golden/oracle_transloc_eps2e-3.txt)."""
    members, starts, which, seeds = [], [], [], []
    for n in ALPHA_NS:
        for s in range(ALPHA_SEEDS):
            p = si.ragged_member(n, 5, seed=3000 + 1000 * n + s, lj_eps=2e-3)
            members.append(p)
            starts.append(si.saw_chain(p, p["seed"]))
            which.append(n)
            seeds.append(s)
    return members, starts, np.array(which), np.array(seeds)


def alpha_gpu_runs(lb):
    """GPU ensembles of the exponent runs per storage: {storage: [(N, s, state,
    t_transloc), ...], "wall_s": {...}}."""
    members, starts, which, seeds = alpha_members()
    out = {"wall_s": {}}
    for st in STORAGES:
        ens = lb.Ensemble([dict(m, storage=st) for m in members], starts)
        ens.autotune(2)
        t0 = time.perf_counter()
        ens.run(150000, check_every=2048)
        out["wall_s"][st] = time.perf_counter() - t0
        r = ens.results()
        del ens
        out[st] = [(int(n), int(k), int(a), int(b)) for n, k, a, b in
                   zip(which, seeds, r["state"], r["t_transloc"])]
    return out


def oracle_runs():
    """{(N, s): (state, t_transloc)} from the committed oracle file."""
    got = {}
    if os.path.exists(ORACLE_FILE):
        for line in open(ORACLE_FILE):
            if line.strip() and not line.startswith("#"):
                f = line.split()
                got[(int(f[0]), int(f[1]))] = (int(f[3]), int(f[4]))
    return got


def print_alpha(gpu):
    print("## 3. Exponent alpha of mean t ~ N^alpha, eps = 2e-3, 5x5 pore\n")
    print(f"GPU: {ALPHA_SEEDS} seeds per N (s = 0 .. {ALPHA_SEEDS - 1}), one ragged ensemble per storage. "
          "Oracle: the FP64 runs of `tests/golden/oracle_transloc_eps2e-3.txt` (written by "
          "`tests/golden/make_oracle_transloc.py`, one realisation per host core), same seeds and starts.\n")
    print("| storage | " + " | ".join(f"mean t (N={n})" for n in ALPHA_NS) + " | alpha | translocated | wall s |")
    print("|---|" + "---|" * len(ALPHA_NS) + "---|---|---|")
    for st in STORAGES:
        rows = gpu[st]
        means = [np.mean([t for n2, _, a, t in rows if n2 == n and a == 1]) for n in ALPHA_NS]
        ok = sum(1 for r in rows if r[2] == 1)
        print(f"| {st} | " + " | ".join(f"{m:.0f}" for m in means) +
              f" | {alpha_fit(ALPHA_NS, means):.3f} | {ok}/{len(rows)} | {gpu['wall_s'][st]:.0f} |")
    print()
    orc = oracle_runs()
    ns = [n for n in ALPHA_NS if any(k[0] == n for k in orc)]
    if not ns:
        print("(no oracle runs yet)\n")
        return
    print("Against the oracle on the seeds it has run (t of translocated realisations; "
          "95 % interval of the oracle mean; per-seed difference |t_GPU - t_oracle|):\n")
    print("| N | oracle seeds | oracle mean +- 95% | storage | GPU mean, same seeds | |GPU - oracle| / half-width | max per-seed diff | median per-seed diff |")
    print("|---|---|---|---|---|---|---|---|")
    alpha_rows = {}
    for n in ns:
        sd = sorted(k[1] for k in orc if k[0] == n and orc[k][0] == 1)
        to = np.array([orc[(n, k)][1] for k in sd], dtype=float)
        if to.size < 2:
            continue
        mo, ho = ci95(to)
        alpha_rows.setdefault("oracle", []).append((n, mo))
        for st in STORAGES:
            gmap = {k: (a, t) for n2, k, a, t in gpu[st] if n2 == n}
            tg = np.array([gmap[k][1] if gmap[k][0] == 1 else np.nan for k in sd], dtype=float)
            mg = np.nanmean(tg)
            alpha_rows.setdefault(st, []).append((n, mg))
            d = np.abs(tg - to)
            print(f"| {n} | {to.size} | {mo:.1f} +- {ho:.1f} | {st} | {mg:.1f} | {abs(mg - mo) / ho:.2f} | "
                  f"{np.nanmax(d):.0f} | {np.nanmedian(d):.0f} |")
    print()
    if len(alpha_rows.get("oracle", [])) >= 2:
        ao = alpha_fit([n for n, _ in alpha_rows["oracle"]], [m for _, m in alpha_rows["oracle"]])
        print(f"Exponent over N in {{{', '.join(str(n) for n, _ in alpha_rows['oracle'])}}} on the oracle's seeds: "
              f"oracle {ao:.4f}; " + "; ".join(
                  f"{st} {alpha_fit([n for n, _ in alpha_rows[st]], [m for _, m in alpha_rows[st]]):.4f} "
                  f"(|diff| {abs(alpha_fit([n for n, _ in alpha_rows[st]], [m for _, m in alpha_rows[st]]) - ao):.4f})"
                  for st in STORAGES) + ".\n")


def section_alpha(lb, pool, dump=None):
    gpu = alpha_gpu_runs(lb)
    if dump:
        with open(dump, "w") as f:
            json.dump({k: v for k, v in gpu.items()}, f)
    print_alpha(gpu)


def section_solvent(lb):
    print("## 4. With and without the solvent (Sec. III comparison), FP32, eps = 2e-3, 5x5 pore\n")
    ns = (50, 100, 200, 400)
    members, starts, which = [], [], []
    for n in ns:
        for s in range(32):
            p = si.ragged_member(n, 5, seed=3000 + 1000 * n + s, lj_eps=2e-3)
            members.append(p)
            starts.append(si.saw_chain(p, p["seed"]))
            which.append(n)
    which = np.array(which)
    print("| solvent | " + " | ".join(f"mean t (N={n})" for n in ns) + " | alpha | translocated |")
    print("|---|" + "---|" * len(ns) + "---|---|")
    for hydro in (1, 0):
        ens = lb.Ensemble([dict(m, hydrodynamics=hydro) for m in members], starts)
        ens.run(400000, check_every=4096)
        r = ens.results()
        del ens
        ok = r["state"] == lb.TRANSLOCATED
        means = [r["t_transloc"][(which == n) & ok].mean() for n in ns]
        print(f"| {'LB' if hydro else 'none'} | " + " | ".join(f"{m:.0f}" for m in means) +
              f" | {alpha_fit(ns, means):.3f} | {ok.sum()}/{len(members)} |")
    print()
    import torch

    print("Cost per coupled step at constant volume (256x128x128, one chain), CUDA events:\n")
    print("| N | with solvent (ms) | without (ms) |")
    print("|---|---|---|")
    for n in (50, 100, 400):
        row = []
        for hydro in (1, 0):
            p = si.paper_translocation(0, n_beads=n)
            p["hydrodynamics"] = hydro
            sim = lb.Simulation(p, init_pos=si.saw_chain(p, 0))
            sim.step(50)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(sim.stream)
            sim.step(500)
            e1.record(sim.stream)
            torch.cuda.synchronize()
            row.append(e0.elapsed_time(e1) / 500)
            del sim
        print(f"| {n} | {row[0]:.4f} | {row[1]:.4f} |")
    print()


def section_diagnostics(lb):
    print("## 5. Chain diagnostics over ensembles (Sec. III), N = 200, eps = 2e-3, FP32\n")
    print("64 realisations per gamma (96x48x48 box, 5x5 pore), diagnostics every 20 steps; t is "
          "scaled by each realisation's translocation time.\n")
    print("| gamma | translocated | mean t | R_T(t=1) / R_U(t=0) | R_E / R_U(0) in t-bins 0.1..0.9 "
          "| records with S_H > 0 | mean S_H | mean S_E | mean gamma K |")
    print("|---|---|---|---|---|---|---|---|---|")
    for gamma in (0.1, 0.5):
        members, starts = [], []
        for s in range(64):
            p = si.ragged_member(200, 5, seed=7000 + s, lj_eps=2e-3, gamma=gamma,
                                 diag_every=20, diag_capacity=4000)
            members.append(p)
            starts.append(si.saw_chain(p, p["seed"]))
        ens = lb.Ensemble(members, starts)
        ens.run(80000, check_every=4096)
        r = ens.results()
        ratios, bins, sh, se, kin = [], [[] for _ in range(9)], [], [], []
        for k in range(len(members)):
            if r["state"][k] != lb.TRANSLOCATED:
                continue
            d = ens.diagnostics(k)
            T = float(r["t_transloc"][k])
            ru0 = d["r_u"][0]
            ratios.append(d["r_t"][-1] / ru0)
            frac = d["step"] / T
            for b in range(9):
                sel = np.abs(frac - 0.1 * (b + 1)) < 0.05
                if sel.any():
                    bins[b].append(d["r_e"][sel].mean() / ru0)
            sh.append(d["s_h"])
            se.append(d["s_e"])
            kin.append(d["kinetic"])
        del ens
        sh, se, kin = np.concatenate(sh), np.concatenate(se), np.concatenate(kin)
        prof = " ".join(f"{np.mean(b):.2f}" for b in bins)
        print(f"| {gamma} | {len(ratios)}/64 | {r['t_transloc'][r['state'] == 1].mean():.0f} | "
              f"{np.mean(ratios):.3f} | {prof} | {100 * (sh > 0).mean():.1f} % | {sh.mean():.2e} | "
              f"{se.mean():.2e} | {gamma * kin.mean():.2e} |")
    print()


def main():
    if len(sys.argv) > 2 and sys.argv[1] == "alpha-from":
        # section 3 from saved GPU runs and the oracle file (no GPU needed)
        with open(sys.argv[2]) as f:
            print_alpha(json.load(f))
        return 0
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=max(1, os.cpu_count() or 1)) as pool:
        import oracle

        oracle.lib()  # built here, before the pool's first task
        import torch

        if not torch.cuda.is_available():
            print("no CUDA device", file=sys.stderr)
            return 1
        import paper_0710_1272_gb300 as lb

        want = set(sys.argv[1:]) or {"1", "2", "3", "4", "5"}
        print("# Precision of 16-bit population storage against the FP64 oracle\n")
        print(f"Device: {torch.cuda.get_device_name(0)}; host cores: {os.cpu_count()}.\n")
        if "1" in want:
            section_fields(lb, oracle)
        if "2" in want:
            section_transloc(lb, pool)
        if "3" in want:
            section_alpha(lb, pool, os.environ.get("ALPHA_DUMP"))
        if "4" in want:
            section_solvent(lb)
        if "5" in want:
            section_diagnostics(lb)
    return 0


if __name__ == "__main__":
    sys.exit(main())
