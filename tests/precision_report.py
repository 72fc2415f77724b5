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
    storage; and over N in {20, 50, 100} on 4 seeds shared with the oracle.
 4. The same exponent with and without the solvent (Sec. III compares the
    two), and the cost of a step with and without it at constant volume.
 5. The chain diagnostics of Sec. III over ensembles at two friction values:
    R_T(t=1) / R_U(t=0), the effective radius over the event, the sign of
    the fluid's work rate, the mean work rates and the kinetic energy.

  python tests/precision_report.py [section ...]   # needs a CUDA device; default: all

The oracle ensembles run in a spawn-started process pool (one realisation
per worker, one thread each) created before the first GPU call.
"""
from __future__ import annotations

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


def section_alpha(lb, pool):
    print("## 3. Exponent alpha of mean t ~ N^alpha, eps = 2e-3, 5x5 pore\n")
    ns = (50, 100, 200, 400)
    members, starts, which = [], [], []
    for n in ns:
        for s in range(32):
            p = si.ragged_member(n, 5, seed=3000 + 1000 * n + s, lj_eps=2e-3)
            members.append(p)
            starts.append(si.saw_chain(p, p["seed"]))
            which.append(n)
    which = np.array(which)
    print("| storage | " + " | ".join(f"mean t (N={n})" for n in ns) + " | alpha | translocated | wall s |")
    print("|---|" + "---|" * len(ns) + "---|---|---|")
    for st in STORAGES:
        ens = lb.Ensemble([dict(m, storage=st) for m in members], starts)
        ens.autotune(2)
        t0 = time.perf_counter()
        ens.run(150000, check_every=2048)
        wall = time.perf_counter() - t0
        r = ens.results()
        del ens
        ok = r["state"] == lb.TRANSLOCATED
        means = [r["t_transloc"][(which == n) & ok].mean() for n in ns]
        print(f"| {st} | " + " | ".join(f"{m:.0f}" for m in means) +
              f" | {alpha_fit(ns, means):.3f} | {ok.sum()}/{len(members)} | {wall:.0f} |")
    print()
    # shared seeds with the oracle on the small boxes
    ns2 = (20, 50, 100)
    members, starts, which = [], [], []
    for n in ns2:
        for s in range(4):
            p = si.ragged_member(n, 5, seed=4000 + 1000 * n + s, lj_eps=2e-3)
            members.append(p)
            starts.append(si.saw_chain(p, p["seed"]))
            which.append(n)
    which = np.array(which)
    t_o = np.array(pool.map(_oracle_run, [(p, pos, 20000) for p, pos in zip(members, starts)]))
    mo = [t_o[which == n].mean() for n in ns2]
    print("| N in {20, 50, 100}, 4 shared seeds | " + " | ".join(f"mean t (N={n})" for n in ns2)
          + " | alpha | max per-seed |t_GPU - t_oracle| |")
    print("|---|" + "---|" * len(ns2) + "---|---|")
    print("| oracle | " + " | ".join(f"{m:.1f}" for m in mo) + f" | {alpha_fit(ns2, mo):.4f} | - |")
    for st in STORAGES:
        ens = lb.Ensemble([dict(m, storage=st) for m in members], starts)
        ens.run(20000, check_every=512)
        r = ens.results()
        del ens
        mg = [r["t_transloc"][which == n].mean() for n in ns2]
        print(f"| {st} | " + " | ".join(f"{m:.1f}" for m in mg) + f" | {alpha_fit(ns2, mg):.4f} | "
              f"{np.abs(r['t_transloc'] - t_o).max()} |")
    print()


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
            section_alpha(lb, pool)
        if "4" in want:
            section_solvent(lb)
        if "5" in want:
            section_diagnostics(lb)
    return 0


if __name__ == "__main__":
    sys.exit(main())
