"""Translocation times of the FP64 oracle over the chain lengths of the
time-versus-length exponent (Sec. III: mean t ~ N^alpha), written to
``oracle_transloc_eps2e-3.txt`` beside this script.

Workload: ragged-ensemble realisations (box (4 N^0.6, 2 N^0.6, 2 N^0.6)
rounded to 16, wall at x = N_x / 2, centred 5x5 pore, the paper's bead
parameters with eps = 2e-3), N in {50, 100, 200, 400}, realisation seeds
3000 + 1000 N + s for s = 0 .. SEEDS-1 -- the seeds the GPU ensembles of the
precision report use, so the two sides run the same starts.  Each realisation
runs until it leaves the running state or reaches CAP steps.

One realisation per worker process (one OpenMP thread each), longest chains
first unless the lengths are given (then in the order given).  Every finished realisation is appended as one line at once, so an
interrupted run keeps what it finished and a re-run skips those.  Only the
oracle and the seeded input generators are called.

  python tests/golden/make_oracle_transloc.py [workers] [N ...]   # default: all lengths
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_transloc_eps2e-3.txt")
LENGTHS = (400, 200, 100, 50)
SEEDS = 16
CAP = 150_000
EPS = 2e-3


def member(n: int, s: int):
    import seeded_inputs as si

    p = si.ragged_member(n, 5, seed=3000 + 1000 * n + s, lj_eps=EPS)
    return p, si.saw_chain(p, p["seed"])


def run_one(job):
    n, s = job
    import oracle

    oracle.set_threads(1)
    p, pos = member(n, s)
    orc = oracle.OracleSim(p, init_pos=pos)
    t0 = time.perf_counter()
    while True:
        st = orc.status()
        if st["state"] != oracle.RUNNING or st["step"] >= CAP:
            break
        orc.step(25)
    return n, s, p["seed"], int(st["state"]), int(st["t_transloc"]), int(st["step"]), time.perf_counter() - t0


def done_jobs():
    got = set()
    if os.path.exists(OUT):
        for line in open(OUT):
            if line.strip() and not line.startswith("#"):
                f = line.split()
                got.add((int(f[0]), int(f[1])))
    return got


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    lengths = tuple(int(a) for a in sys.argv[2:]) or LENGTHS
    have = done_jobs()
    jobs = [(n, s) for n in lengths for s in range(SEEDS) if (n, s) not in have]
    if not os.path.exists(OUT):
        with open(OUT, "w") as f:
            f.write("# FP64 oracle translocation runs, eps = 2e-3, 5x5 pore, ragged-ensemble boxes\n")
            f.write(f"# written by tests/golden/make_oracle_transloc.py (cap {CAP} steps)\n")
            f.write("# state: 1 translocated, 2 retracted, 3 non-finite, 4 constraint failure, 0 cap\n")
            f.write("# N s seed state t_transloc steps wall_s\n")
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=workers) as pool:
        for r in pool.imap_unordered(run_one, jobs):
            with open(OUT, "a") as f:
                f.write("%d %d %d %d %d %d %.0f\n" % r)
                f.flush()
                os.fsync(f.fileno())
            print(*r, flush=True)


if __name__ == "__main__":
    main()
