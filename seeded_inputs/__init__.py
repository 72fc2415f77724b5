"""Seeded synthetic inputs shared by the CUDA-path tests, the oracle tests and the bench.

This module holds workload descriptions (parameter dicts), initial polymer
conformations and initial flow fields.  It contains none of the method's
arithmetic (no lattice-Boltzmann update, no bead force, no coupling) and it
imports neither the oracle nor the CUDA library.

Workloads follow the paper's runs (Sec. III): a box N_x = 2 N_y = 2 N_z split
by a one-node wall at x = N_x/2 with a centred square pore, a bead-spring
polymer of bond length 1.2 with LJ sigma = 1.8, friction gamma = 0.1, a pulling
force of 0.02 inside the pore, kT = 1e-4 and M = 5 MD substeps per LB step.
"""
from __future__ import annotations

import math

import numpy as np

# LB units; Sec. III parameter list (sigma, b, gamma, beta, f_drive, M) with
# the box / tau / eps of the benchmark workloads.
BASE = dict(
    wall_thickness=1, pore_y0=-1, pore_z0=-1, y_walls=0,
    tau=1.0, rho0=1.0, body_force=(0.0, 0.0, 0.0),
    forcing="paper", coupling="trilinear",
    md_substeps=5, bead_mass=1.0, gamma=0.1, kT=1e-4, lj_sigma=1.8, lj_eps=1.0,
    kappa_phi=0.0, f_drive=0.02, bond_len=1.2,
)


def small_translocation(seed: int = 0, n_beads: int = 20) -> dict:
    """32x16x16 box, wall at x = 16, 3x3 pore, 20-bead chain, tau = 1."""
    p = dict(BASE)
    p.update(nx=32, ny=16, nz=16, wall_x=16, pore_d=3, n_beads=n_beads, seed=seed)
    return p


def paper_translocation(seed: int = 0, n_beads: int = 400) -> dict:
    """256x128x128 box, wall at x = 128, 5x5 pore, 400-bead chain, tau = 1."""
    p = dict(BASE)
    p.update(nx=256, ny=128, nz=128, wall_x=128, pore_d=5, n_beads=n_beads, seed=seed)
    return p


def periodic_solvent(n: int, tau: float = 1.0, g: float = 1e-6) -> dict:
    """Periodic n^3 box, no wall, no beads, body force g along x."""
    p = dict(BASE)
    p.update(nx=n, ny=n, nz=n, wall_x=-1, pore_d=0, n_beads=0, tau=tau,
             body_force=(g, 0.0, 0.0), seed=0)
    return p


def poiseuille_channel(nx: int = 256, ny: int = 128, nz: int = 128,
                       tau: float = 1.0, g: float = 1e-6) -> dict:
    """Channel with solid rows y = 0 and y = ny-1, body force g along x."""
    p = periodic_solvent(nx, tau, g)
    p.update(ny=ny, nz=nz, y_walls=1)
    return p


def ensemble_box(n_beads: int) -> tuple[int, int, int]:
    """Box of a ragged-ensemble realisation: (4 N^0.6, 2 N^0.6, 2 N^0.6), each
    rounded half-up to a multiple of 16, at least 32 x 16 x 16."""
    def r16(v):
        return int(math.floor(v / 16.0 + 0.5)) * 16
    a = n_beads ** 0.6
    return max(r16(4 * a), 32), max(r16(2 * a), 16), max(r16(2 * a), 16)


def ragged_member(n_beads: int, pore_d: int, seed: int, **overrides) -> dict:
    """One realisation of the ragged ensemble: box from ensemble_box(N), wall
    at x = N_x / 2 with a centred d x d pore, paper bead parameters."""
    nx, ny, nz = ensemble_box(n_beads)
    p = dict(BASE)
    p.update(nx=nx, ny=ny, nz=nz, wall_x=nx // 2, pore_d=pore_d, n_beads=n_beads, seed=seed)
    p.update(overrides)
    return p


def ragged_ensemble(count: int, seed: int = 0, lengths=(20, 50, 100, 200, 400), pores=(3, 5),
                    **overrides):
    """`count` realisations with N drawn uniformly from `lengths` and d from
    `pores` (seeded), realisation k seeded with seed * 1_000_003 + k, each with
    its own self-avoiding start.  Returns (list of params, list of (N, 3))."""
    rng = np.random.default_rng(seed)
    members, starts = [], []
    for k in range(count):
        n = int(rng.choice(lengths))
        d = int(rng.choice(pores))
        p = ragged_member(n, d, seed * 1_000_003 + k, **overrides)
        members.append(p)
        starts.append(saw_chain(p, p["seed"]))
    return members, starts


def taylor_green_field(nx: int, ny: int, nz: int, amp: float) -> np.ndarray:
    """u = A (sin kx cos ky, -cos kx sin ky, 0), k = 2 pi / L; shape (3, nz, ny, nx)."""
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    u = np.zeros((3, nz, ny, nx))
    u[0] = amp * np.sin(kx * x) * np.cos(ky * y)
    u[1] = -amp * np.cos(kx * x) * np.sin(ky * y)
    return u


def random_flow(shape, seed: int, rho_spread: float = 0.1, u_max: float = 0.05):
    """Random density in [1 - s, 1 + s] and velocity components in [-u_max, u_max]."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_spread * (2 * rng.random(shape) - 1)
    u = u_max * (2 * rng.random((3,) + tuple(shape)) - 1)
    return rho, u


def pore_geometry(p: dict):
    """(y0, z0, d) of the pore nodes: y in [y0, y0 + d), likewise z."""
    d = p["pore_d"]
    y0 = p["pore_y0"] if p.get("pore_y0", -1) >= 0 else (p["ny"] - d) // 2
    z0 = p["pore_z0"] if p.get("pore_z0", -1) >= 0 else (p["nz"] - d) // 2
    return y0, z0, d


def solid_mask(p: dict) -> np.ndarray:
    """Boolean (nz, ny, nx) of the solid nodes: the wall minus the pore, plus
    the optional rows y = 0 and y = ny - 1."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    s = np.zeros((nz, ny, nx), dtype=bool)
    if p.get("wall_x", -1) >= 0:
        y0, z0, d = pore_geometry(p)
        for t in range(p.get("wall_thickness", 1)):
            s[:, :, (p["wall_x"] + t) % nx] = True
        if d > 0:
            s[z0:z0 + d, y0:y0 + d, [(p["wall_x"] + t) % nx for t in range(p.get("wall_thickness", 1))]] = False
    if p.get("y_walls", 0):
        s[:, 0, :] = True
        s[:, ny - 1, :] = True
    return s


def saw_chain(p: dict, seed: int, max_rejects: int = 1000, max_restarts: int = 1000) -> np.ndarray:
    """Seeded off-lattice self-avoiding walk on the cis side (x > wall), bead 0
    in the pore mouth: bead 0 at (x_w + t, pore centre), bead 1 a bond further
    along +x, every later bead a random unit direction times the bond length,
    rejected if it comes within 2^(1/6) sigma of a non-neighbour bead (minimum
    image), of the wall plane, or of a solid node.  Returns (N, 3) float64."""
    rng = np.random.default_rng(seed)
    N = int(p["n_beads"])
    b = float(p["bond_len"])
    rc = 2 ** (1 / 6) * float(p["lj_sigma"])
    L = np.array([p["nx"], p["ny"], p["nz"]], dtype=np.float64)
    t = int(p.get("wall_thickness", 1))
    xw = int(p["wall_x"])
    if xw < 0:
        y0 = z0 = 0
        d = 1
        start = np.array([L[0] / 2, L[1] / 2, L[2] / 2])
    else:
        y0, z0, d = pore_geometry(p)
        start = np.array([xw + t, y0 + (d - 1) / 2, z0 + (d - 1) / 2], dtype=np.float64)
    solid = np.argwhere(solid_mask(p))[:, ::-1].astype(np.float64)  # (x, y, z)
    x_lo = (xw + t - 1 + rc) if xw >= 0 else -np.inf
    x_hi = (xw + L[0] - rc) if xw >= 0 else np.inf

    def near_solid(r):
        if solid.shape[0] == 0:
            return False
        dd = solid - np.mod(r, L)
        dd -= L * np.floor(dd / L + 0.5)
        return bool(np.any(np.einsum("ij,ij->i", dd, dd) < rc * rc))

    for _ in range(max_restarts):
        pos = np.zeros((N, 3))
        if N == 0:
            return pos
        pos[0] = start
        if N > 1:
            pos[1] = start + np.array([b, 0.0, 0.0])
        ok = True
        for i in range(2, N):
            placed = False
            for _try in range(max_rejects):
                v = rng.normal(size=3)
                v /= np.linalg.norm(v)
                cand = pos[i - 1] + b * v
                if xw >= 0 and not (x_lo <= cand[0] <= x_hi):
                    continue
                dd = pos[: i - 1] - cand
                dd -= L * np.floor(dd / L + 0.5)
                if np.any(np.einsum("ij,ij->i", dd, dd) < rc * rc):
                    continue
                if near_solid(cand):
                    continue
                pos[i] = cand
                placed = True
                break
            if not placed:
                ok = False
                break
        if ok:
            return pos
    raise RuntimeError("self-avoiding walk: too many restarts")
