"""FP64 CPU oracle of the coupled LB / polymer-MD step (arXiv:0710.1272, Sec. II-III).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It builds and loads
``liblbmd_oracle.so`` from ``lbmd_oracle.c`` (plain C + OpenMP, double
precision) and shares no code with the CUDA library.

Parameters are plain dicts with the keys of :data:`PARAM_KEYS`; missing keys
take the values of :data:`DEFAULTS`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblbmd_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 19

DEFAULTS = dict(
    nx=32, ny=16, nz=16,
    wall_x=-1, wall_thickness=1, pore_d=3, pore_y0=-1, pore_z0=-1, y_walls=0,
    tau=1.0, rho0=1.0, body_force=(0.0, 0.0, 0.0),
    forcing="paper", coupling="trilinear",
    n_beads=0, md_substeps=5,
    bead_mass=1.0, gamma=0.1, kT=1e-4, lj_sigma=1.8, lj_eps=1.0,
    kappa_phi=0.0, f_drive=0.02, bond_len=1.2,
    shake_tol=1e-12, shake_max_iter=10000, seed=0, hydrodynamics=1, kT_fluid=0.0,
)
PARAM_KEYS = tuple(DEFAULTS)

RUNNING, TRANSLOCATED, RETRACTED, NAN, SHAKE_FAIL = range(5)


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("wall_x", C.c_int32), ("wall_thickness", C.c_int32),
        ("pore_d", C.c_int32), ("pore_y0", C.c_int32), ("pore_z0", C.c_int32),
        ("y_walls", C.c_int32), ("forcing", C.c_int32), ("coupling", C.c_int32),
        ("n_beads", C.c_int32), ("md_substeps", C.c_int32),
        ("n_bonds", C.c_int32), ("shake_max_iter", C.c_int32),
        ("hydrodynamics", C.c_int32),
        ("tau", C.c_double), ("rho0", C.c_double), ("g", C.c_double * 3),
        ("mass", C.c_double), ("gamma", C.c_double), ("kT", C.c_double),
        ("lj_sigma", C.c_double), ("lj_eps", C.c_double),
        ("kappa_phi", C.c_double), ("f_drive", C.c_double),
        ("shake_tol", C.c_double), ("kT_fluid", C.c_double), ("seed", C.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (gcc, -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.POINTER(_Params), P, P, P, P, P, P, P]
        L.orc_destroy.argtypes = [P]
        L.orc_step.argtypes = [P, C.c_int64]
        L.orc_step.restype = C.c_int
        for name in ("orc_get_populations", "orc_set_populations"):
            getattr(L, name).argtypes = [P, dp]
        L.orc_get_fields.argtypes = [P, dp, dp]
        L.orc_get_beads.argtypes = [P, dp, dp]
        L.orc_set_beads.argtypes = [P, dp, dp]
        L.orc_get_bead_aux.argtypes = [P, dp, dp]
        L.orc_get_force_field.argtypes = [P, dp]
        L.orc_get_solid.argtypes = [P, np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")]
        L.orc_get_status.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
        L.orc_get_sweeps.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.orc_forces.argtypes = [P, dp, dp]
        L.orc_forces.restype = C.c_double
        L.orc_gather.argtypes = [P, dp, dp]
        L.orc_mode_basis.argtypes = [dp, dp]
        L.orc_mode_basis.restype = None
        L.orc_fluct_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_double, C.c_double,
                                      C.c_double, dp]
        L.orc_fluct_noise.restype = None
        L.orc_diagnostics.argtypes = [P, dp, dp, dp, dp]
        L.orc_diagnostics.restype = None
        L.orc_state_diagnostics.argtypes = [P, dp]
        L.orc_state_diagnostics.restype = None
        L.orc_spread.argtypes = [P, dp, dp, dp]
        L.orc_transfer_weights.argtypes = [P, dp, np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS"), dp]
        L.orc_transfer_weights.restype = C.c_int
        L.orc_shake.argtypes = [P, dp, dp, C.POINTER(C.c_int32)]
        L.orc_shake.restype = C.c_int
        L.orc_rattle.argtypes = [P, dp, dp, C.POINTER(C.c_int32)]
        L.orc_rattle.restype = C.c_int
        L.orc_equilibrium.argtypes = [C.c_double, dp, dp]
        L.orc_moments.argtypes = [dp, dp, C.c_int, C.POINTER(C.c_double), dp]
        L.orc_collide.argtypes = [dp, C.c_double, dp, dp, C.c_int, dp]
        u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_gauss3.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_uint32, C.c_uint32, dp]
        L.orc_weights_table.argtypes = [dp, i32p]
        L.orc_weights_table.restype = C.c_int
        L.orc_max_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def full_params(p: dict | None = None) -> dict:
    out = dict(DEFAULTS)
    if p:
        unknown = set(p) - set(DEFAULTS) - {"bonds"}
        if unknown:
            raise KeyError(f"unknown parameter(s): {sorted(unknown)}")
        out.update(p)
    return out


def linear_chain_bonds(n: int, b: float):
    bi = np.arange(max(n - 1, 0), dtype=np.int32)
    return bi, bi + 1, np.full(max(n - 1, 0), float(b))


def _c_params(p: dict, n_bonds: int) -> _Params:
    cp = _Params()
    for k in ("nx", "ny", "nz", "wall_x", "wall_thickness", "pore_d", "pore_y0",
              "pore_z0", "y_walls", "n_beads", "md_substeps", "shake_max_iter",
              "hydrodynamics"):
        setattr(cp, k, int(p[k]))
    cp.forcing = {"paper": 0, "guo": 1}[p["forcing"]]
    cp.coupling = {"trilinear": 0, "ngp": 1}[p["coupling"]]
    cp.n_bonds = n_bonds
    cp.tau, cp.rho0 = float(p["tau"]), float(p["rho0"])
    for a in range(3):
        cp.g[a] = float(p["body_force"][a])
    cp.mass, cp.gamma, cp.kT = float(p["bead_mass"]), float(p["gamma"]), float(p["kT"])
    cp.lj_sigma, cp.lj_eps = float(p["lj_sigma"]), float(p["lj_eps"])
    cp.kappa_phi, cp.f_drive = float(p["kappa_phi"]), float(p["f_drive"])
    cp.shake_tol, cp.seed = float(p["shake_tol"]), int(p["seed"]) & ((1 << 64) - 1)
    cp.kT_fluid = float(p["kT_fluid"])
    return cp


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleSim:
    """One box, one chain: FP64 state stepped by the oracle library."""

    def __init__(self, params: dict | None = None, init_pos=None, init_vel=None,
                 init_rho=None, init_u=None, bonds=None):
        L = lib()
        self.p = full_params(params)
        p = self.p
        self.shape = (p["nz"], p["ny"], p["nx"])
        self.V = p["nx"] * p["ny"] * p["nz"]
        N = int(p["n_beads"])
        if bonds is None:
            bonds = self.p.get("bonds")
        if bonds is None:
            bonds = linear_chain_bonds(N, p["bond_len"])
        self.bi = np.ascontiguousarray(bonds[0], dtype=np.int32)
        self.bj = np.ascontiguousarray(bonds[1], dtype=np.int32)
        self.b0 = np.ascontiguousarray(bonds[2], dtype=np.float64)
        cp = _c_params(p, len(self.bi))
        pos = None
        if N > 0:
            if init_pos is None:
                raise ValueError("init_pos is required when n_beads > 0")
            pos = np.ascontiguousarray(init_pos, dtype=np.float64).reshape(N, 3)
        vel = None if init_vel is None else np.ascontiguousarray(init_vel, dtype=np.float64).reshape(N, 3)
        rho = None if init_rho is None else np.ascontiguousarray(init_rho, dtype=np.float64).reshape(self.shape)
        u = None if init_u is None else np.ascontiguousarray(init_u, dtype=np.float64).reshape((3,) + self.shape)
        self._keep = (pos, vel, rho, u)
        self._h = L.orc_create(C.byref(cp), _ptr(self.bi), _ptr(self.bj), _ptr(self.b0),
                               _ptr(pos), _ptr(vel), _ptr(rho), _ptr(u))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self._L = L

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    # -- stepping and read-outs -------------------------------------------
    def step(self, n: int = 1) -> int:
        return self._L.orc_step(self._h, int(n))

    def populations(self) -> np.ndarray:
        f = np.empty((Q,) + self.shape)
        self._L.orc_get_populations(self._h, f)
        return f

    def set_populations(self, f) -> None:
        self._L.orc_set_populations(self._h, np.ascontiguousarray(f, dtype=np.float64))

    def fields(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        self._L.orc_get_fields(self._h, rho, u)
        return rho, u

    def beads(self):
        N = self.p["n_beads"]
        pos, vel = np.empty((N, 3)), np.empty((N, 3))
        if N:
            self._L.orc_get_beads(self._h, pos, vel)
        return pos, vel

    def set_beads(self, pos, vel) -> None:
        self._L.orc_set_beads(self._h, np.ascontiguousarray(pos, dtype=np.float64),
                              np.ascontiguousarray(vel, dtype=np.float64))

    def bead_aux(self):
        N = self.p["n_beads"]
        ui, J = np.empty((N, 3)), np.empty((N, 3))
        if N:
            self._L.orc_get_bead_aux(self._h, ui, J)
        return ui, J

    def force_field(self) -> np.ndarray:
        F = np.empty((3,) + self.shape)
        self._L.orc_get_force_field(self._h, F)
        return F

    def solid(self) -> np.ndarray:
        s = np.empty(self.shape, dtype=np.uint8)
        self._L.orc_get_solid(self._h, s)
        return s

    def status(self):
        step, nt, st, tt = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64()
        self._L.orc_get_status(self._h, C.byref(step), C.byref(nt), C.byref(st), C.byref(tt))
        return dict(step=step.value, n_trans=nt.value, state=st.value, t_transloc=tt.value)

    def sweeps(self):
        a, b = C.c_int32(), C.c_int32()
        self._L.orc_get_sweeps(self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def diagnostics(self, pos=None, vel=None, ui=None) -> dict:
        """Sec. III chain diagnostics (R_U, R_T, R_E, S_H, S_E, K, N_T) of the
        current state, or of the given positions / velocities / u_i."""
        out = np.empty(7)
        if pos is None:
            self._L.orc_state_diagnostics(self._h, out)
        else:
            N = self.p["n_beads"]
            a = [np.ascontiguousarray(x, dtype=np.float64).reshape(N, 3) for x in (pos, vel, ui)]
            self._L.orc_diagnostics(self._h, a[0], a[1], a[2], out)
        return dict(r_u=out[0], r_t=out[1], r_e=out[2], s_h=out[3], s_e=out[4], kinetic=out[5],
                    n_trans=int(out[6]))

    # -- single stages, for the pin tests ---------------------------------
    def forces(self, pos):
        N = self.p["n_beads"]
        F = np.zeros((N, 3))
        E = self._L.orc_forces(self._h, np.ascontiguousarray(pos, dtype=np.float64), F)
        return E, F

    def gather(self, pos):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        ui = np.empty_like(pos)
        self._L.orc_gather(self._h, pos, ui)
        return ui

    def spread(self, pos, J):
        F = np.empty((3,) + self.shape)
        self._L.orc_spread(self._h, np.ascontiguousarray(pos, dtype=np.float64),
                           np.ascontiguousarray(J, dtype=np.float64), F)
        return F

    def transfer_weights(self, r):
        node = np.zeros(8, dtype=np.int64)
        w = np.zeros(8)
        n = self._L.orc_transfer_weights(self._h, np.ascontiguousarray(r, dtype=np.float64), node, w)
        return node[:n], w[:n]

    def shake(self, r_old, r_new):
        r_new = np.array(r_new, dtype=np.float64, order="C")
        sw = C.c_int32()
        rc = self._L.orc_shake(self._h, np.ascontiguousarray(r_old, dtype=np.float64), r_new, C.byref(sw))
        return rc, r_new, sw.value

    def rattle(self, r, v):
        v = np.array(v, dtype=np.float64, order="C")
        sw = C.c_int32()
        rc = self._L.orc_rattle(self._h, np.ascontiguousarray(r, dtype=np.float64), v, C.byref(sw))
        return rc, v, sw.value


# -- stateless helpers ------------------------------------------------------
def lattice():
    w = np.empty(Q)
    c = np.empty(3 * Q, dtype=np.int32)
    lib().orc_weights_table(w, c)
    return w, c.reshape(Q, 3)


def equilibrium(rho: float, u) -> np.ndarray:
    out = np.empty(Q)
    lib().orc_equilibrium(float(rho), np.ascontiguousarray(u, dtype=np.float64), out)
    return out


def moments(f, g=(0.0, 0.0, 0.0), forcing="paper"):
    rho = C.c_double()
    u = np.empty(3)
    lib().orc_moments(np.ascontiguousarray(f, dtype=np.float64), np.asarray(g, dtype=np.float64),
                      {"paper": 0, "guo": 1}[forcing], C.byref(rho), u)
    return rho.value, u


def collide(f, tau, Fb=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0), forcing="paper") -> np.ndarray:
    out = np.empty(Q)
    lib().orc_collide(np.ascontiguousarray(f, dtype=np.float64), float(tau),
                      np.asarray(Fb, dtype=np.float64), np.asarray(g, dtype=np.float64),
                      {"paper": 0, "guo": 1}[forcing], out)
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


def gauss3(seed: int, bead: int, step: int, substep: int, stream: int = 0) -> np.ndarray:
    xi = np.empty(3)
    lib().orc_gauss3(int(seed) & ((1 << 64) - 1), int(bead), int(step), int(substep), int(stream), xi)
    return xi


def mode_basis():
    """Weight-orthogonal D3Q19 mode basis e[k][p] and norms b_k."""
    e, b = np.empty((Q, Q)), np.empty(Q)
    lib().orc_mode_basis(e, b)
    return e, b


def fluct_noise(seed: int, node: int, step: int, rho: float, tau: float, kT: float) -> np.ndarray:
    """Thermal source F_p of one node at one LB step."""
    xi = np.empty(Q)
    lib().orc_fluct_noise(int(seed) & ((1 << 64) - 1), int(node), int(step), float(rho), float(tau),
                          float(kT), xi)
    return xi


def max_threads() -> int:
    return lib().orc_max_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))
