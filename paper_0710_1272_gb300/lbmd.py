"""Thin ctypes binding of ``include/lbmd.h`` (argument marshalling only).

Every step of the coupled LB / polymer-MD path runs in the CUDA kernels of
``liblbmd.so``; this module only converts Python values to the C structs and
pointers, and uses PyTorch for the device workspace and the stream.  There is
no CPU fallback: if the library is missing or no CUDA device is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LBMD_OK, LBMD_EINVAL, LBMD_ESIZE, LBMD_ECUDA, LBMD_EUNSUPPORTED = 0, -1, -2, -3, -4
RUNNING, TRANSLOCATED, RETRACTED, NAN, SHAKE_FAIL = range(5)
ENS_XPAIR = 3  # ensemble tuning: two x-adjacent nodes per thread (16-bit storage)
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
FORCING = {"paper": 0, "guo": 1}
COUPLING = {"trilinear": 0, "ngp": 1}
STREAMING = {"pull": 0, "aa": 1}
MAX_BEADS = 1024

# names of the parameter dict (shared with the oracle's wrapper and the
# seeded input module) and their defaults
DEFAULTS = dict(
    nx=32, ny=16, nz=16,
    wall_x=-1, wall_thickness=1, pore_d=3, pore_y0=-1, pore_z0=-1, y_walls=0,
    storage="f32", forcing="paper", coupling="trilinear",
    n_beads=0, md_substeps=5,
    tau=1.0, rho0=1.0, body_force=(0.0, 0.0, 0.0),
    bead_mass=1.0, gamma=0.1, kT=1e-4, lj_sigma=1.8, lj_eps=1.0,
    kappa_phi=0.0, f_drive=0.02, bond_len=1.2,
    shake_tol=1e-6, shake_max_iter=12, init_tg_amp=0.0, seed=0, hydrodynamics=1,
    diag_every=0, diag_capacity=0, kT_fluid=0.0, streaming="pull",
)
IGNORED_KEYS = {"bonds"}  # oracle-only keys


class lbmd_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("wall_x", C.c_int32), ("wall_thickness", C.c_int32),
        ("pore_d", C.c_int32), ("pore_y0", C.c_int32), ("pore_z0", C.c_int32),
        ("y_walls", C.c_int32), ("storage", C.c_int32), ("forcing", C.c_int32),
        ("coupling", C.c_int32), ("n_beads", C.c_int32), ("md_substeps", C.c_int32),
        ("n_constraints", C.c_int32), ("shake_max_iter", C.c_int32),
        ("solvent_free", C.c_int32), ("diag_every", C.c_int32), ("diag_capacity", C.c_int32),
        ("streaming", C.c_int32),
        ("tau", C.c_double), ("rho0", C.c_double), ("body_force", C.c_double * 3),
        ("bead_mass", C.c_double), ("gamma", C.c_double), ("kT", C.c_double),
        ("lj_sigma", C.c_double), ("lj_eps", C.c_double), ("kappa_phi", C.c_double),
        ("f_drive", C.c_double), ("bond_length", C.c_double), ("shake_tol", C.c_double),
        ("init_tg_amp", C.c_double), ("kT_fluid", C.c_double), ("seed", C.c_uint64),
        ("bond_i", C.c_void_p), ("bond_j", C.c_void_p), ("bond_len", C.c_void_p),
        ("init_pos", C.c_void_p), ("init_vel", C.c_void_p),
        ("init_rho", C.c_void_p), ("init_u", C.c_void_p),
    ]


class lbmd_status_word(C.Structure):
    _fields_ = [("step", C.c_int64), ("t_transloc", C.c_int64), ("n_trans", C.c_int32),
                ("state", C.c_int32)]


class lbmd_diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_trans", C.c_int32), ("reserved", C.c_int32),
                ("r_u", C.c_double), ("r_t", C.c_double), ("r_e", C.c_double),
                ("s_h", C.c_double), ("s_e", C.c_double), ("kinetic", C.c_double)]


DIAG_FIELDS = ("step", "n_trans", "r_u", "r_t", "r_e", "s_h", "s_e", "kinetic")

_lib = None

ENSEMBLE_FUNCTIONS = (
    "lbmd_ensemble_workspace_size", "lbmd_ensemble_create", "lbmd_ensemble_step", "lbmd_ensemble_run",
    "lbmd_ensemble_results", "lbmd_ensemble_live", "lbmd_ensemble_read_beads",
    "lbmd_ensemble_read_populations", "lbmd_ensemble_set_tuning", "lbmd_ensemble_get_tuning",
    "lbmd_ensemble_autotune", "lbmd_ensemble_set_kernel_timing", "lbmd_ensemble_kernel_times",
    "lbmd_ensemble_destroy",
)


class LbmdError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = load()
        msg = L.lbmd_last_message().decode(errors="replace")
        super().__init__(f"{where}: {L.lbmd_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def load(build_if_missing: bool = True):
    """Load liblbmd.so (building it in-tree first if needed); raises if it
    cannot be built or loaded -- there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; run paper_0710_1272_gb300.build.build()")
    L = C.CDLL(path)
    P = C.c_void_p
    L.lbmd_workspace_size.argtypes = [C.POINTER(lbmd_params), C.POINTER(C.c_size_t)]
    L.lbmd_create.argtypes = [C.POINTER(lbmd_params), P, C.c_size_t, P, C.POINTER(P)]
    L.lbmd_step.argtypes = [P, C.c_int64]
    L.lbmd_read_fields.argtypes = [P, P, P, C.c_int]
    L.lbmd_read_populations.argtypes = [P, P, C.c_int]
    L.lbmd_read_beads.argtypes = [P, P, P, C.c_int]
    L.lbmd_read_bead_aux.argtypes = [P, P, P, C.c_int]
    L.lbmd_read_beads_async.argtypes = [P, P, C.c_size_t]
    L.lbmd_step_read_async.argtypes = [P, P, C.c_size_t]
    L.lbmd_status.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                              C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    L.lbmd_solver_stats.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.lbmd_set_kernel_timing.argtypes = [P, C.c_int]
    L.lbmd_lb_kernel_time.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.lbmd_kernel_times.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.lbmd_lb_step_noalloc.argtypes = [C.POINTER(lbmd_params), P, P, P]
    L.lbmd_destroy.argtypes = [P]
    L.lbmd_read_diagnostics.argtypes = [P, P, C.c_int32, C.POINTER(C.c_int32)]
    L.lbmd_ensemble_read_diagnostics.argtypes = [P, C.c_int32, P, C.c_int32, C.POINTER(C.c_int32)]
    PI32, PI64, PD = C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double)
    L.lbmd_ensemble_workspace_size.argtypes = [C.POINTER(lbmd_params), C.c_int32, C.POINTER(C.c_size_t)]
    L.lbmd_ensemble_create.argtypes = [C.POINTER(lbmd_params), C.c_int32, P, C.c_size_t, P, C.POINTER(P)]
    L.lbmd_ensemble_step.argtypes = [P, C.c_int64]
    L.lbmd_ensemble_run.argtypes = [P, C.c_int64, C.c_int64, PI64]
    L.lbmd_ensemble_results.argtypes = [P, P, P, P, P]
    L.lbmd_ensemble_live.argtypes = [P, PI32]
    L.lbmd_ensemble_read_beads.argtypes = [P, C.c_int32, P, P, C.c_int]
    L.lbmd_ensemble_read_populations.argtypes = [P, C.c_int32, P, C.c_int]
    L.lbmd_ensemble_set_tuning.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    L.lbmd_ensemble_get_tuning.argtypes = [P, PI32, PI32, PI32, PI32]
    L.lbmd_ensemble_autotune.argtypes = [P, C.c_int32, PD]
    L.lbmd_ensemble_set_kernel_timing.argtypes = [P, C.c_int]
    L.lbmd_ensemble_kernel_times.argtypes = [P, PD, PD, PI64]
    L.lbmd_ensemble_destroy.argtypes = [P]
    L.lbmd_strerror.argtypes = [C.c_int]
    L.lbmd_strerror.restype = C.c_char_p
    L.lbmd_last_message.restype = C.c_char_p
    for name in ("lbmd_workspace_size", "lbmd_create", "lbmd_step", "lbmd_read_fields",
                 "lbmd_read_populations", "lbmd_read_beads", "lbmd_read_bead_aux", "lbmd_status",
                 "lbmd_read_beads_async", "lbmd_step_read_async",
                 "lbmd_set_kernel_timing", "lbmd_lb_kernel_time", "lbmd_destroy", "lbmd_version",
                 "lbmd_solver_stats", "lbmd_kernel_times", "lbmd_lb_step_noalloc",
                 "lbmd_read_diagnostics", "lbmd_ensemble_read_diagnostics", *ENSEMBLE_FUNCTIONS):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int, where: str) -> None:
    if rc != LBMD_OK:
        raise LbmdError(rc, where)


def full_params(p: dict | None) -> dict:
    out = dict(DEFAULTS)
    if p:
        unknown = set(p) - set(DEFAULTS) - IGNORED_KEYS
        if unknown:
            raise KeyError(f"unknown parameter(s): {sorted(unknown)}")
        out.update({k: v for k, v in p.items() if k not in IGNORED_KEYS})
    return out


def make_params(p: dict, init_pos=None, init_vel=None, init_rho=None, init_u=None, bonds=None):
    """Fill an lbmd_params struct; returns (struct, keep-alive list)."""
    p = full_params(p)
    cp = lbmd_params()
    for k in ("nx", "ny", "nz", "wall_x", "wall_thickness", "pore_d", "pore_y0", "pore_z0",
              "y_walls", "n_beads", "md_substeps", "shake_max_iter", "diag_every", "diag_capacity"):
        setattr(cp, k, int(p[k]))
    cp.solvent_free = 0 if int(p["hydrodynamics"]) else 1  # the oracle's key, inverted
    cp.storage = STORAGE[p["storage"]]
    cp.forcing = FORCING[p["forcing"]]
    cp.coupling = COUPLING[p["coupling"]]
    cp.streaming = STREAMING[p["streaming"]]
    for k in ("tau", "rho0", "bead_mass", "gamma", "kT", "lj_sigma", "lj_eps", "kappa_phi",
              "f_drive", "shake_tol", "init_tg_amp", "kT_fluid"):
        setattr(cp, k, float(p[k]))
    cp.bond_length = float(p["bond_len"])
    for a in range(3):
        cp.body_force[a] = float(p["body_force"][a])
    cp.seed = int(p["seed"]) & ((1 << 64) - 1)
    keep = []

    def arr(x, dtype, shape=None):
        if x is None:
            return None
        a = np.ascontiguousarray(x, dtype=dtype)
        if shape is not None:
            a = a.reshape(shape)
        keep.append(a)
        return a.ctypes.data

    N = int(p["n_beads"])
    V = int(p["nx"]) * int(p["ny"]) * int(p["nz"])
    if bonds is None:
        cp.n_constraints = -1
    else:
        bi, bj, bl = bonds
        cp.n_constraints = len(bi)
        cp.bond_i = arr(bi, np.int32)
        cp.bond_j = arr(bj, np.int32)
        cp.bond_len = arr(bl, np.float64)
    cp.init_pos = arr(init_pos, np.float64, (N * 3,))
    cp.init_vel = arr(init_vel, np.float64, (N * 3,))
    cp.init_rho = arr(init_rho, np.float64, (V,))
    cp.init_u = arr(init_u, np.float64, (3 * V,))
    return cp, keep


# -- the C-ABI entry points under their own names --------------------------
def lbmd_workspace_size(params: lbmd_params) -> int:
    n = C.c_size_t()
    _check(load().lbmd_workspace_size(C.byref(params), C.byref(n)), "lbmd_workspace_size")
    return n.value


def lbmd_create(params: lbmd_params, workspace_ptr: int, nbytes: int, stream_ptr: int):
    h = C.c_void_p()
    _check(load().lbmd_create(C.byref(params), C.c_void_p(workspace_ptr), nbytes,
                              C.c_void_p(stream_ptr), C.byref(h)), "lbmd_create")
    return h


def lbmd_step(ctx, n: int) -> None:
    _check(load().lbmd_step(ctx, int(n)), "lbmd_step")


def lbmd_read_fields(ctx, rho_ptr, u_ptr, dst_is_device: int) -> None:
    _check(load().lbmd_read_fields(ctx, rho_ptr, u_ptr, dst_is_device), "lbmd_read_fields")


def lbmd_read_populations(ctx, f_ptr, dst_is_device: int) -> None:
    _check(load().lbmd_read_populations(ctx, f_ptr, dst_is_device), "lbmd_read_populations")


def lbmd_read_beads(ctx, pos_ptr, vel_ptr, dst_is_device: int) -> None:
    _check(load().lbmd_read_beads(ctx, pos_ptr, vel_ptr, dst_is_device), "lbmd_read_beads")


def bead_block_bytes(n_beads: int) -> int:
    """Bytes of the block lbmd_read_beads_async writes (LBMD_BEAD_BLOCK_BYTES)."""
    return 32 + 48 * int(n_beads)


def lbmd_step_read_async(ctx, dst_ptr, nbytes: int) -> None:
    """One coupled step and the read-out of its bead block into ``dst_ptr``
    (as lbmd_step(ctx, 1) + lbmd_read_beads_async, one graph launch for
    page-locked memory the device can address)."""
    _check(load().lbmd_step_read_async(ctx, dst_ptr, int(nbytes)), "lbmd_step_read_async")


def lbmd_read_beads_async(ctx, dst_ptr, nbytes: int) -> None:
    """Enqueue the status word, positions and velocities into page-locked host
    memory at ``dst_ptr`` (layout of LBMD_BEAD_BLOCK_BYTES); no synchronisation."""
    _check(load().lbmd_read_beads_async(ctx, dst_ptr, int(nbytes)), "lbmd_read_beads_async")


def decode_bead_block(block: np.ndarray, n_beads: int):
    """(status dict, positions (N, 3), velocities (N, 3)) of a uint8 block."""
    b = np.asarray(block, dtype=np.uint8)
    w = lbmd_status_word.from_buffer_copy(b[:C.sizeof(lbmd_status_word)].tobytes())
    d = b[32:32 + 48 * n_beads].view(np.float64)
    status = dict(step=w.step, n_trans=w.n_trans, state=w.state, t_transloc=w.t_transloc)
    return status, d[:3 * n_beads].reshape(n_beads, 3), d[3 * n_beads:].reshape(n_beads, 3)


def lbmd_read_bead_aux(ctx, ui_ptr, j_ptr, dst_is_device: int) -> None:
    _check(load().lbmd_read_bead_aux(ctx, ui_ptr, j_ptr, dst_is_device), "lbmd_read_bead_aux")


def lbmd_status(ctx) -> dict:
    s, nt, st, tt = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64()
    _check(load().lbmd_status(ctx, C.byref(s), C.byref(nt), C.byref(st), C.byref(tt)), "lbmd_status")
    return dict(step=s.value, n_trans=nt.value, state=st.value, t_transloc=tt.value)


def lbmd_solver_stats(ctx):
    it, bad = C.c_int32(), C.c_int32()
    _check(load().lbmd_solver_stats(ctx, C.byref(it), C.byref(bad)), "lbmd_solver_stats")
    return dict(newton_iters_last_step=it.value, failed_steps=bad.value)


def lbmd_set_kernel_timing(ctx, enable: bool) -> None:
    _check(load().lbmd_set_kernel_timing(ctx, int(bool(enable))), "lbmd_set_kernel_timing")


def lbmd_lb_kernel_time(ctx):
    ms, n = C.c_double(), C.c_int64()
    _check(load().lbmd_lb_kernel_time(ctx, C.byref(ms), C.byref(n)), "lbmd_lb_kernel_time")
    return ms.value, n.value


def lbmd_kernel_times(ctx) -> dict:
    lb, md, sp, n = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
    _check(load().lbmd_kernel_times(ctx, C.byref(lb), C.byref(md), C.byref(sp), C.byref(n)),
           "lbmd_kernel_times")
    return dict(lb_ms=lb.value, md_ms=md.value, spread_ms=sp.value, steps=n.value)


def lbmd_lb_step_noalloc(params: lbmd_params, f_in_ptr: int, f_out_ptr: int, stream_ptr: int) -> None:
    """One solvent stream-collide step on caller-owned device populations
    (pre-collision in, pre-collision out), without any allocation."""
    _check(load().lbmd_lb_step_noalloc(C.byref(params), C.c_void_p(f_in_ptr), C.c_void_p(f_out_ptr),
                                       C.c_void_p(stream_ptr)), "lbmd_lb_step_noalloc")


def _diag_dict(recs, n):
    return {k: np.array([getattr(recs[i], k) for i in range(n)]) for k in DIAG_FIELDS}


def lbmd_read_diagnostics(ctx, max_records: int) -> dict:
    """The chain diagnostic records so far, as a dict of arrays."""
    recs = (lbmd_diag * max(int(max_records), 1))()
    n = C.c_int32()
    _check(load().lbmd_read_diagnostics(ctx, C.cast(recs, C.c_void_p), int(max_records), C.byref(n)),
           "lbmd_read_diagnostics")
    return _diag_dict(recs, min(n.value, int(max_records)))


def lbmd_ensemble_read_diagnostics(ens, member: int, max_records: int) -> dict:
    recs = (lbmd_diag * max(int(max_records), 1))()
    n = C.c_int32()
    _check(load().lbmd_ensemble_read_diagnostics(ens, int(member), C.cast(recs, C.c_void_p),
                                                 int(max_records), C.byref(n)),
           "lbmd_ensemble_read_diagnostics")
    return _diag_dict(recs, min(n.value, int(max_records)))


def lbmd_destroy(ctx) -> None:
    _check(load().lbmd_destroy(ctx), "lbmd_destroy")


def lbmd_version() -> int:
    return load().lbmd_version()


# -- ensemble entry points ----------------------------------------------------
def lbmd_ensemble_workspace_size(members) -> int:
    n = C.c_size_t()
    _check(load().lbmd_ensemble_workspace_size(members, len(members), C.byref(n)),
           "lbmd_ensemble_workspace_size")
    return n.value


def lbmd_ensemble_create(members, workspace_ptr: int, nbytes: int, stream_ptr: int):
    h = C.c_void_p()
    _check(load().lbmd_ensemble_create(members, len(members), C.c_void_p(workspace_ptr), nbytes,
                                       C.c_void_p(stream_ptr), C.byref(h)), "lbmd_ensemble_create")
    return h


def lbmd_ensemble_step(ens, n: int) -> None:
    _check(load().lbmd_ensemble_step(ens, int(n)), "lbmd_ensemble_step")


def lbmd_ensemble_run(ens, max_steps: int, check_every: int = 1024) -> int:
    n = C.c_int64()
    _check(load().lbmd_ensemble_run(ens, int(max_steps), int(check_every), C.byref(n)),
           "lbmd_ensemble_run")
    return n.value


def lbmd_ensemble_results(ens, count: int) -> dict:
    state = np.empty(count, np.int32)
    tt = np.empty(count, np.int64)
    steps = np.empty(count, np.int64)
    nt = np.empty(count, np.int32)
    _check(load().lbmd_ensemble_results(ens, state.ctypes.data, tt.ctypes.data, steps.ctypes.data,
                                        nt.ctypes.data), "lbmd_ensemble_results")
    return dict(state=state, t_transloc=tt, steps=steps, n_trans=nt)


def lbmd_ensemble_live(ens) -> int:
    n = C.c_int32()
    _check(load().lbmd_ensemble_live(ens, C.byref(n)), "lbmd_ensemble_live")
    return n.value


def lbmd_ensemble_read_beads(ens, member: int, pos_ptr, vel_ptr, dst_is_device: int) -> None:
    _check(load().lbmd_ensemble_read_beads(ens, int(member), pos_ptr, vel_ptr, dst_is_device),
           "lbmd_ensemble_read_beads")


def lbmd_ensemble_read_populations(ens, member: int, f_ptr, dst_is_device: int) -> None:
    _check(load().lbmd_ensemble_read_populations(ens, int(member), f_ptr, dst_is_device),
           "lbmd_ensemble_read_populations")


def lbmd_ensemble_set_tuning(ens, rows: int, warps: int, claim: int, cells_per_thread: int = 1) -> None:
    _check(load().lbmd_ensemble_set_tuning(ens, int(rows), int(warps), int(claim), int(cells_per_thread)),
           "lbmd_ensemble_set_tuning")


def lbmd_ensemble_get_tuning(ens) -> dict:
    r, w, c, z = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().lbmd_ensemble_get_tuning(ens, C.byref(r), C.byref(w), C.byref(c), C.byref(z)),
           "lbmd_ensemble_get_tuning")
    return dict(rows=r.value, warps=w.value, claim=c.value, cells_per_thread=z.value)


def lbmd_ensemble_autotune(ens, trials: int = 3) -> float:
    ms = C.c_double()
    _check(load().lbmd_ensemble_autotune(ens, int(trials), C.byref(ms)), "lbmd_ensemble_autotune")
    return ms.value


def lbmd_ensemble_set_kernel_timing(ens, enable: bool) -> None:
    _check(load().lbmd_ensemble_set_kernel_timing(ens, int(bool(enable))),
           "lbmd_ensemble_set_kernel_timing")


def lbmd_ensemble_kernel_times(ens) -> dict:
    lb, st, n = C.c_double(), C.c_double(), C.c_int64()
    _check(load().lbmd_ensemble_kernel_times(ens, C.byref(lb), C.byref(st), C.byref(n)),
           "lbmd_ensemble_kernel_times")
    return dict(lb_ms=lb.value, step_ms=st.value, steps=n.value)


def lbmd_ensemble_destroy(ens) -> None:
    _check(load().lbmd_ensemble_destroy(ens), "lbmd_ensemble_destroy")


# -- convenience wrapper owning a torch workspace ---------------------------
class Simulation:
    """One box with (optionally) one chain, stepped on the GPU.

    The device workspace is a torch uint8 tensor owned by this object; the
    stream is the given torch stream (default: the current stream)."""

    def __init__(self, params: dict, init_pos=None, init_vel=None, init_rho=None, init_u=None,
                 bonds=None, device: str = "cuda", stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.p = full_params(params)
        self.device = torch.device(device)
        self.N = int(self.p["n_beads"])
        self.shape = (int(self.p["nz"]), int(self.p["ny"]), int(self.p["nx"]))
        self.V = self.shape[0] * self.shape[1] * self.shape[2]
        cp, keep = make_params(self.p, init_pos, init_vel, init_rho, init_u, bonds)
        nbytes = lbmd_workspace_size(cp)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.ctx = lbmd_create(cp, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        del keep
        self.workspace_bytes = nbytes

    def close(self) -> None:
        if getattr(self, "ctx", None):
            lbmd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        lbmd_step(self.ctx, n)

    def populations(self) -> np.ndarray:
        f = np.empty((19,) + self.shape, dtype=np.float32)
        lbmd_read_populations(self.ctx, f.ctypes.data, 0)
        return f

    def populations_device(self):
        import torch
        f = torch.empty((19,) + self.shape, dtype=torch.float32, device=self.device)
        lbmd_read_populations(self.ctx, f.data_ptr(), 1)
        return f

    def fields(self):
        rho = np.empty(self.shape, dtype=np.float32)
        u = np.empty((3,) + self.shape, dtype=np.float32)
        lbmd_read_fields(self.ctx, rho.ctypes.data, u.ctypes.data, 0)
        return rho, u

    def fields_device(self):
        import torch
        rho = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        lbmd_read_fields(self.ctx, rho.data_ptr(), u.data_ptr(), 1)
        return rho, u

    def beads(self):
        pos = np.empty((self.N, 3))
        vel = np.empty((self.N, 3))
        if self.N:
            lbmd_read_beads(self.ctx, pos.ctypes.data, vel.ctypes.data, 0)
        return pos, vel

    def bead_aux(self):
        ui = np.empty((self.N, 3))
        J = np.empty((self.N, 3))
        if self.N:
            lbmd_read_bead_aux(self.ctx, ui.ctypes.data, J.ctypes.data, 0)
        return ui, J

    def status(self) -> dict:
        return lbmd_status(self.ctx)

    def solver_stats(self) -> dict:
        return lbmd_solver_stats(self.ctx)

    def set_kernel_timing(self, enable: bool) -> None:
        lbmd_set_kernel_timing(self.ctx, enable)

    def lb_kernel_time(self):
        return lbmd_lb_kernel_time(self.ctx)

    def kernel_times(self) -> dict:
        return lbmd_kernel_times(self.ctx)

    def diagnostics(self) -> dict:
        """Recorded chain diagnostics (params diag_every / diag_capacity)."""
        return lbmd_read_diagnostics(self.ctx, max(int(self.p["diag_capacity"]), 1))


class Ensemble:
    """Many independent realisations (each a params dict with its own box,
    chain and seed; same storage and forcing) stepped together on the GPU.

    ``init_pos[k]`` is the (N_k, 3) start of chain k, or None for the
    library's seeded start; ``init_vel``, ``init_rho`` and ``init_u`` are
    optional lists of per-member arrays (entries may be None).  The device
    workspace is a torch uint8 tensor owned by this object."""

    def __init__(self, members, init_pos=None, device: str = "cuda", stream=None, init_vel=None,
                 init_rho=None, init_u=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        n = len(members)
        per = []
        for name, lst in (("init_pos", init_pos), ("init_vel", init_vel), ("init_rho", init_rho),
                          ("init_u", init_u)):
            if lst is None:
                lst = [None] * n
            if len(lst) != n:
                raise ValueError(f"one {name} entry per member")
            per.append(lst)
        self.p = [full_params(m) for m in members]
        self.count = len(self.p)
        self.device = torch.device(device)
        arr = (lbmd_params * self.count)()
        keep = []
        for k, m in enumerate(self.p):
            cp, kk = make_params(m, init_pos=per[0][k], init_vel=per[1][k], init_rho=per[2][k],
                                 init_u=per[3][k])
            arr[k] = cp
            keep.append(kk)
        nbytes = lbmd_ensemble_workspace_size(arr)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.ens = lbmd_ensemble_create(arr, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        del keep
        self.workspace_bytes = nbytes
        self.N = [int(m["n_beads"]) for m in self.p]
        self.shapes = [(int(m["nz"]), int(m["ny"]), int(m["nx"])) for m in self.p]

    def close(self) -> None:
        if getattr(self, "ens", None):
            lbmd_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        lbmd_ensemble_step(self.ens, n)

    def run(self, max_steps: int, check_every: int = 1024) -> int:
        return lbmd_ensemble_run(self.ens, max_steps, check_every)

    def results(self) -> dict:
        return lbmd_ensemble_results(self.ens, self.count)

    def live(self) -> int:
        return lbmd_ensemble_live(self.ens)

    def beads(self, member: int):
        N = self.N[member]
        pos = np.empty((N, 3))
        vel = np.empty((N, 3))
        lbmd_ensemble_read_beads(self.ens, member, pos.ctypes.data, vel.ctypes.data, 0)
        return pos, vel

    def populations(self, member: int) -> np.ndarray:
        f = np.empty((19,) + self.shapes[member], dtype=np.float32)
        lbmd_ensemble_read_populations(self.ens, member, f.ctypes.data, 0)
        return f

    def set_tuning(self, rows: int, warps: int, claim: int, cells_per_thread: int = 1) -> None:
        lbmd_ensemble_set_tuning(self.ens, rows, warps, claim, cells_per_thread)

    def tuning(self) -> dict:
        return lbmd_ensemble_get_tuning(self.ens)

    def autotune(self, trials: int = 3) -> float:
        return lbmd_ensemble_autotune(self.ens, trials)

    def set_kernel_timing(self, enable: bool) -> None:
        lbmd_ensemble_set_kernel_timing(self.ens, enable)

    def kernel_times(self) -> dict:
        return lbmd_ensemble_kernel_times(self.ens)

    def diagnostics(self, member: int) -> dict:
        return lbmd_ensemble_read_diagnostics(self.ens, member,
                                              max(int(self.p[member]["diag_capacity"]), 1))
