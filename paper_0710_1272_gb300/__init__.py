"""GB300 (sm_103a) implementation of the coupled lattice-Boltzmann / polymer-MD
step of Fyta, Melchionna, Kaxiras and Succi (arXiv:0710.1272).

The compute path is the CUDA library ``liblbmd.so`` (sources in ``csrc/``,
C ABI in ``include/lbmd.h``); :mod:`.lbmd` is its ctypes binding and
:class:`Simulation` (one box) and :class:`Ensemble` (many independent
realisations) are convenience wrappers that own a torch device workspace.
"""
from .lbmd import (  # noqa: F401
    COUPLING, ENS_XPAIR, FORCING, MAX_BEADS, NAN, RETRACTED, RUNNING, SHAKE_FAIL, STORAGE, STREAMING,
    TRANSLOCATED, Ensemble, LbmdError, Simulation, bead_block_bytes, decode_bead_block,
    full_params, lbmd_create, lbmd_destroy,
    lbmd_kernel_times, lbmd_lb_kernel_time, lbmd_lb_step_noalloc, lbmd_read_bead_aux,
    lbmd_read_beads, lbmd_read_beads_async, lbmd_step_read_async, lbmd_read_fields, lbmd_read_populations,
    lbmd_set_kernel_timing, lbmd_solver_stats, lbmd_status, lbmd_status_word, lbmd_step,
    lbmd_version, lbmd_workspace_size, load, make_params,
)
