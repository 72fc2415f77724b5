// lbmd_host.h -- host-side setup shared by the single-box context
// (lbmd_abi.cu) and the ensemble (ensemble_abi.cu): parameter checks, the
// workspace layout of one box, the Sec. III geometry and the upload of the
// initial state.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lbmd_internal.h"

namespace lbmd {

// Records the message returned by lbmd_last_message (per thread) and
// returns `code`.
int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
const char *last_message();

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
inline size_t store_bytes(int storage) { return storage == LBMD_STORE_F32 ? 4 : 2; }

// Byte offsets of every buffer of one box inside its workspace slice.
struct Layout {
  size_t popA, popB, solid, tile, lmask, pos, pos_lo, vel, ui, J, sp_node, sp_w, b0, nl_cnt, wl_cnt,
      nl_list, wl_list, nl_ref, lam, status, diag, owner, acc, sp_src, stage;
  size_t stage_floats;  // staging capacity in floats (0 without a staging buffer)
  size_t total;
  long long Vp;
  int ntx;
  long long chunk_cells;
};

// single_box: the layout of a single-box context (with the host read-out
// staging buffer and the spread records); false: of an ensemble member (the
// ensemble keeps one staging buffer for all its members, and its apply
// converts the spread sums without records).
Layout make_layout(const lbmd_params &p, bool single_box);
// Floats of staging a box needs for chunked host read-outs.
size_t stage_floats_for(const lbmd_params &p);
long long chunk_cells_for(const lbmd_params &p);

int validate(const lbmd_params *p);
bool params_have_bonds(const lbmd_params &p);

// The library's own initial chain for params with init_pos == NULL (Sec. III:
// the chain starts on the cis side with one end in the pore): a seeded
// off-lattice self-avoiding walk, 3 n_beads doubles [i][xyz] (unwrapped).
// Returns LBMD_OK, or LBMD_EINVAL when no such walk fits the box.
int seeded_start(const lbmd_params &p, std::vector<double> &pos);

// Copy the diagnostic records of one chain to the host (synchronises s).
int copy_diagnostics(const DevStatus *status, const DevDiag *diag, int cap, lbmd_diag *records,
                     int32_t max_records, int32_t *n_records, cudaStream_t s);

// Device views of one initialised box and its chain.
struct Instance {
  LbGeom geo;
  LbPhys phys;
  ChainArgs chain;
  char *pop[2];
  DevStatus *status;
  int has_bonds;
};

// Uploads the geometry, the initial populations (pull streaming: post-collision
// buffer pop[0] such that the first pull gives f_eq(rho, u); in-place
// streaming: f_eq(rho, u) itself, kPopAALocal), the beads and the status
// word of box `p` into the workspace slice `ws` laid out by `L`, on stream s,
// and synchronises s (the host staging must outlive the copies).  On error
// returns the CUDA error and sets *what.
cudaError_t init_instance(const lbmd_params &p, const Layout &L, char *ws, cudaStream_t s,
                          Instance &out, const char **what);

}  // namespace lbmd
