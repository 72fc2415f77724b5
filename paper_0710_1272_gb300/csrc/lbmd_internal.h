// lbmd_internal.h -- host/device interface between the C-ABI layer and the
// kernels of the coupled LB / polymer-MD step.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbmd.h"

namespace lbmd {

// Per-chain status word kept in device memory (one per chain).
struct DevStatus {
  long long step;        // LB steps completed
  long long t_transloc;  // first step with N_T = N, -1 before
  int n_trans;           // beads with unwrapped x < wall_x
  int max_trans;         // largest N_T seen
  int state;             // LBMD_RUNNING, ...
  int shake_fail;        // LB steps whose constraint solve hit the iteration cap
  int newton_iters;      // Newton iterations of the last LB step (all substeps)
  int nl_builds;         // neighbour-list builds so far (0: none yet)
  int nl_ok;             // 1 if the current lists hold every pair (no overflow)
  int out_buf;           // ensemble: population buffer (0/1) written by the last step
  int diag_count;        // diagnostic records written
  int pop_bad;           // 1 once a stream-collide met a node whose populations
                         // are not all finite (density not finite)
};

// One record of the Sec. III chain diagnostics (end of an LB step).
struct DevDiag {
  long long step;        // LB steps completed
  int n_trans;           // N_T
  float r_u, r_t, r_e;   // radii of gyration (untranslocated, translocated, effective)
  float s_h, s_e;        // work rates of the fluid (Eq. 13) and of the drive (Eq. 14)
  float kinetic;         // m/2 sum |v|^2
  int pad;
};

// Neighbour-list capacities per bead: bead partners and solid nodes within
// r_c + skin (a sphere of radius 2.83 holds at most ~100 lattice nodes).
constexpr int kMaxPairs = 48;
constexpr int kMaxWall = 128;

// Lattice geometry as the kernels see it.
struct LbGeom {
  int nx, ny, nz;
  int ntx;                      // x-tiles of 32 nodes = words per bitfield row
  long long V;                  // nx * ny * nz
  long long Vp;                 // population stride (V rounded up to 64)
  const uint32_t *solid;        // [nz][ny][ntx] words, bit x & 31 of word x >> 5
  const uint8_t *tile_near;     // [nz][ny][ntx]: 1 if a solid node is within one
                                // node of the tile's 32 cells (incl. themselves)
  const uint32_t *lmask;        // [nz][ny][nx] link mask: bit p (1..18) set if the
                                // pull source x - c_p is solid, bit 0 if x is
};

// Where the populations of a box are held between two steps; this decides
// how the pre-collision value h_p(x, t) is fetched and where the bead source
// of stage (3) is added.
//   kPopPull:    two-buffer pull streaming; the buffer holds the post-collision
//                h*_p(x) of the last step at [p][x].
//   kPopAALocal: in-place (AA) streaming after an odd step (and at the start):
//                the buffer holds the pre-collision h_p(x, t) at [p][x].
//   kPopAASwap:  in-place streaming after an even step: the buffer holds the
//                post-collision h*_p(x) at [opp(p)][x].
constexpr int kPopPull = 0;
constexpr int kPopAALocal = 1;
constexpr int kPopAASwap = 2;

// Collision variant for a zero body force: both forcing schemes then reduce
// to plain BGK (no velocity shift, no source term), so the kernels skip them.
constexpr int kForcingNone = 2;

struct LbPhys {
  float omega;    // 1 / tau
  float rho0;
  float g[3];     // body force density
  int forcing;    // LBMD_FORCING_*
  // thermal source F_p of Eq. 5 (used only by the fluctuating kernels):
  float fl_amp[15];          // a_k = sqrt(3 kT (1 - (1 - omega)^2) / b_k), k = 4..18
  unsigned long long seed;   // Philox key
  const long long *step;     // LB steps completed (the noise counter); null: no noise
  int *nonfinite;            // set to 1 by a collision whose density is not finite
};

// Impulse sum of one transfer node in the bead spread (stage 3): the three
// components as 64-bit fixed point (units of 2^-40) and a flag that is set
// when a contribution was not finite.  Integer addition is associative, so the
// sum -- and the populations it is added to -- do not depend on the order in
// which the (bead, corner) contributions arrive.  At rest all zero.
struct __align__(32) SpreadAcc {
  long long x, y, z;
  long long bad;
};

// Everything the MD kernel needs for one chain.
struct ChainArgs {
  LbGeom geo;
  const void *f;            // populations to gather from (kPop* layout f_mode)
  int f_mode;
  int has_wall, wall_x, wall_t, pore_d, pore_y0, pore_z0, y_walls;  // Sec. III geometry
  float rho0, g[3];
  int forcing, coupling;
  int N, M, has_bonds, shake_maxit;
  float dt, mass, gamma, kT, sigma, eps, kappa, fdrive, shake_tol;
  unsigned long long seed;
  int ox, oy, oz;           // integer origin of the chain's local frame
  float4 *pos, *pos_lo;     // local positions (unwrapped - origin) as hi + lo
  float4 *vel;
  float4 *ui, *J;           // interpolated u and impulse of the last step
  int *sp_node;             // [8N] grid node of each transfer weight, -1 none
  float *sp_w;              // [8N] renormalised transfer weights
  int *owner;               // [V] per node: smallest transfer entry of this step
                            // that hits it (kOwnerFree at rest); null without
                            // a solvent
  SpreadAcc *acc;           // [8N] impulse sums, at the owner entry of each node
  float4 *sp_src;           // [8N] apply records (F_x, F_y, F_z, node) of the
                            // transfer nodes, F the node's summed force; unused
                            // records have node = -1 (single box)
  const double *b0;         // [N-1] bond lengths
  int *nl_cnt, *wl_cnt;     // [N] list lengths
  short *nl_list;           // [N][kMaxPairs] partner beads
  float4 *wl_list;          // [N][kMaxWall] solid nodes (local frame)
  float4 *nl_ref;           // [N] positions at the last list build
  float *lam;               // [N] SHAKE multipliers of the last substep
  DevStatus *status;
  DevDiag *diag;            // [diag_cap] diagnostic records
  int diag_every, diag_cap; // record every diag_every steps (0: never)
};

// One realisation of an ensemble as every ensemble kernel sees it: its box,
// its chain and its two population buffers.  An array of these lives in
// device memory; kernels index it by realisation.
struct EnsMember {
  ChainArgs a;      // chain, geometry (a.geo) and bead buffers; a.f unused
  LbPhys ph;
  void *pop[2];     // post-collision populations, swapped every step
};

// What the ensemble stream-collide needs of one realisation, 16-byte aligned
// so that a block reads it with six vector loads.
struct __align__(16) EnsLb {
  void *pop[2];                 // post-collision populations, swapped every step
  const uint32_t *lmask;        // as LbGeom::lmask
  const uint8_t *tile_near;     // as LbGeom::tile_near
  int nx, ny, nz, ntx;
  int Vp;                       // population stride (19 Vp < 2^31)
  float inv_nx;                 // 1 / nx, for the row of a node in its plane
  float omega, rho0;
  float g[3];
  int forcing;
  int *nonfinite;               // the realisation's DevStatus::pop_bad
};

// Work item of the ensemble stream-collide: 32 x rows consecutive nodes
// r0 .. r0 + 32 rows - 1 (x fastest, clipped to the plane) of z-plane z of
// realisation m.
struct __align__(16) EnsTile {
  int m, z, r0, pad;
};

size_t md_smem_bytes(int N);
int md_threads(int N);
// Opt the MD kernels into the dynamic shared memory of the longest chain.
cudaError_t md_prepare();

// Launchers (each returns the launch error, if any).
cudaError_t launch_lb_stream_collide(int storage, const LbGeom &g, const LbPhys &ph,
                                     const void *src, void *dst, DevStatus *bump,
                                     cudaStream_t s);
// Stream-collide with the thermal source (ph.step != null); `bump` as above.
cudaError_t launch_lb_stream_collide_fluct(int storage, const LbGeom &g, const LbPhys &ph,
                                           const void *src, void *dst, cudaStream_t s);
// Per-mode noise amplitudes a_k (k = 4..18) of the thermal source.
void fluct_amplitudes(double kT, double tau, float amp[15]);
// status->step += 1 (one thread): the step count of a box without beads when
// the stream-collide reads it.
cudaError_t launch_bump_step(DevStatus *status, cudaStream_t s);

// Fill g.lmask from the solid bitfield (once, at set-up).
cudaError_t launch_link_mask(const LbGeom &g, uint32_t *mask, cudaStream_t s);
cudaError_t launch_init_populations(int storage, const LbGeom &g, float rho0,
                                    const float *rho, const float *u, float tg_amp,
                                    void *dst, cudaStream_t s);
// In-place streaming: f = f_eq(rho, u) stored locally (kPopAALocal) on the
// z-slab [z0, z0 + nzc); rho / u (or null) hold the slab's fields with
// component stride `ustride`.
cudaError_t launch_init_local(int storage, const LbGeom &g, float rho0, const float *rho,
                              const float *u, long long ustride, float tg_amp, long long z0,
                              long long nzc, void *dst, cudaStream_t s);
// One in-place (AA-pattern) stream-collide on `buf`: odd = 0 takes the buffer
// from kPopAALocal to kPopAASwap, odd = 1 back.  `bump` as for
// launch_lb_stream_collide; the _fluct variant adds the thermal source.
cudaError_t launch_lb_aa(int storage, const LbGeom &g, const LbPhys &ph, void *buf, int odd,
                         DevStatus *bump, cudaStream_t s);
cudaError_t launch_lb_aa_fluct(int storage, const LbGeom &g, const LbPhys &ph, void *buf,
                               int odd, cudaStream_t s);
// Read-outs of the pre-collision state of populations held in layout `mode`.
cudaError_t launch_read_moments(int storage, const LbGeom &g, const LbPhys &ph,
                                const void *src, int mode, long long z0, long long nzc,
                                float *rho, float *u, long long ustride, cudaStream_t s);
cudaError_t launch_read_pulled(int storage, const LbGeom &g, float rho0, const void *src,
                               int mode, long long z0, long long nzc, float *f,
                               long long fstride, cudaStream_t s);
cudaError_t launch_gather(int storage, const ChainArgs &a, cudaStream_t s);
cudaError_t launch_md_cycle(const ChainArgs &a, int priority, cudaStream_t s);
// Spread of the bead impulses (stage 3), independent of the order of
// concurrent atomics, so that a step gives the same bits in every run:
//  - the gather claims each transfer node for the smallest (bead, corner)
//    entry that hits it: atomicMin on owner[node], which rests at kOwnerFree
//    (every byte 0x7f, so a memset prepares the field);
//  - sum (any time after the MD cycle; all contributions to a box come from
//    its one chain): every entry adds its share -w J_i of the impulse to
//    acc[owner] in 64-bit fixed point; then each owner converts its sum once
//    (into the record sp_src[owner] = (F, node), or in the apply itself) and
//    returns acc and owner[node] to rest;
//  - apply (after the stream-collide): each owner entry adds the source
//    S_p = 3 w_p c_p . F to its node's post-collision populations of `dst` in
//    layout `mode` -- the only write to those words.
// The sums run in kernels of their own after the MD cycle, spread over many
// SMs (global atomics from one SM, in the MD block, were slow while the
// stream-collide saturates HBM).  launch_spread_sum enqueues the sum as two
// kernels, or only the first when the apply converts the sums itself
// (records == false); an ensemble uses launch_ens_spread_accum and converts
// in its apply.
constexpr int kOwnerFree = 0x7f7f7f7f;
cudaError_t launch_spread_sum(const ChainArgs &a, bool records, cudaStream_t s);
// Single box: true when the apply should convert the sums itself (the MD
// branch sets the step), false when the stream-collide sets it -- taken as a
// stream-collide moving 480 MB or more per step (~70 us at the HBM rate, about
// the MD branch of a 400-bead chain beside it): FP32 populations of 3.2 M
// nodes or more.
inline bool spread_take_in_apply(int storage, long long nodes) {
  const long long bytes = 2LL * 19 * nodes * (storage == LBMD_STORE_F32 ? 4 : 2);
  return bytes < 480000000LL;
}
// `take`: the owners' forces from their fixed-point sums (the sum ran with
// records == false), else from the records.  `bump` (may be null):
// status->step += 1 by one thread.
cudaError_t launch_spread_apply(int storage, const LbGeom &g, const ChainArgs &a, void *dst,
                                int mode, bool take, DevStatus *bump, cudaStream_t s);
// Ensemble launchers.  `live` points at the flags of the current step (one int
// per realisation); realisations whose flag is 0 are skipped by every kernel.
// Stream-collide: `grid` blocks of 32 x rows threads (rows 4, 8 or 16;
// registers sized for `warps` = 32 or 48 resident warps per SM), block b
// updating tiles [b claim, (b + 1) claim) of the *n_tiles listed (blocks past
// the end return).  Every realisation must have 19 Vp < 2^31 (32-bit offsets)
// and nx * ny < 2^22 (float row division).
// forcing: LBMD_FORCING_* or kForcingNone (every realisation has g = 0).
// cpt: cells per thread, 1; 2 (two consecutive z-planes); or kEnsXPair (two
// x-adjacent nodes sharing a 32-bit word, 16-bit storage).  The two-cell
// shapes need warps 32 and rows 4 or 8 -- other shapes are
// cudaErrorInvalidValue.
constexpr int kEnsXPair = LBMD_ENS_XPAIR;
cudaError_t launch_ens_stream_collide(int storage, int forcing, int rows, int warps, int cpt,
                                      int claim, int grid, const EnsLb *lbd, const EnsTile *tiles,
                                      const int *n_tiles, const int *live, int cur,
                                      cudaStream_t s);
// Blocks of that kernel that fit on one SM (0: no such shape).
int ens_lb_blocks_per_sm(int storage, int forcing, int rows, int warps, int cpt);
// Gather for every (realisation, bead) of `beads` (padded entries have m < 0).
cudaError_t launch_ens_gather(int storage, const EnsMember *mem, const int2 *beads, int nb,
                              const int *live, int cur, cudaStream_t s);
// MD cycle of the `count` chains listed in `chains`, one block of `threads`
// threads each, with dynamic shared memory for `max_n` beads.
cudaError_t launch_ens_md_cycle(const EnsMember *mem, const int *chains, int count, int threads,
                                int max_n, const int *live, int priority, cudaStream_t s);
// Sum part of the spread of every live realisation (after every MD group).
cudaError_t launch_ens_spread_accum(const EnsMember *mem, const int2 *beads, int nb,
                                    const int *live, cudaStream_t s);
// Apply part of the spread (the owners convert their sums) into pop[1 - cur];
// bumps each live realisation's step
// count and writes its flag for the next step into `live_next` (still running
// and step < *max_steps).
cudaError_t launch_ens_spread(int storage, const EnsMember *mem, const int2 *beads, int nb,
                              const int *live, int *live_next, int cur,
                              const long long *max_steps, cudaStream_t s);

cudaError_t launch_read_beads(const float4 *pos, const float4 *pos_lo, const float4 *vel, int N,
                              int ox, int oy, int oz, double *dpos, double *dvel, cudaStream_t s);
// The block of lbmd_read_beads_async into device memory `out` (32 + 48 N bytes).
constexpr size_t kBeadBlockHeader = 32;
cudaError_t launch_bead_block(const ChainArgs &a, const DevStatus *st, void *out, cudaStream_t s);
// The kernel launch_bead_block launches (to find its node in a captured graph;
// its arguments: pos, pos_lo, vel, N, ox, oy, oz, status, out).
const void *bead_block_kernel();
cudaError_t launch_read_bead_aux(const float4 *ui, const float4 *J, int N, double *dui,
                                 double *dJ, cudaStream_t s);

}  // namespace lbmd
