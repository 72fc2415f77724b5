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
};

struct LbPhys {
  float omega;    // 1 / tau
  float rho0;
  float g[3];     // body force density
  int forcing;    // LBMD_FORCING_*
};

// Everything the MD kernel needs for one chain.
struct ChainArgs {
  LbGeom geo;
  const void *f;            // populations to gather from (post-collision of the
                            // previous step; pulled on the fly)
  const uint8_t *xslab;     // [nx]: 1 if the x-layer holds a solid node
  int has_wall, wall_x, wall_t, pore_d, pore_y0, pore_z0;
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
  const double *b0;         // [N-1] bond lengths
  int *nl_cnt, *wl_cnt;     // [N] list lengths
  short *nl_list;           // [N][kMaxPairs] partner beads
  float4 *wl_list;          // [N][kMaxWall] solid nodes (local frame)
  float4 *nl_ref;           // [N] positions at the last list build
  float *lam;               // [N] SHAKE multipliers of the last substep
  DevStatus *status;
};

size_t md_smem_bytes(int N);
int md_threads(int N);
// Opt the MD kernel into the dynamic shared memory a chain of N beads needs.
cudaError_t md_prepare(int N);

// Launchers (each returns the launch error, if any).
cudaError_t launch_lb_stream_collide(int storage, const LbGeom &g, const LbPhys &ph,
                                     const void *src, void *dst, DevStatus *bump,
                                     cudaStream_t s);
cudaError_t launch_init_populations(int storage, const LbGeom &g, float rho0,
                                    const float *rho, const float *u, float tg_amp,
                                    void *dst, cudaStream_t s);
cudaError_t launch_read_moments(int storage, const LbGeom &g, const LbPhys &ph,
                                const void *src, long long z0, long long nzc,
                                float *rho, float *u, long long ustride, cudaStream_t s);
cudaError_t launch_read_pulled(int storage, const LbGeom &g, float rho0, const void *src,
                               long long z0, long long nzc, float *f, long long fstride,
                               cudaStream_t s);
cudaError_t launch_gather(int storage, const ChainArgs &a, cudaStream_t s);
cudaError_t launch_md_cycle(const ChainArgs &a, int priority, cudaStream_t s);
cudaError_t launch_spread(int storage, const LbGeom &g, const int *sp_node, const float *sp_w,
                          const float4 *J, int N, int nw, void *dst, DevStatus *bump,
                          cudaStream_t s);
cudaError_t launch_read_beads(const float4 *pos, const float4 *pos_lo, const float4 *vel, int N,
                              int ox, int oy, int oz, double *dpos, double *dvel, cudaStream_t s);
cudaError_t launch_read_bead_aux(const float4 *ui, const float4 *J, int N, double *dui,
                                 double *dJ, cudaStream_t s);

}  // namespace lbmd
