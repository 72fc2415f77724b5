// lb_ensemble.cu -- the ensemble stream-collide: one kernel over the tiles of
// every live realisation, and the dispatch over its launch shapes for the
// autotuner.
#include <type_traits>

#include "lb_collide.cuh"

namespace lbmd {

// Ensemble stream-collide: block b updates tiles [b claim, (b + 1) claim) of
// the tile list of every live realisation.  The blocks are not persistent: they
// retire all through the launch, so the MD blocks of the same step, launched
// beside it at a higher priority, find SMs as they become ready (a persistent
// grid held every SM to the end and left the MD blocks that did not fit at
// the start to run after it).  A tile is 32 x ROWS consecutive
// nodes of one z-plane -- or of two consecutive planes with CPT = 2, a thread
// updating the node of each plane at the same (x, y) with all 38 loads issued
// before either collision -- so a warp reads and writes one contiguous run of
// every population whatever the box width (no idle lanes for widths that are
// not a multiple of 32).  With CPT = 3 (16-bit storage) a thread takes two
// x-adjacent nodes instead, whose deviations share a 32-bit word (pair_node),
// and a tile is 64 x ROWS consecutive nodes of one plane (every member's nx
// is even, so a pair never straddles a row).  A warp takes the bounce-back checks if any of its
// nodes needs them.  WARPS is the occupancy the register budget is sized for:
// 48 warps per SM (40 registers, a little spilling) or 32 (64 registers,
// none); population offsets are 32-bit.
template <int S, int FORCING, int ROWS, int WARPS, int CPT>
__global__ void __launch_bounds__(32 * ROWS, WARPS / ROWS)
    k_ens_stream_collide(const EnsLb *__restrict__ lbd, const EnsTile *__restrict__ tiles,
                         const int *__restrict__ n_tiles, const int *__restrict__ live, int cur,
                         int claim) {
  using T = typename Store<S>::T;
  const int n = *n_tiles;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int first = blockIdx.x * claim;
  if (first >= n) return;  // the grid covers the longest tile list since the last upload
  const int last = min(first + claim, n);
  for (int t = first; t < last; ++t) {
    const int4 w = __ldg(reinterpret_cast<const int4 *>(tiles) + t);  // (m, z0, r0, planes)
    if (!__ldg(&live[w.x])) continue;
    EnsLb d;
    {
      const int4 *q = reinterpret_cast<const int4 *>(lbd + w.x);
      int4 *o = reinterpret_cast<int4 *>(&d);
#pragma unroll
      for (int k = 0; k < (int)(sizeof(EnsLb) / 16); ++k) o[k] = __ldg(q + k);
    }
    LbGeom g;
    g.nx = d.nx;
    g.ny = d.ny;
    g.nz = d.nz;
    g.ntx = d.ntx;
    g.V = 0;
    g.Vp = d.Vp;
    g.solid = nullptr;  // the link mask replaces the bitfield here
    g.tile_near = d.tile_near;
    g.lmask = d.lmask;
    LbPhys ph;
    ph.omega = d.omega;
    ph.rho0 = d.rho0;
    ph.g[0] = d.g[0];
    ph.g[1] = d.g[1];
    ph.g[2] = d.g[2];
    ph.forcing = FORCING;
    ph.nonfinite = d.nonfinite;
    // node of this thread: row-major index r in the plane, its row by a
    // float reciprocal with a one-step correction (exact for nx * ny < 2^22)
    const int plane = d.nx * d.ny;
    const int r = w.z + (CPT == 3 ? 2 * tid : tid);
    const bool active = r < plane;
    int y = __float2int_rz((float)r * d.inv_nx);
    int x = r - y * d.nx;
    if (x < 0) {
      --y;
      x += d.nx;
    } else if (x >= d.nx) {
      ++y;
      x -= d.nx;
    }
    const T *src = (const T *)(cur ? d.pop[1] : d.pop[0]);
    T *dst = (T *)(cur ? d.pop[0] : d.pop[1]);
    if constexpr (CPT == 3) {
      using T2 = typename std::conditional<S == LBMD_STORE_F16, __half2, __nv_bfloat162>::type;
      const bool near = __any_sync(0xffffffffu, active && tile_is_near(g, x, y, w.y));
      if (active)
        pair_node<T2, FORCING>(g, ph, (const uint32_t *)src, (uint32_t *)dst, x >> 1, y, w.y, near);
    } else if (CPT == 2 && w.w == 2) {
      const bool near = __any_sync(0xffffffffu, active && (tile_is_near(g, x, y, w.y) ||
                                                            tile_is_near(g, x, y, w.y + 1)));
      if (active) stream_collide_node2<S, FORCING>(g, ph, src, dst, x, y, w.y, near);
    } else {
      const bool near = __any_sync(0xffffffffu, active && tile_is_near(g, x, y, w.y));
      if (active) stream_collide_node<S, FORCING, int>(g, ph, src, dst, x, y, w.y, near);
    }
  }
}

template <int S, int FORCING, int ROWS, int WARPS, int CPT>
static cudaError_t ens_lb_launch(int claim, int grid, const EnsLb *lbd, const EnsTile *tiles,
                                 const int *n_tiles, const int *live, int cur, cudaStream_t s) {
  k_ens_stream_collide<S, FORCING, ROWS, WARPS, CPT><<<grid, dim3(32, ROWS), 0, s>>>(
      lbd, tiles, n_tiles, live, cur, claim);
  return cudaGetLastError();
}

template <int S, int FORCING, int ROWS, int WARPS, int CPT>
static int ens_lb_occupancy() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_stream_collide<S, FORCING, ROWS, WARPS, CPT>,
                                                    32 * ROWS, 0) != cudaSuccess)
    return 0;
  return n;
}

// Dispatch on (storage, forcing, rows, warps per SM, cells per thread) to one
// instantiation.  Two cells per thread need the 64-register budget (warps =
// 32) and come with rows 4 and 8 only; other combinations return null.
struct EnsLbFns {
  cudaError_t (*launch)(int, int, const EnsLb *, const EnsTile *, const int *, const int *, int,
                        cudaStream_t);
  int (*occupancy)();
};
template <int S, int F, int R>
static EnsLbFns ens_fns_warps(int warps, int cpt) {
  if (cpt == 3) {  // x-pairs: 16-bit storage, 64 registers, rows 4 or 8
    if constexpr (S == LBMD_STORE_F32) {
      return {nullptr, nullptr};
    } else {
      if (warps != 32 || R == 16) return {nullptr, nullptr};
      return {&ens_lb_launch<S, F, R, 32, 3>, &ens_lb_occupancy<S, F, R, 32, 3>};
    }
  }
  if (cpt == 2) {
    if (warps != 32 || R == 16) return {nullptr, nullptr};
    return {&ens_lb_launch<S, F, R, 32, 2>, &ens_lb_occupancy<S, F, R, 32, 2>};
  }
  if (warps == 32) return {&ens_lb_launch<S, F, R, 32, 1>, &ens_lb_occupancy<S, F, R, 32, 1>};
  return {&ens_lb_launch<S, F, R, 48, 1>, &ens_lb_occupancy<S, F, R, 48, 1>};
}
template <int S, int F>
static EnsLbFns ens_fns_rows(int rows, int warps, int cpt) {
  if (rows == 4) return ens_fns_warps<S, F, 4>(warps, cpt);
  if (rows == 16) return ens_fns_warps<S, F, 16>(warps, cpt);
  return ens_fns_warps<S, F, 8>(warps, cpt);
}
template <int S>
static EnsLbFns ens_fns_store(int forcing, int rows, int warps, int cpt) {
  if (forcing == kForcingNone) return ens_fns_rows<S, kForcingNone>(rows, warps, cpt);
  if (forcing == LBMD_FORCING_GUO) return ens_fns_rows<S, LBMD_FORCING_GUO>(rows, warps, cpt);
  return ens_fns_rows<S, LBMD_FORCING_PAPER>(rows, warps, cpt);
}
static EnsLbFns ens_fns(int storage, int forcing, int rows, int warps, int cpt) {
  if (storage == LBMD_STORE_F16) return ens_fns_store<LBMD_STORE_F16>(forcing, rows, warps, cpt);
  if (storage == LBMD_STORE_BF16) return ens_fns_store<LBMD_STORE_BF16>(forcing, rows, warps, cpt);
  return ens_fns_store<LBMD_STORE_F32>(forcing, rows, warps, cpt);
}

cudaError_t launch_ens_stream_collide(int storage, int forcing, int rows, int warps, int cpt,
                                      int claim, int grid, const EnsLb *lbd, const EnsTile *tiles,
                                      const int *n_tiles, const int *live, int cur,
                                      cudaStream_t s) {
  if (storage < LBMD_STORE_F32 || storage > LBMD_STORE_BF16) return cudaErrorInvalidValue;
  const EnsLbFns f = ens_fns(storage, forcing, rows, warps, cpt);
  if (!f.launch || grid < 1 || claim < 1) return cudaErrorInvalidValue;
  return f.launch(claim, grid, lbd, tiles, n_tiles, live, cur, s);
}

int ens_lb_blocks_per_sm(int storage, int forcing, int rows, int warps, int cpt) {
  const EnsLbFns f = ens_fns(storage, forcing, rows, warps, cpt);
  return f.occupancy ? f.occupancy() : 0;
}

}  // namespace lbmd
