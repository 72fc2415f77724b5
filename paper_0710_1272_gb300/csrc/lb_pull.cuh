// lb_pull.cuh -- pull streaming with halfway bounce-back, shared by the
// stream-collide kernels, the read-out kernels and the bead gather.
#pragma once

#include "lbmd_common.cuh"

namespace lbmd {

// Pre-collision deviations h_p(x, t+1) of node (x, y, z) from the
// post-collision buffer `src` (Eq. 5 free streaming, pull form):
//   h_p(x) = h*_p(x - c_p)      if x - c_p is fluid,
//   h_p(x) = h*_opp(p)(x)       otherwise (the population that left x towards
//                               the solid node comes back reversed),
// where bit p of `bb` says whether x - c_p is solid (the node's link mask; 0
// for a node known to be far from any solid node).  h*_q(y) sits at [q][y]
// (SWAP = false, kPopPull) or at [opp(q)][y] (SWAP = true, kPopAASwap).  I is
// the index type of the population offsets: int when 19 Vp < 2^31 (cheaper
// address arithmetic), size_t otherwise.
template <int S, typename I = size_t, bool SWAP = false>
__device__ __forceinline__ void pull19_mask(const LbGeom &g,
                                            const typename Store<S>::T *__restrict__ src, int x,
                                            int y, int z, uint32_t bb, float h[kQ]) {
  using St = Store<S>;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int xm = wrap_m1(x, nx), xp = wrap_p1(x, nx);
  const int ym = wrap_m1(y, ny), yp = wrap_p1(y, ny);
  const int zm = wrap_m1(z, nz), zp = wrap_p1(z, nz);
  const I self = ((I)z * ny + y) * nx + x;
  const I Vp = (I)g.Vp;
#pragma unroll
  for (int p = 0; p < kQ; ++p) {
    // source node x - c_p
    const int sx = cx(p) == 1 ? xm : (cx(p) == -1 ? xp : x);
    const int sy = cy(p) == 1 ? ym : (cy(p) == -1 ? yp : y);
    const int sz = cz(p) == 1 ? zm : (cz(p) == -1 ? zp : z);
    const I sidx = (I)(SWAP ? opp(p) : p) * Vp + ((I)sz * ny + sy) * nx + sx;
    const I bidx = (I)(SWAP ? p : opp(p)) * Vp + self;
    h[p] = St::load(src + (((bb >> p) & 1u) ? bidx : sidx));
  }
}

__device__ __forceinline__ bool tile_is_near(const LbGeom &g, int x, int y, int z) {
  return __ldg(&g.tile_near[((size_t)z * g.ny + y) * g.ntx + (x >> 5)]) != 0;
}

// Pre-collision deviations h_p(x, t) of fluid node (x, y, z) for populations
// held in layout `mode` (kPop*), taking the link mask only where a solid node
// is within one node of the node's tile.  For read-outs and the bead gather,
// which run while no kernel writes `src`.
template <int S, typename I = size_t>
__device__ __forceinline__ void fetch19(const LbGeom &g, const typename Store<S>::T *__restrict__ src,
                                        int x, int y, int z, int mode, float h[kQ]) {
  using St = Store<S>;
  const I self = ((I)z * g.ny + y) * g.nx + x;
  if (mode == kPopAALocal) {
#pragma unroll
    for (int p = 0; p < kQ; ++p) h[p] = St::load(src + (I)p * (I)g.Vp + self);
    return;
  }
  const uint32_t bb = tile_is_near(g, x, y, z) ? __ldg(&g.lmask[self]) : 0u;
  if (mode == kPopAASwap)
    pull19_mask<S, I, true>(g, src, x, y, z, bb, h);
  else
    pull19_mask<S, I, false>(g, src, x, y, z, bb, h);
}

// rho - rho0 and the momentum sum_p h_p c_p (sum_p w_p c_p = 0).
__device__ __forceinline__ void moments19(const float h[kQ], float &drho, float &jx, float &jy,
                                          float &jz) {
  drho = 0.f;
  jx = jy = jz = 0.f;
#pragma unroll
  for (int p = 0; p < kQ; ++p) {
    drho += h[p];
    if (cx(p)) jx += cx(p) > 0 ? h[p] : -h[p];
    if (cy(p)) jy += cy(p) > 0 ? h[p] : -h[p];
    if (cz(p)) jz += cz(p) > 0 ? h[p] : -h[p];
  }
}

}  // namespace lbmd
