// lb_aa.cuh -- in-place (AA-pattern) streaming of the D3Q19 populations
// (Bailey, Myre, Walsh, Lilja and Saar, ICPP 2009): one population buffer
// instead of two, the same Eq. 5 update and the same bytes moved per node.
//
// Two kinds of step alternate, and each reads and writes the same 19 slots
// per node, so every update is race-free in place:
//   even step (buffer kPopAALocal -> kPopAASwap): node x reads its own
//     h_p(x) at [p][x], collides, and writes h*_p(x) to [opp(p)][x];
//   odd step (buffer kPopAASwap -> kPopAALocal): node x pulls
//       h_p(x) = [opp(p)][x - c_p]  (h*_p(x - c_p), streamed), or
//                [p][x]             (h*_opp(p)(x), bounced back) if x - c_p is solid,
//     collides, and pushes h*_p(x) to
//       [p][x + c_p]                (the next even step's h_p(x + c_p)), or
//       [opp(p)][x]                 (its h_opp(p)(x): halfway bounce-back) if x + c_p is solid.
// Re-indexed with q = opp(p), the odd step's write set at x is
// {[opp(q)][x - c_q] : x - c_q fluid} u {[q][x] : x - c_q solid}, its read set;
// a slot belongs to one fluid node only, and no node reads a slot of a solid
// node.  The bounce-back of Eq. 5's pull form is thus reproduced exactly.
//
// The buffer is read and written by the same kernel, so it is accessed
// through a plain (non-restrict, non-const) pointer: no load may take the
// read-only data path.
#pragma once

#include "lb_collide.cuh"

namespace lbmd {

template <int S, int FORCING, typename I, bool ODD, bool FLUCT>
__device__ __forceinline__ void aa_node(const LbGeom &g, const LbPhys &ph,
                                        typename Store<S>::T *buf, int x, int y, int z,
                                        bool near) {
  using St = Store<S>;
  const int nx = g.nx, ny = g.ny;
  const I self = ((I)z * ny + y) * nx + x;
  const I Vp = (I)g.Vp;
  uint32_t bb = 0u;  // link mask; constant zero away from solid nodes
  if (near) {
    bb = __ldg(&g.lmask[self]);
    if (bb & 1u) return;  // solid node
  }
  float h[kQ];
  if (!ODD) {
#pragma unroll
    for (int p = 0; p < kQ; ++p) h[p] = St::load_plain(buf + (I)p * Vp + self);
    collide19<FORCING, FLUCT>(h, ph, (uint32_t)self);
    // The store addresses are the load addresses permuted; hiding the base
    // behind an empty asm makes the compiler recompute them after the
    // collision instead of keeping 19 of them live across it (which spills).
    typename Store<S>::T *out = buf + self;
    asm volatile("" : "+l"(out));
#pragma unroll
    for (int p = 0; p < kQ; ++p) St::store(out + (I)opp(p) * Vp, h[p]);
    return;
  }
  const int xm = wrap_m1(x, nx), xp = wrap_p1(x, nx);
  const int ym = wrap_m1(y, ny), yp = wrap_p1(y, ny);
  const int zm = wrap_m1(z, g.nz), zp = wrap_p1(z, g.nz);
#pragma unroll
  for (int p = 0; p < kQ; ++p) {
    // source node x - c_p
    const int sx = cx(p) == 1 ? xm : (cx(p) == -1 ? xp : x);
    const int sy = cy(p) == 1 ? ym : (cy(p) == -1 ? yp : y);
    const int sz = cz(p) == 1 ? zm : (cz(p) == -1 ? zp : z);
    const I sidx = (I)opp(p) * Vp + ((I)sz * ny + sy) * nx + sx;
    const I bidx = (I)p * Vp + self;
    h[p] = St::load_plain(buf + (((bb >> p) & 1u) ? bidx : sidx));
  }
  collide19<FORCING, FLUCT>(h, ph, (uint32_t)self);
  // As in the even step: the store offsets equal the load offsets of the
  // opposite directions, so the coordinates are hidden behind an empty asm
  // and the offsets recomputed rather than kept live across the collision.
  typename Store<S>::T *out = buf;
  int ox = x, oy = y, oz = z;
  asm volatile("" : "+l"(out), "+r"(ox), "+r"(oy), "+r"(oz));
  const int oxm = wrap_m1(ox, nx), oxp = wrap_p1(ox, nx);
  const int oym = wrap_m1(oy, ny), oyp = wrap_p1(oy, ny);
  const int ozm = wrap_m1(oz, g.nz), ozp = wrap_p1(oz, g.nz);
  const I oself = ((I)oz * ny + oy) * nx + ox;
#pragma unroll
  for (int p = 0; p < kQ; ++p) {
    // destination node x + c_p; bit opp(p) of the mask: x + c_p is solid
    const int tx = cx(p) == 1 ? oxp : (cx(p) == -1 ? oxm : ox);
    const int ty = cy(p) == 1 ? oyp : (cy(p) == -1 ? oym : oy);
    const int tz = cz(p) == 1 ? ozp : (cz(p) == -1 ? ozm : oz);
    const I didx = (I)p * Vp + ((I)tz * ny + ty) * nx + tx;
    const I bidx = (I)opp(p) * Vp + oself;
    St::store(out + (((bb >> opp(p)) & 1u) ? bidx : didx), h[p]);
  }
}

// One thread per node, a warp per 32 consecutive x of a row, as the pull
// kernel; without the thermal source six 256-thread blocks per SM for the
// even step and five for the odd step (whose shifted stores need more
// registers: at six it spills, and runs 1.7 % slower on a 256^3 solvent).
template <int S, int FORCING, typename I, bool ODD, bool FLUCT>
__global__ void __launch_bounds__(32 * kRowsPerBlock, FLUCT ? 1 : (ODD ? 5 : 6))
    k_aa_stream_collide(LbGeom g, LbPhys ph, typename Store<S>::T *buf, DevStatus *bump) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = blockIdx.z;
  if (bump != nullptr && x == 0 && y == 0 && z == 0) bump->step += 1;
  if (x >= g.nx || y >= g.ny) return;
  aa_node<S, FORCING, I, ODD, FLUCT>(g, ph, buf, x, y, z, tile_is_near(g, x, y, z));
}

template <int S, typename I, bool FLUCT>
cudaError_t aa_launch(const LbGeom &g, const LbPhys &ph, void *buf, int odd, DevStatus *bump,
                      cudaStream_t s) {
  using T = typename Store<S>::T;
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, g.nz);
  T *b = (T *)buf;
  const bool none = ph.g[0] == 0.f && ph.g[1] == 0.f && ph.g[2] == 0.f;
  if (odd) {
    if (none)
      k_aa_stream_collide<S, kForcingNone, I, true, FLUCT><<<grid, block, 0, s>>>(g, ph, b, bump);
    else if (ph.forcing == LBMD_FORCING_GUO)
      k_aa_stream_collide<S, LBMD_FORCING_GUO, I, true, FLUCT><<<grid, block, 0, s>>>(g, ph, b, bump);
    else
      k_aa_stream_collide<S, LBMD_FORCING_PAPER, I, true, FLUCT><<<grid, block, 0, s>>>(g, ph, b, bump);
  } else {
    if (none)
      k_aa_stream_collide<S, kForcingNone, I, false, FLUCT><<<grid, block, 0, s>>>(g, ph, b, bump);
    else if (ph.forcing == LBMD_FORCING_GUO)
      k_aa_stream_collide<S, LBMD_FORCING_GUO, I, false, FLUCT><<<grid, block, 0, s>>>(g, ph, b, bump);
    else
      k_aa_stream_collide<S, LBMD_FORCING_PAPER, I, false, FLUCT><<<grid, block, 0, s>>>(g, ph, b, bump);
  }
  return cudaGetLastError();
}

template <bool FLUCT>
cudaError_t aa_launch_storage(int storage, const LbGeom &g, const LbPhys &ph, void *buf, int odd,
                              DevStatus *bump, cudaStream_t s) {
  // 32-bit offsets when every population index fits
  const bool small = (long long)kQ * g.Vp < 0x7fffffffLL;
  switch (storage) {
    case LBMD_STORE_F32:
      return small ? aa_launch<LBMD_STORE_F32, int, FLUCT>(g, ph, buf, odd, bump, s)
                   : aa_launch<LBMD_STORE_F32, size_t, FLUCT>(g, ph, buf, odd, bump, s);
    case LBMD_STORE_F16:
      return small ? aa_launch<LBMD_STORE_F16, int, FLUCT>(g, ph, buf, odd, bump, s)
                   : aa_launch<LBMD_STORE_F16, size_t, FLUCT>(g, ph, buf, odd, bump, s);
    case LBMD_STORE_BF16:
      return small ? aa_launch<LBMD_STORE_BF16, int, FLUCT>(g, ph, buf, odd, bump, s)
                   : aa_launch<LBMD_STORE_BF16, size_t, FLUCT>(g, ph, buf, odd, bump, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbmd
