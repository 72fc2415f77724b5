// lb_collide.cuh -- the D3Q19 collision of Eq. 5 (BGK relaxation to the Eq. 6
// equilibrium, body-force source, optional thermal source F_p) and the update
// of one node (pull streaming + collision + store), shared by the
// stream-collide kernels.
#pragma once

#include "lb_pull.cuh"

namespace lbmd {

constexpr int kRowsPerBlock = 8;  // block = 32 x 8 threads

// Weight-orthogonal D3Q19 mode basis, row k at velocity c_p:
// 0: 1; 1-3: c_x, c_y, c_z; 4: c^2 - 1; 5: 3c_x^2 - c^2; 6: c_y^2 - c_z^2;
// 7-9: c_x c_y, c_y c_z, c_z c_x; 10-12: (3c^2 - 5) c_x, c_y, c_z;
// 13: (c_y^2 - c_z^2) c_x; 14: (c_z^2 - c_x^2) c_y; 15: (c_x^2 - c_y^2) c_z;
// 16: 3c^4 - 6c^2 + 1; 17: (2c^2 - 3)(3c_x^2 - c^2); 18: (2c^2 - 3)(c_y^2 - c_z^2).
__host__ __device__ constexpr int mode_row(int k, int p) {
  const int x = cx(p), y = cy(p), z = cz(p), c2 = x * x + y * y + z * z;
  return k == 0 ? 1 : k == 1 ? x : k == 2 ? y : k == 3 ? z
       : k == 4 ? c2 - 1 : k == 5 ? 3 * x * x - c2 : k == 6 ? y * y - z * z
       : k == 7 ? x * y : k == 8 ? y * z : k == 9 ? z * x
       : k == 10 ? (3 * c2 - 5) * x : k == 11 ? (3 * c2 - 5) * y : k == 12 ? (3 * c2 - 5) * z
       : k == 13 ? (y * y - z * z) * x : k == 14 ? (z * z - x * x) * y
       : k == 15 ? (x * x - y * y) * z : k == 16 ? 3 * c2 * c2 - 6 * c2 + 1
       : k == 17 ? (2 * c2 - 3) * (3 * x * x - c2) : (2 * c2 - 3) * (y * y - z * z);
}

// Thermal source F_p of Eq. 5 (fluctuating LB, Adhikari et al. 2005, in the
// mode form of Duenweg, Schiller and Ladd 2007) at node `node`, density rho:
//   xi_p = w_p sum_{k=4}^{18} e_kp a_k sqrt(rho) r_k,
//   a_k = sqrt((kT / c_s^2) (1 - (1 - omega)^2) / b_k)   (ph.fl_amp[k - 4]),
// with fifteen standard normals r_k from Box-Muller on four Philox blocks,
// counter (node, step lo, step hi, block | 2 << 8), key (seed lo, seed hi).
// The noise touches only non-conserved modes: mass and momentum are exact.
__device__ __forceinline__ void thermal_source(const LbPhys &ph, uint32_t node, float rho,
                                               float xi[kQ]) {
  const long long step = *ph.step;
  float r[16];
#pragma unroll
  for (uint32_t j = 0; j < 4; ++j) {
    const U4 c{node, (uint32_t)(unsigned long long)step, (uint32_t)((unsigned long long)step >> 32),
               j | (2u << 8)};
    const U4 x = philox4x32_10(c, (uint32_t)ph.seed, (uint32_t)(ph.seed >> 32));
    const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float rad = sqrtf(-2.0f * logf(uniform23(xs[2 * h])));
      float sn, cs;
      sincospif(2.0f * uniform23(xs[2 * h + 1]), &sn, &cs);
      r[4 * j + 2 * h] = rad * cs;
      r[4 * j + 2 * h + 1] = rad * sn;
    }
  }
  const float sr = sqrtf(rho);
  float t[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) t[k] = ph.fl_amp[k] * sr * r[k];
#pragma unroll
  for (int p = 0; p < kQ; ++p) {
    float acc = 0.f;
#pragma unroll
    for (int k = 4; k < kQ; ++k)
      if (mode_row(k, p) != 0) acc = fmaf((float)mode_row(k, p), t[k - 4], acc);
    xi[p] = wq(p) * acc;
  }
}

// Arithmetic of the collision, on one node (Ops1: float) or on two nodes at
// once (Ops2: float2, the paired FP32 instructions of sm_100 and later).  A
// paired operation is two independent correctly rounded operations, so both
// give the same bits for the same node.  Every operation is written out with
// its rounding (no contraction left to the compiler), so every stream-collide
// kernel -- pull, in-place, ensemble, one or two nodes per thread -- rounds
// identically.
struct Ops1 {
  using V = float;
  static __device__ __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __fadd_rn(a, -b); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ V neg(V a) { return -a; }
  static __device__ __forceinline__ V splat(float s) { return s; }
  static __device__ __forceinline__ V rcp(V a) { return __frcp_rn(a); }  // as 1.0f / a
  static __device__ __forceinline__ bool finite(V a) { return isfinite(a); }
};
struct Ops2 {
  using V = float2;
  static __device__ __forceinline__ V neg(V a) { return make_float2(-a.x, -a.y); }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __fadd2_rn(a, neg(b)); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ V splat(float s) { return make_float2(s, s); }
  static __device__ __forceinline__ V rcp(V a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }
  static __device__ __forceinline__ bool finite(V a) { return isfinite(a.x) && isfinite(a.y); }
};

// rho - rho0 and j = sum_p h_p c_p, each a sum in the population order, the
// momentum components as signed sums (no products with c_p).
template <class O>
__device__ __forceinline__ void moments_t(const typename O::V h[kQ], typename O::V &drho,
                                          typename O::V &jx, typename O::V &jy, typename O::V &jz) {
  drho = h[0];
  jx = h[1];
  jy = h[3];
  jz = h[5];
#pragma unroll
  for (int p = 1; p < kQ; ++p) {
    drho = O::add(drho, h[p]);
    if (p != 1 && cx(p) != 0) jx = cx(p) > 0 ? O::add(jx, h[p]) : O::sub(jx, h[p]);
    if (p != 3 && cy(p) != 0) jy = cy(p) > 0 ? O::add(jy, h[p]) : O::sub(jy, h[p]);
    if (p != 5 && cz(p) != 0) jz = cz(p) > 0 ? O::add(jz, h[p]) : O::sub(jz, h[p]);
  }
}

// c_p . u for odd p (the first nonzero component of c_p is +1) as a signed sum.
template <class O>
__device__ __forceinline__ typename O::V cdotu_t(int p, typename O::V ux, typename O::V uy,
                                                 typename O::V uz) {
  typename O::V r = cx(p) != 0 ? ux : (cy(p) != 0 ? uy : uz);
  if (cx(p) != 0 && cy(p) != 0) r = cy(p) > 0 ? O::add(r, uy) : O::sub(r, uy);
  if ((cx(p) != 0 || cy(p) != 0) && cz(p) != 0) r = cz(p) > 0 ? O::add(r, uz) : O::sub(r, uz);
  return r;
}

// Post-collision deviation of every population of one node (or two, Ops2)
// from its pre-collision deviations (Eq. 5, omega = 1/tau, Delta t = 1):
//   h*_p = (1 - omega) h_p + omega heq_p + S_p,
//   heq_p = w_p [ (rho - rho0) + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u) ]   (Eq. 6),
//   paper forcing: S_p = 3 w_p c_p . g;
//   Guo forcing:   u = (j + g/2)/rho, S_p = (1 - omega/2) w_p [3 (c - u) + 9 (c.u) c] . g;
//   kForcingNone (g = 0): u = j/rho, S_p = 0;
//   FLUCT (Ops1 only): plus the thermal source F_p of Eq. 5 (thermal_source).
// Opposite directions p, opp(p) = p + 1 (odd p) share c.u up to the sign, so
// heq splits into the even part w_p [(rho - rho0) - 3/2 rho u.u + 9/2 rho (c.u)^2]
// and the odd part +-3 w_p rho c.u, computed once per pair.  A node whose
// density is not finite (a population is not) sets *ph.nonfinite.
template <class O, int FORCING, bool FLUCT = false>
__device__ __forceinline__ void collide_t(typename O::V h[kQ], const LbPhys &ph, uint32_t node = 0) {
  using V = typename O::V;
  static_assert(!FLUCT || sizeof(V) == sizeof(float), "thermal source: one node per call");
  V drho, jx, jy, jz;
  moments_t<O>(h, drho, jx, jy, jz);
  const V rho = O::add(O::splat(ph.rho0), drho);
  // one compare and a predicated store per node
  if (!O::finite(rho)) *ph.nonfinite = 1;
  const V inv = O::rcp(rho);
  V ux, uy, uz;
  if (FORCING == LBMD_FORCING_GUO) {
    ux = O::mul(O::fma(O::splat(0.5f), O::splat(ph.g[0]), jx), inv);
    uy = O::mul(O::fma(O::splat(0.5f), O::splat(ph.g[1]), jy), inv);
    uz = O::mul(O::fma(O::splat(0.5f), O::splat(ph.g[2]), jz), inv);
  } else {
    ux = O::mul(jx, inv);
    uy = O::mul(jy, inv);
    uz = O::mul(jz, inv);
  }
  const float om = ph.omega, om1 = 1.0f - om;
  const V vom1 = O::splat(om1);
  const V usq = O::fma(uz, uz, O::fma(uy, uy, O::mul(ux, ux)));
  const V A = O::fma(O::neg(O::mul(O::splat(1.5f), rho)), usq, drho);
  const V r3 = O::mul(O::splat(3.0f), rho), r45 = O::mul(O::splat(4.5f), rho);
  V gu = O::splat(0.f);
  if (FORCING == LBMD_FORCING_GUO)
    gu = O::fma(O::splat(ph.g[2]), uz, O::fma(O::splat(ph.g[1]), uy, O::mul(O::splat(ph.g[0]), ux)));
  const float kguo = fmaf(-0.5f, om, 1.0f);
  // h*_p from the relaxed part, plus the source S_p (c_p . u = cu)
  auto add_source = [&](int p, V cu, V v) -> V {
    const float cg = cx(p) * ph.g[0] + cy(p) * ph.g[1] + cz(p) * ph.g[2];  // one value per kernel
    if (FORCING == LBMD_FORCING_GUO) {
      const V t = O::fma(O::mul(O::splat(9.0f), cu), O::splat(cg),
                         O::mul(O::splat(3.0f), O::sub(O::splat(cg), gu)));
      return O::add(v, O::mul(O::splat(__fmul_rn(kguo, wq(p))), t));
    }
    if (FORCING == LBMD_FORCING_PAPER) return O::add(v, O::splat(__fmul_rn(3.0f * wq(p), cg)));
    return v;
  };
  float xi[kQ];
  if constexpr (FLUCT) thermal_source(ph, node, rho, xi);
  h[0] = add_source(0, O::splat(0.f), O::fma(O::splat(__fmul_rn(om, wq(0))), A, O::mul(vom1, h[0])));
  if constexpr (FLUCT) h[0] = O::add(h[0], xi[0]);
#pragma unroll
  for (int p = 1; p < kQ; p += 2) {
    const V cu = cdotu_t<O>(p, ux, uy, uz);  // c_opp(p) . u = -cu
    const V even = O::fma(O::mul(r45, cu), cu, A);
    const V ow = O::splat(__fmul_rn(om, wq(p)));
    h[p] = add_source(p, cu, O::fma(ow, O::fma(r3, cu, even), O::mul(vom1, h[p])));
    h[p + 1] = add_source(p + 1, O::neg(cu), O::fma(ow, O::fma(O::neg(r3), cu, even), O::mul(vom1, h[p + 1])));
    if constexpr (FLUCT) {
      h[p] = O::add(h[p], xi[p]);
      h[p + 1] = O::add(h[p + 1], xi[p + 1]);
    }
  }
}

template <int FORCING, bool FLUCT = false>
__device__ __forceinline__ void collide19(float h[kQ], const LbPhys &ph, uint32_t node = 0) {
  collide_t<Ops1, FORCING, FLUCT>(h, ph, node);
}

// Stream and collide node (x, y, z) of one box: pull, Eq. 5 collision, store.
// near: take the bounce-back checks (required if a solid node is within one
// node of (x, y, z); allowed everywhere).
template <int S, int FORCING, typename I, bool FLUCT = false>
__device__ __forceinline__ void stream_collide_node(const LbGeom &g, const LbPhys &ph,
                                                    const typename Store<S>::T *__restrict__ src,
                                                    typename Store<S>::T *__restrict__ dst, int x,
                                                    int y, int z, bool near) {
  using St = Store<S>;
  const I self = ((I)z * g.ny + y) * g.nx + x;
  float h[kQ];
  if (near) {
    const uint32_t bb = __ldg(&g.lmask[self]);
    if (bb & 1u) return;  // solid node
    pull19_mask<S, I>(g, src, x, y, z, bb, h);
  } else {
    pull19_mask<S, I>(g, src, x, y, z, 0u, h);  // constant mask: no selects
  }
  collide19<FORCING, FLUCT>(h, ph, (uint32_t)self);
  const I Vp = (I)g.Vp;
#pragma unroll
  for (int p = 0; p < kQ; ++p) St::store(dst + (I)p * Vp + self, h[p]);
}


// Nodes (x, y, z) and (x, y, z + 1) of one box (z + 1 < nz), with all 38
// loads issued before either collision.  near: take the bounce-back checks
// for both.
template <int S, int FORCING>
__device__ __forceinline__ void stream_collide_node2(const LbGeom &g, const LbPhys &ph,
                                                     const typename Store<S>::T *__restrict__ src,
                                                     typename Store<S>::T *__restrict__ dst, int x,
                                                     int y, int z, bool near) {
  using St = Store<S>;
  const int self_a = (z * g.ny + y) * g.nx + x, self_b = self_a + g.nx * g.ny;
  float ha[kQ], hb[kQ];
  uint32_t ma = 0u, mb = 0u;
  if (near) {
    ma = __ldg(&g.lmask[self_a]);
    mb = __ldg(&g.lmask[self_b]);
    pull19_mask<S, int>(g, src, x, y, z, ma, ha);
    pull19_mask<S, int>(g, src, x, y, z + 1, mb, hb);
  } else {
    pull19_mask<S, int>(g, src, x, y, z, 0u, ha);  // constant masks: no selects
    pull19_mask<S, int>(g, src, x, y, z + 1, 0u, hb);
  }
  const int Vp = (int)g.Vp;
  if (!(ma & 1u)) {  // a solid node is pulled but not written
    collide19<FORCING>(ha, ph);
#pragma unroll
    for (int p = 0; p < kQ; ++p) St::store(dst + p * Vp + self_a, ha[p]);
  }
  if (!(mb & 1u)) {
    collide19<FORCING>(hb, ph);
#pragma unroll
    for (int p = 0; p < kQ; ++p) St::store(dst + p * Vp + self_b, hb[p]);
  }
}

// 16-bit storage, two x-adjacent nodes (2 xw, 2 xw + 1) of one box per
// call: their deviations of one population share a 32-bit word (nx even, so
// a pair never straddles a row).  Every population is one 32-bit load for
// c_x = 0 and two for c_x = +-1 (the neighbouring word supplies the shifted
// half; one byte permute assembles the pair), one 32-bit store, and the
// collision runs once for both nodes on float2 with the paired FP32
// instructions -- the same bits as stream_collide_node for either node.
// near: take the bounce-back checks (required if a solid node is within one
// node of the pair; allowed everywhere).  Word offsets are 32-bit
// (19 Vp < 2^31).
template <typename T2> struct Pair16;
template <> struct Pair16<__half2> {
  static __device__ __forceinline__ float2 unpack(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
  }
  static __device__ __forceinline__ uint32_t pack(float2 v) {
    const __half2 h = __float22half2_rn(v);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
};
template <> struct Pair16<__nv_bfloat162> {
  static __device__ __forceinline__ float2 unpack(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
  }
  static __device__ __forceinline__ uint32_t pack(float2 v) {
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
};

template <typename T2, int FORCING>
__device__ __forceinline__ void pair_node(const LbGeom &g, const LbPhys &ph,
                                          const uint32_t *__restrict__ src,
                                          uint32_t *__restrict__ dst, int xw, int y, int z,
                                          bool near) {
  using P = Pair16<T2>;
  const int wpr = g.nx >> 1;  // words per row
  const int Vw = (int)(g.Vp >> 1);
  const int ny = g.ny;
  const int self = (z * ny + y) * wpr + xw;
  // link masks of the two nodes (bit 0: solid; bit p: the pull source is solid)
  uint2 bb = make_uint2(0u, 0u);
  if (near) bb = __ldg(reinterpret_cast<const uint2 *>(g.lmask) + self);
  if ((bb.x & bb.y) & 1u) return;  // both solid: nothing to write
  const int ym = wrap_m1(y, ny), yp = wrap_p1(y, ny);
  const int zm = wrap_m1(z, g.nz), zp = wrap_p1(z, g.nz);
  const int xl = xw == 0 ? wpr - 1 : xw - 1, xr = xw == wpr - 1 ? 0 : xw + 1;
  float2 h[kQ];
#pragma unroll
  for (int p = 0; p < kQ; ++p) {
    // source row of x - c_p; the pair's sources are x - c_x, x - c_x + 1
    const int sy = cy(p) == 1 ? ym : (cy(p) == -1 ? yp : y);
    const int sz = cz(p) == 1 ? zm : (cz(p) == -1 ? zp : z);
    const uint32_t *rowp = src + p * Vw + (sz * ny + sy) * wpr;
    const uint32_t w0 = __ldg(rowp + xw);
    uint32_t w = w0;
    if (cx(p) == 1) w = __byte_perm(__ldg(rowp + xl), w0, 0x5432);   // (x - 1, x)
    if (cx(p) == -1) w = __byte_perm(w0, __ldg(rowp + xr), 0x5432);  // (x + 1, x + 2)
    h[p] = P::unpack(w);
  }
  if (near) {
    // halfway bounce-back: a population whose source is solid comes back as
    // the node's own post-collision opposite population
#pragma unroll
    for (int p = 1; p < kQ; ++p) {
      const bool ba = (bb.x >> p) & 1u, bbb = (bb.y >> p) & 1u;
      if (ba || bbb) {
        const float2 r = P::unpack(__ldg(src + opp(p) * Vw + self));
        if (ba) h[p].x = r.x;
        if (bbb) h[p].y = r.y;
      }
    }
    // a solid node of the pair: harmless inputs, and zero written back
    if (bb.x & 1u)
#pragma unroll
      for (int p = 0; p < kQ; ++p) h[p].x = 0.f;
    if (bb.y & 1u)
#pragma unroll
      for (int p = 0; p < kQ; ++p) h[p].y = 0.f;
  }
  collide_t<Ops2, FORCING>(h, ph);
  if (near) {
    if (bb.x & 1u)
#pragma unroll
      for (int p = 0; p < kQ; ++p) h[p].x = 0.f;
    if (bb.y & 1u)
#pragma unroll
      for (int p = 0; p < kQ; ++p) h[p].y = 0.f;
  }
#pragma unroll
  for (int p = 0; p < kQ; ++p) dst[p * Vw + self] = P::pack(h[p]);
}

}  // namespace lbmd
