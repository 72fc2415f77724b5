// md_kernels.cu -- bead <-> fluid coupling and the constrained polymer MD cycle
// (arXiv:0710.1272, Sec. II: Eqs. 1-4, 10, the four-stage LB step; Sec. III:
// pulling force, wall, translocation bookkeeping).
//
// k_gather computes, for every (bead, corner) pair, the transfer weight and
// the fluid velocity of the pulled pre-collision populations, and sums them
// per bead (trilinear over the fluid corners, or nearest grid point).
// k_md_cycle then runs one thread block per chain, one thread per bead, and
// M substeps of
//     F = F_WCA + F_bend + F_wall + F_drive - m gamma (v - u_i) + F_r,
//     v += dt F / m,  r~ = r + dt v,
//     SHAKE: Newton on the N-1 bond multipliers, the tridiagonal Jacobian
//            solved by parallel cyclic reduction in shared memory,
//     v = (r' - r) / dt,  r = r',
//     RATTLE: one tridiagonal solve removes the bond-parallel relative
//             velocities,
//     J_i += dt (F_drag + F_r);
//   then the translocation bookkeeping.  The spread hands -J_i to the fluid
//   with the gather weights (Eq. 10 with the reaction sign): the gather claims
//   each transfer node for its smallest (bead, corner) entry, the impulses are
//   summed at that owner in 64-bit fixed point, and the owner adds the source
//   to the node's post-collision populations once -- so a step gives the same
//   bits whatever order the atomics take.
#include "lb_pull.cuh"

namespace lbmd {

constexpr float kTwoSixth = 1.122462048309373f;  // 2^(1/6)
constexpr float kSkin = 0.8f;  // neighbour-list skin: lists hold pairs within r_c + skin

struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 f3(float4 v) { return F3{v.x, v.y, v.z}; }
__device__ __forceinline__ float4 f4(F3 v) { return make_float4(v.x, v.y, v.z, 0.f); }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return F3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return F3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return F3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Threads of the MD block: one per bead, rounded up to a warp.
int md_threads(int N) { return (N + 31) / 32 * 32; }

// Shared memory of the MD block: positions (hi, lo), displacements, bond
// vectors, velocities, the tridiagonal work arrays, the pair lists and, for
// chains of up to 512 beads, up to 32 solid nodes of each bead's wall list as
// integer coordinates of the chain's local frame (longer wall lists are read
// from the workspace).
constexpr int kWallShared = 32;
constexpr int kWallSharedMaxN = 512;

// Bytes before the shared wall lists, rounded up to 16 (the short4 entries
// need 8-byte alignment; 180 N bytes is not a multiple of 8 for odd N).
__host__ __device__ inline size_t md_smem_head(int N) {
  const size_t head = (size_t)N * (5 * sizeof(float4) + sizeof(float) + kMaxPairs * sizeof(short));
  return (head + 15) / 16 * 16;
}

size_t md_smem_bytes(int N) {
  const size_t walls = N <= kWallSharedMaxN ? (size_t)N * kWallShared * sizeof(short4) : 0;
  return md_smem_head(N) + walls;
}

// Double-float helpers: a coordinate is hi + lo with |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float d) {
  const float s = hi + d;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (d - bp);
  const float l = lo + e;
  hi = s + l;
  lo = l - (hi - s);
}
__device__ __forceinline__ F3 diff_hl(float4 ah, float4 al, float4 bh, float4 bl) {
  return F3{(ah.x - bh.x) + (al.x - bl.x), (ah.y - bh.y) + (al.y - bl.y),
            (ah.z - bh.z) + (al.z - bl.z)};
}
// Index into [0, n): one add or subtract for indices within a period of the
// box (the common case), the integer remainder otherwise.
__device__ __forceinline__ int wrap_near(int a, int n) {
  if (a < 0) a += n;
  if (a >= n) a -= n;
  if ((unsigned)a >= (unsigned)n) a = wrapi(a, n);
  return a;
}

// Wrapped node index and fraction of global = origin + hi + lo.
__device__ __forceinline__ void cell_frac_hl(float hi, float lo, int origin, int n, int &cell,
                                             float &frac) {
  const float fl = floorf(hi);
  frac = (hi - fl) + lo;
  cell = wrap_near(origin + (int)fl, n);
}

// 2x2 matrices for the interface system of the tridiagonal solve.
struct M2 {
  float a, b, c, d;  // [[a, b], [c, d]]
};
__device__ __forceinline__ M2 mmul(M2 x, M2 y) {
  return M2{x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c,
            x.c * y.b + x.d * y.d};
}
__device__ __forceinline__ M2 madd(M2 x, M2 y) { return M2{x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }

// Hardware reciprocal approximation (relative error ~2^-23) for the
// tridiagonal solves: they are latency-bound chains, and a correctly rounded
// reciprocal costs several dependent instructions.
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ M2 minv(M2 x) {
  const float r = rcp_fast(x.a * x.d - x.b * x.c);
  return M2{x.d * r, -x.b * r, -x.c * r, x.a * r};
}
__device__ __forceinline__ M2 mshfl_up(M2 x, int s) {
  return M2{__shfl_up_sync(0xffffffffu, x.a, s), __shfl_up_sync(0xffffffffu, x.b, s),
            __shfl_up_sync(0xffffffffu, x.c, s), __shfl_up_sync(0xffffffffu, x.d, s)};
}
__device__ __forceinline__ M2 mshfl_down(M2 x, int s) {
  return M2{__shfl_down_sync(0xffffffffu, x.a, s), __shfl_down_sync(0xffffffffu, x.b, s),
            __shfl_down_sync(0xffffffffu, x.c, s), __shfl_down_sync(0xffffffffu, x.d, s)};
}

// Tridiagonal solve over rows 0..n-1 of the block (row i held by thread i:
// a x_{i-1} + b x_i + c x_{i+1} = d, with a_0 = c_{n-1} = 0).  Every thread
// of the block calls it; returns x_i and, in x_prev, x_{i-1}.
//
// SPIKE-type partition by warps: each warp reduces its 32 rows by cyclic
// reduction over lane shuffles, for the right-hand side and for the two
// coupling columns to the neighbouring warps (the "spikes" v and w), giving
// x_i = y_i - v_i x_last(prev warp) - w_i x_first(next warp).  The first and
// last unknowns of neighbouring warps form a block tridiagonal system with
// 2x2 blocks, one block row per warp boundary, which warp 0 solves by block
// cyclic reduction.  Two block barriers, none when n <= 32.
__device__ float spike_tri_solve(int n, float a, float b, float c, float d, float &x_prev) {
  __shared__ float sh_y[6 * 32];  // per warp: y, v, w of its first and last row
  __shared__ float sh_x[64];      // x of the last row [0, 32) and first row [32, 64) per warp
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nch = (n + 31) >> 5;
  if (t >= n) {
    a = 0.f;
    b = 1.f;
    c = 0.f;
    d = 0.f;
  }
  float al = lane == 0 ? 0.f : a, be = b, ga = lane == 31 ? 0.f : c;
  float r0 = d, r1 = lane == 0 ? a : 0.f, r2 = lane == 31 ? c : 0.f;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const float am = __shfl_up_sync(0xffffffffu, al, s), bm = __shfl_up_sync(0xffffffffu, be, s);
    const float gm = __shfl_up_sync(0xffffffffu, ga, s);
    const float r0m = __shfl_up_sync(0xffffffffu, r0, s), r1m = __shfl_up_sync(0xffffffffu, r1, s);
    const float r2m = __shfl_up_sync(0xffffffffu, r2, s);
    const float ap = __shfl_down_sync(0xffffffffu, al, s), bp = __shfl_down_sync(0xffffffffu, be, s);
    const float gp = __shfl_down_sync(0xffffffffu, ga, s);
    const float r0p = __shfl_down_sync(0xffffffffu, r0, s), r1p = __shfl_down_sync(0xffffffffu, r1, s);
    const float r2p = __shfl_down_sync(0xffffffffu, r2, s);
    const bool hm = lane >= s, hp = lane + s < 32;
    const float k1 = hm ? al * rcp_fast(bm) : 0.f;
    const float k2 = hp ? ga * rcp_fast(bp) : 0.f;
    const float nal = hm ? -k1 * am : 0.f, nga = hp ? -k2 * gp : 0.f;
    be = be - k1 * gm - k2 * ap;
    r0 = r0 - k1 * r0m - k2 * r0p;
    r1 = r1 - k1 * r1m - k2 * r1p;
    r2 = r2 - k1 * r2m - k2 * r2p;
    al = nal;
    ga = nga;
  }
  const float ib = rcp_fast(be);
  const float y = r0 * ib, v = r1 * ib, sw = r2 * ib;
  if (nch > 1) {
    if (lane == 0 && w < nch) {
      sh_y[6 * w] = y;
      sh_y[6 * w + 1] = v;
      sh_y[6 * w + 2] = sw;
    }
    if (lane == 31 && w < nch) {
      sh_y[6 * w + 3] = y;
      sh_y[6 * w + 4] = v;
      sh_y[6 * w + 5] = sw;
    }
    __syncthreads();
    if (w == 0) {
      // block row k: unknowns (x_last(k), x_first(k+1)) at the boundary of
      // warps k and k+1; rows beyond nch-2 are identity rows
      M2 L{0.f, 0.f, 0.f, 0.f}, D{1.f, 0.f, 0.f, 1.f}, U{0.f, 0.f, 0.f, 0.f};
      float q0 = 0.f, q1 = 0.f;
      if (lane < nch - 1) {
        D.b = sh_y[6 * lane + 5];        // w of the last row of warp k
        D.c = sh_y[6 * (lane + 1) + 1];  // v of the first row of warp k+1
        L.a = sh_y[6 * lane + 4];        // v of the last row of warp k
        U.d = sh_y[6 * (lane + 1) + 2];  // w of the first row of warp k+1
        q0 = sh_y[6 * lane + 3];
        q1 = sh_y[6 * (lane + 1)];
      }
      // block cyclic reduction over the nch - 1 boundary rows; each lane
      // inverts its own diagonal block and the neighbours' inverses arrive by
      // shuffle
      for (int s = 1; s < nch - 1; s <<= 1) {
        const M2 Di = minv(D);
        const M2 Lm = mshfl_up(L, s), Dim = mshfl_up(Di, s), Um = mshfl_up(U, s);
        const float q0m = __shfl_up_sync(0xffffffffu, q0, s), q1m = __shfl_up_sync(0xffffffffu, q1, s);
        const M2 Lp = mshfl_down(L, s), Dip = mshfl_down(Di, s), Up = mshfl_down(U, s);
        const float q0p = __shfl_down_sync(0xffffffffu, q0, s), q1p = __shfl_down_sync(0xffffffffu, q1, s);
        M2 al2{0.f, 0.f, 0.f, 0.f}, ga2{0.f, 0.f, 0.f, 0.f};
        if (lane >= s) {
          const M2 t2 = mmul(L, Dim);
          al2 = M2{-t2.a, -t2.b, -t2.c, -t2.d};
        }
        if (lane + s < 32) {
          const M2 t2 = mmul(U, Dip);
          ga2 = M2{-t2.a, -t2.b, -t2.c, -t2.d};
        }
        const M2 nL = mmul(al2, Lm), nU = mmul(ga2, Up);
        D = madd(D, madd(mmul(al2, Um), mmul(ga2, Lp)));
        const float nq0 = q0 + al2.a * q0m + al2.b * q1m + ga2.a * q0p + ga2.b * q1p;
        const float nq1 = q1 + al2.c * q0m + al2.d * q1m + ga2.c * q0p + ga2.d * q1p;
        L = nL;
        U = nU;
        q0 = nq0;
        q1 = nq1;
      }
      const M2 Di = minv(D);
      if (lane < nch - 1) {
        sh_x[lane] = Di.a * q0 + Di.b * q1;           // x_last of warp k
        sh_x[32 + lane + 1] = Di.c * q0 + Di.d * q1;  // x_first of warp k+1
      }
    }
    __syncthreads();
  }
  float x = y;
  if (nch > 1) {
    if (w > 0 && w < nch) x -= v * sh_x[w - 1];
    if (w + 1 < nch) x -= sw * sh_x[32 + w + 1];
  }
  const float xu = __shfl_up_sync(0xffffffffu, x, 1);
  x_prev = lane > 0 ? xu : (w > 0 && w < nch && nch > 1 ? sh_x[w - 1] : 0.f);
  return x;
}

// Eq. 2 truncated at 2^(1/6) sigma: adds -dV/dd for separation d.
__device__ __forceinline__ void wca_add(F3 d, float sig2, float rc2, float eps24, F3 &F) {
  const float r2 = dot(d, d);
  if (r2 < rc2) {
    const float ir2 = 1.0f / r2;
    const float sr2 = sig2 * ir2;
    const float sr6 = sr2 * sr2 * sr2;
    const float f = eps24 * (2.0f * sr6 * sr6 - sr6) * ir2;
    F = F + f * d;
  }
}

// Eq. 3 bending at the angle of beads (a, b, c) given the two bond vectors
// b1 = r_b - r_a and b2 = r_c - r_b: the force on bead `which` (0 = a, 1 = b,
// 2 = c), F = -dV/dr with V = kappa phi^2 / 2.
__device__ __forceinline__ F3 bend_force(F3 b1, F3 b2, float kappa, int which) {
  const float l1 = sqrtf(dot(b1, b1)), l2 = sqrtf(dot(b2, b2));
  float cphi = dot(b1, b2) / (l1 * l2);
  cphi = fminf(1.f, fmaxf(-1.f, cphi));
  const float phi = acosf(cphi);
  const float A = phi < 1e-4f ? kappa : kappa * phi / sinf(phi);
  const F3 g1 = (1.0f / (l1 * l2)) * b2 - (cphi / (l1 * l1)) * b1;
  const F3 g2 = (1.0f / (l1 * l2)) * b1 - (cphi / (l2 * l2)) * b2;
  if (which == 0) return (-A) * g1;
  if (which == 1) return A * (g1 - g2);
  return A * g2;
}

// WCA pair forces on bead i from every other non-bonded bead (minimum image).
__device__ __forceinline__ F3 all_pair_forces(const ChainArgs &a, int i, float4 rh, float4 rl,
                                              const float4 *s_rh, const float4 *s_rl) {
  const LbGeom &g = a.geo;
  const float sig2 = a.sigma * a.sigma;
  const float rc = kTwoSixth * a.sigma, rc2 = rc * rc;
  const float eps24 = 24.0f * a.eps;
  const float Lx = (float)g.nx, Ly = (float)g.ny, Lz = (float)g.nz;
  const float iLx = 1.0f / Lx, iLy = 1.0f / Ly, iLz = 1.0f / Lz;
  F3 F{0.f, 0.f, 0.f};
  for (int j = 0; j < a.N; ++j) {
    const int dij = j - i;
    if (dij == 0 || (a.has_bonds && (dij == 1 || dij == -1))) continue;
    F3 d = diff_hl(rh, rl, s_rh[j], s_rl[j]);
    d.x -= Lx * rintf(d.x * iLx);
    d.y -= Ly * rintf(d.y * iLy);
    d.z -= Lz * rintf(d.z * iLz);
    wca_add(d, sig2, rc2, eps24, F);
  }
  return F;
}

// Sec. III pulling force on a bead at the local position rh + rl: -f_drive x
// inside the channel of the pore cross-section and the x-layers within 1.5
// nodes of the wall.
__device__ __forceinline__ F3 drive_force_at(const ChainArgs &a, float4 rh, float4 rl) {
  const LbGeom &g = a.geo;
  F3 F{0.f, 0.f, 0.f};
  if (a.has_wall && a.pore_d > 0 && a.fdrive != 0.f) {
    int c[3];
    float sf[3];
    cell_frac_hl(rh.x, rl.x, a.ox, g.nx, c[0], sf[0]);
    cell_frac_hl(rh.y, rl.y, a.oy, g.ny, c[1], sf[1]);
    cell_frac_hl(rh.z, rl.z, a.oz, g.nz, c[2], sf[2]);
    const int di = wrap_near(c[0] - a.wall_x + g.nx / 2, g.nx) - g.nx / 2;
    const float dx = (float)di + sf[0] - 0.5f * (float)(a.wall_t - 1);
    const float half = 0.5f * (float)(a.wall_t - 1) + 1.5f;
    const float ry = (float)c[1] + sf[1], rz = (float)c[2] + sf[2];
    if (fabsf(dx) <= half && ry >= a.pore_y0 - 0.5f && ry < a.pore_y0 + a.pore_d - 0.5f &&
        rz >= a.pore_z0 - 0.5f && rz < a.pore_z0 + a.pore_d - 0.5f)
      F.x -= a.fdrive;
  }
  return F;
}

// Bending (Eq. 3) and the Sec. III pulling force on bead i.
__device__ F3 bend_drive_forces(const ChainArgs &a, int i, const float4 *s_rh, const float4 *s_rl) {
  const int N = a.N;
  F3 F{0.f, 0.f, 0.f};
  if (a.kappa != 0.f && a.has_bonds) {
    // bond vectors b_{i-2}, b_{i-1}, b_i, b_{i+1} around bead i
    F3 bm2{0, 0, 0}, bm1{0, 0, 0}, b0{0, 0, 0}, bp1{0, 0, 0};
    if (i >= 2) bm2 = diff_hl(s_rh[i - 1], s_rl[i - 1], s_rh[i - 2], s_rl[i - 2]);
    if (i >= 1) bm1 = diff_hl(s_rh[i], s_rl[i], s_rh[i - 1], s_rl[i - 1]);
    if (i + 1 < N) b0 = diff_hl(s_rh[i + 1], s_rl[i + 1], s_rh[i], s_rl[i]);
    if (i + 2 < N) bp1 = diff_hl(s_rh[i + 2], s_rl[i + 2], s_rh[i + 1], s_rl[i + 1]);
    if (i >= 2) F = F + bend_force(bm2, bm1, a.kappa, 2);
    if (i >= 1 && i + 1 < N) F = F + bend_force(bm1, b0, a.kappa, 1);
    if (i + 2 < N) F = F + bend_force(b0, bp1, a.kappa, 0);
  }
  // pulling force inside the channel through the pore
  return F + drive_force_at(a, s_rh[i], s_rl[i]);
}

// Sum of K values over the block (every thread gets the sums).  red holds
// 32 K partials and K results; a result is rewritten only after every thread
// has passed the next call's first barrier, i.e. has read it.
template <int K>
__device__ __forceinline__ void block_sum(float (&v)[K], float *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int m = 16; m > 0; m >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], m);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float t = lane < nw ? red[lane * K + k] : 0.f;
      for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
      if (lane == 0) red[32 * K + k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = red[32 * K + k];
}

// Solid node test from the Sec. III geometry itself (the wall layers
// wall_x .. wall_x + wall_t - 1 minus the d x d pore, and the rows y = 0 and
// y = ny - 1 with y-walls): the rule the solid bitfield is built from, with
// no memory read.  Coordinates inside the box.
__device__ __forceinline__ bool wall_layer(const ChainArgs &a, int x) {
  int dx = x - a.wall_x;
  if (dx < 0) dx += a.geo.nx;
  return a.has_wall && dx < a.wall_t;
}
__device__ __forceinline__ bool solid_geom(const ChainArgs &a, int x, int y, int z) {
  if (a.y_walls && (y == 0 || y == a.geo.ny - 1)) return true;
  if (!wall_layer(a, x)) return false;
  return !(a.pore_d > 0 && y >= a.pore_y0 && y < a.pore_y0 + a.pore_d && z >= a.pore_z0 &&
           z < a.pore_z0 + a.pore_d);
}

// Solid nodes around a bead within `radius` (node offsets n with
// |n - s| < radius per axis), visited in x, y, z order.  For each solid node
// calls fn(node coordinate in the chain's local frame).
template <typename Fn>
__device__ __forceinline__ void for_solid_nodes(const ChainArgs &a, float4 rh, float4 rl,
                                                float radius, Fn fn) {
  const LbGeom &g = a.geo;
  if (!a.has_wall && !a.y_walls) return;
  int c[3];
  float sf[3];
  cell_frac_hl(rh.x, rl.x, a.ox, g.nx, c[0], sf[0]);
  cell_frac_hl(rh.y, rl.y, a.oy, g.ny, c[1], sf[1]);
  cell_frac_hl(rh.z, rl.z, a.oz, g.nz, c[2], sf[2]);
  const float fx = floorf(rh.x), fy = floorf(rh.y), fz = floorf(rh.z);
  const int lo0 = (int)ceilf(sf[0] - radius), hi0 = (int)floorf(sf[0] + radius);
  const int lo1 = (int)ceilf(sf[1] - radius), hi1 = (int)floorf(sf[1] + radius);
  const int lo2 = (int)ceilf(sf[2] - radius), hi2 = (int)floorf(sf[2] + radius);
  for (int ox = lo0; ox <= hi0; ++ox) {
    const int x = wrap_near(c[0] + ox, g.nx);
    if (!a.y_walls && !wall_layer(a, x)) continue;  // no solid node in this layer
    for (int oy = lo1; oy <= hi1; ++oy) {
      const int y = wrap_near(c[1] + oy, g.ny);
      for (int oz = lo2; oz <= hi2; ++oz) {
        const int z = wrap_near(c[2] + oz, g.nz);
        if (!solid_geom(a, x, y, z)) continue;
        fn(make_float4(fx + (float)ox, fy + (float)oy, fz + (float)oz, 0.f));
      }
    }
  }
}

// Eq. 2 between the bead and a solid node given in the local frame.
__device__ __forceinline__ void wall_add(float4 rh, float4 rl, float4 node, float sig2, float rc2,
                                         float eps24, F3 &F) {
  wca_add(F3{(rh.x - node.x) + rl.x, (rh.y - node.y) + rl.y, (rh.z - node.z) + rl.z}, sig2, rc2,
          eps24, F);
}

// Bead i's pair forces from its shared-memory list and wall forces from its
// solid-node list: the shared-memory copy SW (column i, entry q at SW[q N])
// when nws >= 0, else the workspace list.
__device__ __forceinline__ F3 list_forces(const ChainArgs &a, int i, float4 rh, float4 rl,
                                          const float4 *s_rh, const float4 *s_rl,
                                          const short *L, int np, const short4 *SW, int nws) {
  const LbGeom &g = a.geo;
  const float sig2 = a.sigma * a.sigma;
  const float rc = kTwoSixth * a.sigma, rc2 = rc * rc;
  const float eps24 = 24.0f * a.eps;
  const float Lx = (float)g.nx, Ly = (float)g.ny, Lz = (float)g.nz;
  const float iLx = 1.0f / Lx, iLy = 1.0f / Ly, iLz = 1.0f / Lz;
  F3 F{0.f, 0.f, 0.f};
  for (int q = 0; q < np; ++q) {
    const int j = L[q * a.N];
    F3 d = diff_hl(rh, rl, s_rh[j], s_rl[j]);
    d.x -= Lx * rintf(d.x * iLx);
    d.y -= Ly * rintf(d.y * iLy);
    d.z -= Lz * rintf(d.z * iLz);
    wca_add(d, sig2, rc2, eps24, F);
  }
  if (nws >= 0) {
#pragma unroll 4
    for (int q = 0; q < nws; ++q) {
      const short4 w = SW[q * a.N];
      wall_add(rh, rl, make_float4((float)w.x, (float)w.y, (float)w.z, 0.f), sig2, rc2, eps24, F);
    }
    return F;
  }
  const int nw = a.wl_cnt[i];
  const float4 *W = a.wl_list + (size_t)i * kMaxWall;
#pragma unroll 4
  for (int q = 0; q < nw; ++q) wall_add(rh, rl, W[q], sig2, rc2, eps24, F);
  return F;
}

// A wall node's local coordinates fit the shared-memory entry.
__device__ __forceinline__ bool fits_short(float4 n) {
  return fabsf(n.x) <= 32000.f && fabsf(n.y) <= 32000.f && fabsf(n.z) <= 32000.f;
}

// Rebuild bead i's lists with cutoff r_c + skin: pair list (shared memory,
// column i, entry q at L[q N]; copied to the workspace for the next launch)
// and solid-node list (workspace, and its shared copy SW when not null and
// it fits: *nws = its length, else -1).  Solid nodes are kept within the
// sphere of radius r_c + skin (a node beyond it exerts no force while the
// bead stays within half the skin of the build position).  Returns the pair
// count, or -1 on overflow.
__device__ int build_lists(const ChainArgs &a, int i, float4 rh, float4 rl, const float4 *s_rh,
                           const float4 *s_rl, short *L, short4 *SW, int *nws) {
  const LbGeom &g = a.geo;
  const int N = a.N;
  const float rlist = kTwoSixth * a.sigma + kSkin, rl2 = rlist * rlist;
  const float Lx = (float)g.nx, Ly = (float)g.ny, Lz = (float)g.nz;
  const float iLx = 1.0f / Lx, iLy = 1.0f / Ly, iLz = 1.0f / Lz;
  short *G = a.nl_list + (size_t)i * kMaxPairs;
  int np = 0;
  for (int j = 0; j < N; ++j) {
    const int dij = j - i;
    if (dij == 0 || (a.has_bonds && (dij == 1 || dij == -1))) continue;
    F3 d = diff_hl(rh, rl, s_rh[j], s_rl[j]);
    d.x -= Lx * rintf(d.x * iLx);
    d.y -= Ly * rintf(d.y * iLy);
    d.z -= Lz * rintf(d.z * iLz);
    if (dot(d, d) < rl2) {
      if (np < kMaxPairs) {
        L[np * N] = (short)j;
        G[np] = (short)j;
      }
      ++np;
    }
  }
  float4 *W = a.wl_list + (size_t)i * kMaxWall;
  int nw = 0;
  bool packed = SW != nullptr;
  for_solid_nodes(a, rh, rl, rlist, [&](float4 node) {
    const F3 d{(rh.x - node.x) + rl.x, (rh.y - node.y) + rl.y, (rh.z - node.z) + rl.z};
    if (!(dot(d, d) < rl2)) return;
    if (nw < kMaxWall) W[nw] = node;
    if (packed && nw < kWallShared && fits_short(node))
      SW[nw * N] = make_short4((short)node.x, (short)node.y, (short)node.z, 0);
    else
      packed = false;
    ++nw;
  });
  *nws = packed ? nw : -1;
  a.nl_cnt[i] = min(np, kMaxPairs);
  a.wl_cnt[i] = min(nw, kMaxWall);
  a.nl_ref[i] = rh;
  return (np <= kMaxPairs && nw <= kMaxWall) ? np : -1;
}

// Without lists (overflow): wall forces by scanning the stencil.
__device__ F3 wall_stencil_forces(const ChainArgs &a, float4 rh, float4 rl) {
  const float sig2 = a.sigma * a.sigma;
  const float rc = kTwoSixth * a.sigma, rc2 = rc * rc;
  const float eps24 = 24.0f * a.eps;
  F3 F{0.f, 0.f, 0.f};
  for_solid_nodes(a, rh, rl, rc, [&](float4 node) { wall_add(rh, rl, node, sig2, rc2, eps24, F); });
  return F;
}

// Fixed point of the spread: units of 2^-40.  The impulses of a node (|F| of
// order 1e-2) keep ~30 significant bits, far below a float ulp of the
// populations they reach.  The conversions are built from 32-bit ones: 64-bit
// integer <-> float conversions run at a small fraction of the FP32 rate on
// this GPU.
constexpr float kFixOne = 1099511627776.0f;  // 2^40

// round(v 2^40) for |v| < 2^10 as a 64-bit integer, rounded to nearest even
// like the direct conversion: with a = |v| 2^8 = hi + f (hi integral,
// 0 <= f <= 1 - 2^-24; a, hi and f exact in float), |v| 2^40 = hi 2^32 +
// f 2^32, only f 2^32 (< 2^32) needs rounding, and rounding to nearest even
// is symmetric in the sign.
__device__ __forceinline__ long long fix40(float v) {
  const float a = fabsf(v) * 256.0f;
  const float hi = floorf(a);
  const unsigned lo = __float2uint_rn((a - hi) * 4294967296.0f);
  const long long m = (long long)(((unsigned long long)__float2uint_rn(hi) << 32) | lo);
  return v < 0.f ? -m : m;
}

// q 2^-40 as a float: hi 2^-8 + lo 2^-40 with q = hi 2^32 + lo (0 <= lo <
// 2^32), the low word rounded to float first and the sum rounded once more.
__device__ __forceinline__ float unfix40(long long q) {
  const int hi = (int)(q >> 32);
  const unsigned lo = (unsigned)(unsigned long long)q;
  return __fmaf_rn((float)hi, 1.0f / 256.0f, __uint2float_rn(lo) * (1.0f / kFixOne));
}

// Adds entry e's share -w_e J_i of the impulse to the sum at the owner of its
// node (64-bit integer atomics: the result does not depend on their order).
// A share that is not finite, or too large for the fixed point (|F| >= 2^10:
// then even all 8 N <= 2^13 shares of a chain on one node stay below 2^63 in
// units of 2^-40), marks the sum instead, and the node receives NaN -- a
// stable step hands the fluid impulses of order 1e-2.
__device__ __forceinline__ void spread_add(const ChainArgs &a, int e, float4 j) {
  const int node = a.sp_node[e];
  if (node < 0) return;
  const float w = a.sp_w[e];
  const float fx = -w * j.x, fy = -w * j.y, fz = -w * j.z;
  SpreadAcc *q = a.acc + a.owner[node];
  const float lim = 1024.0f;  // 2^10
  if (!(fabsf(fx) < lim && fabsf(fy) < lim && fabsf(fz) < lim)) {
    atomicOr(reinterpret_cast<unsigned long long *>(&q->bad), 1ull);
    return;
  }
  atomicAdd(reinterpret_cast<unsigned long long *>(&q->x), (unsigned long long)fix40(fx));
  atomicAdd(reinterpret_cast<unsigned long long *>(&q->y), (unsigned long long)fix40(fy));
  atomicAdd(reinterpret_cast<unsigned long long *>(&q->z), (unsigned long long)fix40(fz));
}

// The owner's conversion: the summed force of node `node` (NaN if a
// contribution was not finite); the sum and the node's owner return to rest.
// The sum is read through L2 (it was written by atomics of an earlier kernel).
__device__ __forceinline__ F3 spread_take(const ChainArgs &a, int node, int e) {
  SpreadAcc *q = a.acc + e;
  const long long x = __ldcg(&q->x), y = __ldcg(&q->y), z = __ldcg(&q->z), bad = __ldcg(&q->bad);
  *q = SpreadAcc{0, 0, 0, 0};
  a.owner[node] = kOwnerFree;
  if (bad) {
    const float nan = __int_as_float(0x7fc00000);
    return F3{nan, nan, nan};
  }
  return F3{unfix40(x), unfix40(y), unfix40(z)};
}

// After every contribution is summed: entry e's record for the apply --
// (F, node) if e owns its node, node = -1 otherwise.
__device__ __forceinline__ void spread_finalize(const ChainArgs &a, int e) {
  const int node = a.sp_node[e];
  float4 out = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
  if (node >= 0 && a.owner[node] == e) {
    const F3 F = spread_take(a, node, e);
    out = make_float4(F.x, F.y, F.z, __int_as_float(node));
  }
  a.sp_src[e] = out;
}

// (2) the M MD substeps of one chain, one thread per bead, and (5) the
// bookkeeping; `a` may live in parameter or shared memory.
template <bool WS>
__device__ __forceinline__ void md_cycle_body(const ChainArgs &a) {
  extern __shared__ float4 smem4[];
  const int N = a.N;
  const int i = threadIdx.x;  // bead of this thread
  const bool bead = i < N;
  float4 *s_rh = smem4;       // positions, hi part (start of the substep)
  float4 *s_rl = s_rh + N;    // positions, lo part
  float4 *s_t = s_rl + N;     // displacement of the substep
  float4 *s_b = s_t + N;      // bond vectors
  float4 *s_v = s_b + N;      // velocities (RATTLE)
  float *s_lam = (float *)(s_v + N);  // N: SHAKE multipliers of the last substep
  short *s_nl = (short *)(s_lam + N);  // [kMaxPairs][N] pair lists, column per bead
  // [kWallShared][N] wall lists, column per bead (WS: chains of <= 512 beads)
  short4 *s_w = WS ? (short4 *)((char *)smem4 + md_smem_head(N)) : nullptr;
  int nws = -1;  // length of this bead's shared wall list, -1: read the workspace

  const long long step = a.status->step;
  int nl_ok = a.status->nl_ok && a.status->nl_builds > 0;
  float4 rh = make_float4(0, 0, 0, 0), rl = rh, ref = rh;
  F3 v{0.f, 0.f, 0.f}, ui{0.f, 0.f, 0.f};
  int np = 0;  // length of this bead's pair list
  if (bead) {
    rh = a.pos[i];
    rl = a.pos_lo[i];
    ref = a.nl_ref[i];
    v = f3(a.vel[i]);
    ui = f3(a.ui[i]);  // (1) interpolated by k_gather, frozen for the M substeps
    s_rh[i] = rh;
    s_rl[i] = rl;
    s_lam[i] = a.lam[i];
    if (nl_ok) {
      np = a.nl_cnt[i];
      const short *G = a.nl_list + (size_t)i * kMaxPairs;
      for (int q = 0; q < np; ++q) s_nl[q * N + i] = G[q];
      if (WS) {
        // this launch's substeps read the wall list from shared memory
        const int nw = a.wl_cnt[i];
        if (nw <= kWallShared) {
          const float4 *W = a.wl_list + (size_t)i * kMaxWall;
          bool fit = true;
#pragma unroll 4
          for (int q = 0; q < nw; ++q) {
            const float4 node = W[q];
            fit = fit && fits_short(node);
            s_w[q * N + i] = make_short4((short)node.x, (short)node.y, (short)node.z, 0);
          }
          nws = fit ? nw : -1;
        }
      }
    }
  }
  const float half_skin2 = 0.25f * kSkin * kSkin;
  auto moved = [&]() {
    const float dx = rh.x - ref.x, dy = rh.y - ref.y, dz = rh.z - ref.z;
    return !(dx * dx + dy * dy + dz * dz <= half_skin2);
  };
  int rebuild = __syncthreads_or(bead && (!nl_ok || moved()));
  F3 J{0.f, 0.f, 0.f};
  const float dt = a.dt, m = a.mass, im = 1.0f / a.mass, idt = 1.0f / a.dt;
  const float sig_r = sqrtf(2.0f * m * a.gamma * a.kT / dt);
  const double b0 = (bead && i < N - 1 && a.has_bonds) ? a.b0[i] : 1.0;
  const float tol = fmaxf(a.shake_tol, 5e-7f);
  int shake_bad = 0, newton_total = 0, builds = 0;

  for (int k = 0; k < a.M; ++k) {  // (2) M MD substeps
    if (rebuild && a.eps != 0.f) {
      // neighbour lists: pairs and solid nodes within r_c + skin
      int cnt = 0;
      if (bead) {
        cnt = build_lists(a, i, rh, rl, s_rh, s_rl, s_nl + i, WS ? s_w + i : nullptr, &nws);
        ref = rh;
      }
      nl_ok = __syncthreads_and(cnt >= 0);
      np = cnt < 0 ? 0 : cnt;
      ++builds;
    }
    F3 D{0.f, 0.f, 0.f};
    if (bead) {
      F3 Fc = bend_drive_forces(a, i, s_rh, s_rl);
      if (a.eps != 0.f) {
        if (nl_ok)
          Fc = Fc + list_forces(a, i, rh, rl, s_rh, s_rl, s_nl + i, np, WS ? s_w + i : nullptr,
                                WS ? nws : -1);
        else
          Fc = Fc + all_pair_forces(a, i, rh, rl, s_rh, s_rl) + wall_stencil_forces(a, rh, rl);
      }
      const float3 xi = gauss3(a.seed, (uint32_t)i, step, (uint32_t)k, 0u);
      const F3 fdrag = (-m * a.gamma) * (v - ui);
      const F3 fr = sig_r * F3{xi.x, xi.y, xi.z};
      v = v + (dt * im) * (Fc + fdrag + fr);
      J = J + dt * (fdrag + fr);
      D = dt * v;  // unconstrained displacement r~ - r
    }
    if (a.has_bonds) {
      // SHAKE on displacements: D_i = dt v_i + (lam_i s_i - lam_{i-1} s_{i-1}) / m
      // with the old bond vectors s_b; Newton on G_b = |s_b + D_{b+1} - D_b|^2 - b0^2.
      // The residual is evaluated in double (old bond from the double-float
      // positions); the Jacobian and the corrections stay in float.
      // Warm start: the multipliers of the previous substep applied along the
      // new old-bond vectors (the constraint forces change slowly).
      float lam = 0.f;
      F3 sb{0.f, 0.f, 0.f};
      if (bead) {
        F3 sm{0.f, 0.f, 0.f};
        if (i > 0) sm = diff_hl(rh, rl, s_rh[i - 1], s_rl[i - 1]);
        if (i < N - 1) {
          sb = diff_hl(s_rh[i + 1], s_rl[i + 1], rh, rl);
          s_b[i] = f4(sb);
          lam = s_lam[i];
          D = D + (lam * im) * sb;
        }
        if (i > 0) D = D - (s_lam[i - 1] * im) * sm;
        s_t[i] = f4(D);
      }
      __syncthreads();
      const float b02 = (float)(b0 * b0);
      for (int it = 0;; ++it) {
        float G = 0.f, diag = 1.f, sub = 0.f, sup = 0.f;
        bool ok = true;
        if (i < N - 1) {
          // old bond from the double-float positions, displacements small: the
          // float residual is good to ~1e-7 of b0^2
          const F3 d = sb + (f3(s_t[i + 1]) - f3(s_t[i]));
          G = dot(d, d) - b02;
          ok = fabsf(G) <= tol * b02;
          diag = -4.0f * im * dot(d, sb);
          if (i > 0) sub = 2.0f * im * dot(d, f3(s_b[i - 1]));
          if (i < N - 2) sup = 2.0f * im * dot(d, f3(s_b[i + 1]));
        }
        if (__syncthreads_and(ok)) break;
        if (it >= a.shake_maxit) {
          const bool bad = (i < N - 1) && !(fabsf(G) <= 1e-3f * b02);
          if (__syncthreads_or(bad)) shake_bad = 1;
          break;
        }
        ++newton_total;
        float xm;
        const float x = spike_tri_solve(N - 1, sub, diag, sup, -G, xm);
        if (bead) {
          F3 dd = f3(s_t[i]);
          if (i < N - 1) {
            dd = dd + (x * im) * f3(s_b[i]);
            lam += x;
          }
          if (i > 0) dd = dd - (xm * im) * f3(s_b[i - 1]);
          s_t[i] = f4(dd);
        }
        __syncthreads();
      }
      if (i < N - 1) s_lam[i] = lam;  // read again only after later barriers
      if (bead) D = f3(s_t[i]);
    }
    if (bead) {
      // v = (r' - r) / dt evaluated as D / dt (no cancellation); r' = r + D
      v = idt * D;
      two_sum_add(rh.x, rl.x, D.x);
      two_sum_add(rh.y, rl.y, D.y);
      two_sum_add(rh.z, rl.z, D.z);
    }
    if (a.has_bonds) {
      // RATTLE: v_i += (mu_i d_i - mu_{i-1} d_{i-1}) / m with the new bond
      // vectors d_b = s_b + D_{b+1} - D_b, so that d_b . (v_{b+1} - v_b) = 0.
      if (bead) s_v[i] = f4(v);
      F3 dnew{0.f, 0.f, 0.f};
      if (i < N - 1) dnew = f3(s_b[i]) + (f3(s_t[i + 1]) - f3(s_t[i]));
      __syncthreads();  // s_v complete; every read of s_b / s_t above done
      if (i < N - 1) s_b[i] = f4(dnew);
      __syncthreads();
      float rhs = 0.f, diag = 1.f, sub = 0.f, sup = 0.f;
      if (i < N - 1) {
        rhs = dot(dnew, f3(s_v[i + 1]) - v);
        diag = -2.0f * im * dot(dnew, dnew);
        if (i > 0) sub = im * dot(dnew, f3(s_b[i - 1]));
        if (i < N - 2) sup = im * dot(dnew, f3(s_b[i + 1]));
      }
      float mum;
      const float mu = spike_tri_solve(N - 1, sub, diag, sup, -rhs, mum);
      if (bead) {
        if (i < N - 1) v = v + (mu * im) * f3(s_b[i]);
        if (i > 0) v = v - (mum * im) * f3(s_b[i - 1]);
      }
    }
    // every read of s_rh / s_rl of this substep precedes a barrier of the
    // constraint solves; without constraints one barrier is needed here
    if (!a.has_bonds) __syncthreads();
    if (bead) {
      s_rh[i] = rh;
      s_rl[i] = rl;
    }
    rebuild = __syncthreads_or(bead && moved());
  }

  if (bead) {
    a.pos[i] = rh;
    a.pos_lo[i] = rl;
    a.vel[i] = f4(v);
    a.J[i] = f4(J);
    a.lam[i] = s_lam[i];
  }
  // Translocation bookkeeping (Sec. III): unwrapped x = origin + hi + lo
  const float xrel = bead ? ((float)(a.ox - a.wall_x) + rh.x) + rl.x : 0.f;
  const bool finite = isfinite(rh.x) && isfinite(rh.y) && isfinite(rh.z) && isfinite(v.x) &&
                      isfinite(v.y) && isfinite(v.z);
  const int nt = __syncthreads_count(bead && a.has_wall && xrel < 0.f);
  const int nan = __syncthreads_or(bead && !finite);
  const int out = __syncthreads_and(!bead || xrel > (float)(a.wall_t - 1) + 1.5f);
  const int bad = __syncthreads_or(shake_bad);
  if (i == 0) {
    DevStatus *st = a.status;
    st->n_trans = nt;
    if (nt > st->max_trans) st->max_trans = nt;
    if (bad) st->shake_fail += 1;
    st->newton_iters = newton_total;
    st->nl_builds += builds;
    st->nl_ok = nl_ok;
    if (st->state == LBMD_RUNNING) {
      if (nan)
        st->state = LBMD_NAN;
      else if (bad)
        st->state = LBMD_SHAKE_FAIL;
      else if (a.has_wall && N > 0) {
        if (nt == N) {
          st->state = LBMD_TRANSLOCATED;
          st->t_transloc = step + 1;
        } else if (st->max_trans >= 1 && out) {
          st->state = LBMD_RETRACTED;
        }
      }
    }
  }
  // Sec. III chain diagnostics at the end of every diag_every-th step: radii
  // of gyration of the translocated (x < x_wall, as N_T) and untranslocated
  // beads from two block sums (centres, then squared distances), the work
  // rates of Eqs. 13-14 and the kinetic energy
  if (a.diag_every > 0 && (step + 1) % a.diag_every == 0) {
    __shared__ float s_red[32 * 6 + 6];
    const bool tr = bead && a.has_wall && xrel < 0.f, un = bead && !tr;
    const F3 r{rh.x + rl.x, rh.y + rl.y, rh.z + rl.z};  // local frame
    float c[6] = {tr ? r.x : 0.f, tr ? r.y : 0.f, tr ? r.z : 0.f,
                  un ? r.x : 0.f, un ? r.y : 0.f, un ? r.z : 0.f};
    block_sum<6>(c, s_red);
    const int nu = N - nt;
    const float it = nt > 0 ? 1.0f / (float)nt : 0.f, iu = nu > 0 ? 1.0f / (float)nu : 0.f;
    const F3 dt_{r.x - c[0] * it, r.y - c[1] * it, r.z - c[2] * it};
    const F3 du_{r.x - c[3] * iu, r.y - c[4] * iu, r.z - c[5] * iu};
    const F3 fd = bead ? drive_force_at(a, rh, rl) : F3{0.f, 0.f, 0.f};
    float q[5] = {tr ? dot(dt_, dt_) : 0.f, un ? dot(du_, du_) : 0.f, bead ? dot(v, ui) : 0.f,
                  dot(fd, v), bead ? dot(v, v) : 0.f};
    block_sum<5>(q, s_red);
    if (i == 0) {
      DevStatus *st = a.status;
      const int k = st->diag_count;
      if (k < a.diag_cap) {
        DevDiag d;
        d.step = step + 1;
        d.n_trans = nt;
        d.r_t = nt > 0 ? sqrtf(q[0] * it) : 0.f;
        d.r_u = nu > 0 ? sqrtf(q[1] * iu) : 0.f;
        d.r_e = powf(powf(d.r_t, 1.0f / 0.6f) + powf(d.r_u, 1.0f / 0.6f), 0.6f);
        d.s_h = a.mass * a.gamma * q[2];
        d.s_e = q[3];
        d.kinetic = 0.5f * a.mass * q[4];
        d.pad = 0;
        a.diag[k] = d;
        st->diag_count = k + 1;
      }
    }
  }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_md_cycle(ChainArgs a) {
  md_cycle_body<BLOCK <= kWallSharedMaxN>(a);
}

// Ensemble variant: block b runs chain chains[b] if its realisation is live.
// The chain's arguments are copied to shared memory once.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_ens_md_cycle(const EnsMember *__restrict__ mem, const int *__restrict__ chains,
                   const int *__restrict__ live) {
  __shared__ ChainArgs s_a;
  const int m = chains[blockIdx.x];
  if (!live[m]) return;  // the whole block leaves together
  static_assert(sizeof(ChainArgs) % sizeof(int) == 0, "ChainArgs copied as ints");
  const int *src = reinterpret_cast<const int *>(&mem[m].a);
  int *dst = reinterpret_cast<int *>(&s_a);
  for (int k = threadIdx.x; k < (int)(sizeof(ChainArgs) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  md_cycle_body<BLOCK <= kWallSharedMaxN>(s_a);
}

// Stage (1) for (bead, corner) pair e = 8 i + k handled by one thread; the
// eight lanes of a bead are consecutive, so the weight normalisation and the
// sum over corners are lane shuffles.  Writes the transfer weights for the
// spread and returns the bead's interpolated u (on every lane of the bead).
template <int S>
__device__ F3 gather_pair(const ChainArgs &a, const void *f, int e, bool valid) {
  using T = typename Store<S>::T;
  const LbGeom &g = a.geo;
  const int i = e >> 3, k = e & 7;
  int node = -1;
  float w = 0.f;
  if (valid) {
    const float4 rh = a.pos[i], rl = a.pos_lo[i];
    int c0[3];
    float s[3];
    cell_frac_hl(rh.x, rl.x, a.ox, g.nx, c0[0], s[0]);
    cell_frac_hl(rh.y, rl.y, a.oy, g.ny, c0[1], s[1]);
    cell_frac_hl(rh.z, rl.z, a.oz, g.nz, c0[2], s[2]);
    int x, y, z;
    if (a.coupling == LBMD_COUPLING_NGP) {
      x = s[0] >= 0.5f ? wrap_p1(c0[0], g.nx) : c0[0];
      y = s[1] >= 0.5f ? wrap_p1(c0[1], g.ny) : c0[1];
      z = s[2] >= 0.5f ? wrap_p1(c0[2], g.nz) : c0[2];
      w = k == 0 ? 1.f : 0.f;
    } else {
      const int ox = k & 1, oy = (k >> 1) & 1, oz = (k >> 2) & 1;
      x = ox ? wrap_p1(c0[0], g.nx) : c0[0];
      y = oy ? wrap_p1(c0[1], g.ny) : c0[1];
      z = oz ? wrap_p1(c0[2], g.nz) : c0[2];
      w = (ox ? s[0] : 1.f - s[0]) * (oy ? s[1] : 1.f - s[1]) * (oz ? s[2] : 1.f - s[2]);
    }
    if (w != 0.f && !solid_at(g.solid, g.ntx, g.ny, x, y, z))
      node = (int)(((size_t)z * g.ny + y) * g.nx + x);
    else
      w = 0.f;
  }
  float wsum = w;
  wsum += __shfl_xor_sync(0xffffffffu, wsum, 1);
  wsum += __shfl_xor_sync(0xffffffffu, wsum, 2);
  wsum += __shfl_xor_sync(0xffffffffu, wsum, 4);
  const float wn = wsum > 0.f ? w / wsum : 0.f;
  if (wn == 0.f) node = -1;
  F3 u{0.f, 0.f, 0.f};
  if (valid) {
    a.sp_node[e] = node;
    a.sp_w[e] = wn;
    if (node >= 0) {
      if (a.owner != nullptr) atomicMin(a.owner + node, e);  // the node's spread owner: its smallest entry
      const int x = node % g.nx, yz = node / g.nx;
      const int y = yz % g.ny, z = yz / g.ny;
      float h[kQ];
      fetch19<S>(g, (const T *)f, x, y, z, a.f_mode, h);
      float drho, jx, jy, jz;
      moments19(h, drho, jx, jy, jz);
      if (a.forcing == LBMD_FORCING_GUO) {
        jx += 0.5f * a.g[0];
        jy += 0.5f * a.g[1];
        jz += 0.5f * a.g[2];
      }
      const float rinv = wn / (a.rho0 + drho);
      u = F3{jx * rinv, jy * rinv, jz * rinv};
    }
  }
#pragma unroll
  for (int m = 1; m < 8; m <<= 1) {
    u.x += __shfl_xor_sync(0xffffffffu, u.x, m);
    u.y += __shfl_xor_sync(0xffffffffu, u.y, m);
    u.z += __shfl_xor_sync(0xffffffffu, u.z, m);
  }
  return u;
}

template <int S>
__global__ void __launch_bounds__(256) k_gather(ChainArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = e < 8 * a.N;
  const F3 u = gather_pair<S>(a, a.f, e, valid);
  if (valid && (e & 7) == 0) a.ui[e >> 3] = f4(u);
}

// Ensemble gather: thread e serves corner e & 7 of padded bead slot e >> 3,
// beads[slot] = (realisation, bead) or m < 0 for padding.  Every realisation's
// slots start at a multiple of four, so a warp never mixes realisations.
template <int S>
__global__ void __launch_bounds__(256)
    k_ens_gather(const EnsMember *__restrict__ mem, const int2 *__restrict__ beads, int nb,
                 const int *__restrict__ live, int cur) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int slot = e >> 3;
  int2 mi = make_int2(-1, 0);
  if (slot < nb) mi = beads[slot];
  const bool valid = mi.x >= 0 && live[mi.x];
  const EnsMember &M = mem[valid ? mi.x : 0];
  const F3 u = gather_pair<S>(M.a, valid ? M.pop[cur] : nullptr, 8 * mi.y + (e & 7), valid);
  if (valid && (e & 7) == 0) M.a.ui[mi.y] = f4(u);
}

cudaError_t md_prepare() {
  const int s512 = (int)md_smem_bytes(kWallSharedMaxN), s1024 = (int)md_smem_bytes(LBMD_MAX_BEADS);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_md_cycle<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, s512)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_md_cycle<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1024)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_ens_md_cycle<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, s512)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_ens_md_cycle<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1024);
}

cudaError_t launch_gather(int storage, const ChainArgs &a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const int blocks = (8 * a.N + 255) / 256;
  switch (storage) {
    case LBMD_STORE_F32: k_gather<LBMD_STORE_F32><<<blocks, 256, 0, s>>>(a); break;
    case LBMD_STORE_F16: k_gather<LBMD_STORE_F16><<<blocks, 256, 0, s>>>(a); break;
    case LBMD_STORE_BF16: k_gather<LBMD_STORE_BF16><<<blocks, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// The MD block is launched at the highest stream priority so that, when it
// and the stream-collide become ready together, its block is placed first.
cudaError_t launch_md_cycle(const ChainArgs &a, int priority, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const int threads = md_threads(a.N);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = md_smem_bytes(a.N);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = priority;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (threads <= 512) return cudaLaunchKernelEx(&cfg, k_md_cycle<512>, a);
  return cudaLaunchKernelEx(&cfg, k_md_cycle<1024>, a);
}

// The sum of the spread as two kernels, one thread per (bead, corner) entry.
__global__ void __launch_bounds__(256) k_spread_accum(ChainArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * a.N) return;
  spread_add(a, e, a.J[e >> 3]);
}
__global__ void __launch_bounds__(256) k_spread_finalize(ChainArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * a.N) return;
  spread_finalize(a, e);
}

// (3) extrapolation of the forces: node x_k receives -sum_i w_ik J_i as the
// source S_p = 3 w_p c_p . F (Eq. 10, reaction sign), added by the node's
// owner entry to the post-collision populations h*_p(x_k), wherever layout
// `mode` holds them: [p][x_k] (pull), [opp(p)][x_k] (in place, after an even
// step), or [p][x_k + c_p] -- [opp(p)][x_k] if x_k + c_p is solid -- (in
// place, after an odd step).  No other thread writes those words in this
// kernel: FP32 adds with one atomic each (no read-back); 16-bit storage reads
// the 18 words first and writes each rounded once.  The owner's force comes
// from its record sp_src[e] (TAKE = false: converted by k_spread_finalize) or
// straight from its fixed-point sum (TAKE = true: the conversion of
// spread_finalize done here, one launch fewer after the MD cycle).
template <int S, bool TAKE>
__global__ void __launch_bounds__(256)
    k_spread_apply(LbGeom g, ChainArgs a, int nw, typename Store<S>::T *dst, int mode,
                   DevStatus *bump) {
  using St = Store<S>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (bump != nullptr && e == 0) {
    bump->step += 1;
    // populations that are not finite end the run as a bead NaN does
    if (bump->pop_bad && bump->state == LBMD_RUNNING) bump->state = LBMD_NAN;
  }
  if (e >= nw) return;
  int node;
  F3 F;
  if (TAKE) {
    node = a.sp_node[e];
    if (node < 0 || a.owner[node] != e) return;  // not an owner
    F = spread_take(a, node, e);
  } else {
    const float4 v = a.sp_src[e];
    node = __float_as_int(v.w);
    if (node < 0) return;  // not an owner
    F = F3{v.x, v.y, v.z};
  }
  const size_t Vp = (size_t)g.Vp;
  uint32_t bb = 0u;
  int x = 0, y = 0, z = 0;
  if (mode == kPopAALocal) {
    x = node % g.nx;
    const int yz = node / g.nx;
    y = yz % g.ny;
    z = yz / g.ny;
    bb = __ldg(&g.lmask[node]);  // bit opp(p): x_k + c_p is solid
  }
  size_t at[kQ];
#pragma unroll
  for (int p = 1; p < kQ; ++p) {
    if (mode == kPopAALocal) {
      const size_t t = ((size_t)wrapi(z + cz(p), g.nz) * g.ny + wrapi(y + cy(p), g.ny)) * g.nx +
                       wrapi(x + cx(p), g.nx);
      at[p] = ((bb >> opp(p)) & 1u) ? (size_t)opp(p) * Vp + node : (size_t)p * Vp + t;
    } else {
      at[p] = (size_t)(mode == kPopAASwap ? opp(p) : p) * Vp + node;
    }
  }
  if (S == LBMD_STORE_F32) {
#pragma unroll
    for (int p = 1; p < kQ; ++p)
      St::add(dst + at[p], 3.0f * wq(p) * (cx(p) * F.x + cy(p) * F.y + cz(p) * F.z));
  } else {
    // all 18 loads first, then the stores: one memory latency, not eighteen
    float hv[kQ];
#pragma unroll
    for (int p = 1; p < kQ; ++p) hv[p] = St::load_plain(dst + at[p]);
#pragma unroll
    for (int p = 1; p < kQ; ++p)
      St::store(dst + at[p], hv[p] + 3.0f * wq(p) * (cx(p) * F.x + cy(p) * F.y + cz(p) * F.z));
  }
}

cudaError_t launch_spread_sum(const ChainArgs &a, bool records, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const int blocks = (8 * a.N + 255) / 256;
  k_spread_accum<<<blocks, 256, 0, s>>>(a);
  if (records) k_spread_finalize<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <int S>
static void apply_as(bool take, int blocks, const LbGeom &g, const ChainArgs &a, int nw, void *dst,
                     int mode, DevStatus *bump, cudaStream_t s) {
  using T = typename Store<S>::T;
  if (take)
    k_spread_apply<S, true><<<blocks, 256, 0, s>>>(g, a, nw, (T *)dst, mode, bump);
  else
    k_spread_apply<S, false><<<blocks, 256, 0, s>>>(g, a, nw, (T *)dst, mode, bump);
}

cudaError_t launch_spread_apply(int storage, const LbGeom &g, const ChainArgs &a, void *dst,
                                int mode, bool take, DevStatus *bump, cudaStream_t s) {
  // no records and no sums without a coupled chain
  const int nw = (take ? a.owner != nullptr : a.sp_src != nullptr) ? 8 * a.N : 0;
  const int blocks = nw > 0 ? (nw + 255) / 256 : 1;
  switch (storage) {
    case LBMD_STORE_F32: apply_as<LBMD_STORE_F32>(take, blocks, g, a, nw, dst, mode, bump, s); break;
    case LBMD_STORE_F16: apply_as<LBMD_STORE_F16>(take, blocks, g, a, nw, dst, mode, bump, s); break;
    case LBMD_STORE_BF16: apply_as<LBMD_STORE_BF16>(take, blocks, g, a, nw, dst, mode, bump, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Ensemble apply: same lane layout as k_ens_gather; each owner entry converts
// its node's sum (k_ens_spread_accum) and adds the source as k_spread_apply
// does.  The first lane of every realisation bumps its step count (if live)
// and decides whether it takes part in the next step.
template <int S>
__global__ void __launch_bounds__(256)
    k_ens_spread(const EnsMember *__restrict__ mem, const int2 *__restrict__ beads, int nb,
                 const int *__restrict__ live, int *__restrict__ live_next, int cur,
                 const long long *__restrict__ max_steps) {
  using St = Store<S>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int slot = e >> 3, k = e & 7;
  int2 mi = make_int2(-1, 0);
  if (slot < nb) mi = beads[slot];
  const bool valid = mi.x >= 0 && live[mi.x];
  if (valid && mem[mi.x].a.owner) {
    const ChainArgs &a = mem[mi.x].a;
    const int e2 = 8 * mi.y + k;
    const int node = a.sp_node[e2];
    if (node >= 0 && a.owner[node] == e2) {  // the owner converts its node's sum
      const F3 F = spread_take(a, node, e2);
      typename St::T *dst = (typename St::T *)mem[mi.x].pop[cur ^ 1];
      const size_t Vp = (size_t)a.geo.Vp;
      if (S == LBMD_STORE_F32) {
#pragma unroll
        for (int p = 1; p < kQ; ++p)
          St::add(dst + (size_t)p * Vp + node, 3.0f * wq(p) * (cx(p) * F.x + cy(p) * F.y + cz(p) * F.z));
      } else {
        float hv[kQ];
#pragma unroll
        for (int p = 1; p < kQ; ++p) hv[p] = St::load_plain(dst + (size_t)p * Vp + node);
#pragma unroll
        for (int p = 1; p < kQ; ++p)
          St::store(dst + (size_t)p * Vp + node,
                    hv[p] + 3.0f * wq(p) * (cx(p) * F.x + cy(p) * F.y + cz(p) * F.z));
      }
    }
  }
  if (mi.x >= 0 && mi.y == 0 && k == 0) {
    int next = 0;
    if (valid) {
      DevStatus *st = mem[mi.x].a.status;
      const long long s = st->step + 1;
      st->step = s;
      st->out_buf = cur ^ 1;
      if (st->pop_bad && st->state == LBMD_RUNNING) st->state = LBMD_NAN;
      next = st->state == LBMD_RUNNING && s < *max_steps;
    }
    live_next[mi.x] = next;
  }
}

cudaError_t launch_ens_gather(int storage, const EnsMember *mem, const int2 *beads, int nb,
                              const int *live, int cur, cudaStream_t s) {
  const int blocks = nb > 0 ? (8 * nb + 255) / 256 : 1;
  switch (storage) {
    case LBMD_STORE_F32: k_ens_gather<LBMD_STORE_F32><<<blocks, 256, 0, s>>>(mem, beads, nb, live, cur); break;
    case LBMD_STORE_F16: k_ens_gather<LBMD_STORE_F16><<<blocks, 256, 0, s>>>(mem, beads, nb, live, cur); break;
    case LBMD_STORE_BF16: k_ens_gather<LBMD_STORE_BF16><<<blocks, 256, 0, s>>>(mem, beads, nb, live, cur); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_ens_md_cycle(const EnsMember *mem, const int *chains, int count, int threads,
                                int max_n, const int *live, int priority, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)count);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = md_smem_bytes(max_n);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = priority;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (threads <= 512) return cudaLaunchKernelEx(&cfg, k_ens_md_cycle<512>, mem, chains, live);
  return cudaLaunchKernelEx(&cfg, k_ens_md_cycle<1024>, mem, chains, live);
}

// Ensemble sum part of the spread, after every MD group: one thread per
// (realisation, bead, corner) entry as in k_ens_gather, adding the entry's
// share to its owner's fixed-point sum (spread_add).
__global__ void __launch_bounds__(256)
    k_ens_spread_accum(const EnsMember *__restrict__ mem, const int2 *__restrict__ beads, int nb,
                       const int *__restrict__ live) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int slot = e >> 3, k = e & 7;
  if (slot >= nb) return;
  const int2 mi = beads[slot];
  if (mi.x < 0 || !live[mi.x]) return;
  const ChainArgs &a = mem[mi.x].a;
  if (a.owner == nullptr) return;  // no solvent: nothing to spread
  spread_add(a, 8 * mi.y + k, a.J[mi.y]);
}

cudaError_t launch_ens_spread_accum(const EnsMember *mem, const int2 *beads, int nb,
                                    const int *live, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  k_ens_spread_accum<<<(8 * nb + 255) / 256, 256, 0, s>>>(mem, beads, nb, live);
  return cudaGetLastError();
}

cudaError_t launch_ens_spread(int storage, const EnsMember *mem, const int2 *beads, int nb,
                              const int *live, int *live_next, int cur,
                              const long long *max_steps, cudaStream_t s) {
  const int blocks = nb > 0 ? (8 * nb + 255) / 256 : 1;
  switch (storage) {
    case LBMD_STORE_F32: k_ens_spread<LBMD_STORE_F32><<<blocks, 256, 0, s>>>(mem, beads, nb, live, live_next, cur, max_steps); break;
    case LBMD_STORE_F16: k_ens_spread<LBMD_STORE_F16><<<blocks, 256, 0, s>>>(mem, beads, nb, live, live_next, cur, max_steps); break;
    case LBMD_STORE_BF16: k_ens_spread<LBMD_STORE_BF16><<<blocks, 256, 0, s>>>(mem, beads, nb, live, live_next, cur, max_steps); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void k_read_beads(const float4 *pos, const float4 *pos_lo, const float4 *vel, int N,
                             int ox, int oy, int oz, double *dpos, double *dvel) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (dpos) {
    const float4 r = pos[i];
    const float4 l = pos_lo ? pos_lo[i] : make_float4(0, 0, 0, 0);
    dpos[3 * i] = (double)ox + (double)r.x + (double)l.x;
    dpos[3 * i + 1] = (double)oy + (double)r.y + (double)l.y;
    dpos[3 * i + 2] = (double)oz + (double)r.z + (double)l.z;
  }
  if (dvel) {
    const float4 v = vel[i];
    dvel[3 * i] = v.x;
    dvel[3 * i + 1] = v.y;
    dvel[3 * i + 2] = v.z;
  }
}

cudaError_t launch_read_beads(const float4 *pos, const float4 *pos_lo, const float4 *vel, int N,
                              int ox, int oy, int oz, double *dpos, double *dvel, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_read_beads<<<(N + 255) / 256, 256, 0, s>>>(pos, pos_lo, vel, N, ox, oy, oz, dpos, dvel);
  return cudaGetLastError();
}

// The block of lbmd_read_beads_async: the status word at offset 0, then the
// unwrapped positions and the velocities (3N doubles each) from offset 32.
__global__ void k_bead_block(const float4 *pos, const float4 *pos_lo, const float4 *vel, int N,
                             int ox, int oy, int oz, const DevStatus *st, char *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    lbmd_status_word *w = (lbmd_status_word *)out;
    w->step = st->step;
    w->t_transloc = st->t_transloc;
    w->n_trans = st->n_trans;
    // a box without beads has no apply kernel to fold the population flag in
    w->state = st->state == LBMD_RUNNING && st->pop_bad ? LBMD_NAN : st->state;
    // the header's padding reads zero: every byte of the block is defined
    for (size_t b = sizeof(lbmd_status_word); b < kBeadBlockHeader; b += sizeof(int)) *(int *)(out + b) = 0;
  }
  if (i >= N) return;
  double *dpos = (double *)(out + kBeadBlockHeader), *dvel = dpos + 3 * (size_t)N;
  const float4 r = pos[i], l = pos_lo[i], v = vel[i];
  dpos[3 * i] = (double)ox + (double)r.x + (double)l.x;
  dpos[3 * i + 1] = (double)oy + (double)r.y + (double)l.y;
  dpos[3 * i + 2] = (double)oz + (double)r.z + (double)l.z;
  dvel[3 * i] = v.x;
  dvel[3 * i + 1] = v.y;
  dvel[3 * i + 2] = v.z;
}

const void *bead_block_kernel() { return reinterpret_cast<const void *>(&k_bead_block); }

cudaError_t launch_bead_block(const ChainArgs &a, const DevStatus *st, void *out, cudaStream_t s) {
  const int n = a.N > 0 ? a.N : 1;
  k_bead_block<<<(n + 255) / 256, 256, 0, s>>>(a.pos, a.pos_lo, a.vel, a.N, a.ox, a.oy, a.oz, st,
                                               (char *)out);
  return cudaGetLastError();
}

cudaError_t launch_read_bead_aux(const float4 *ui, const float4 *J, int N, double *dui,
                                 double *dJ, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_read_beads<<<(N + 255) / 256, 256, 0, s>>>(ui, nullptr, J, N, 0, 0, 0, dui, dJ);
  return cudaGetLastError();
}

}  // namespace lbmd
