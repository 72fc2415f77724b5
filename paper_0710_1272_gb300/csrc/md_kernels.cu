// md_kernels.cu -- bead <-> fluid coupling and the constrained polymer MD cycle
// (arXiv:0710.1272, Sec. II: Eqs. 1-4, 10, the four-stage LB step; Sec. III:
// pulling force, wall, translocation bookkeeping).
//
// k_md_cycle runs one thread block per chain, one thread per bead:
//   gather u_i (trilinear over fluid corners, or nearest grid point) from the
//   pulled pre-collision populations, then M substeps of
//     F = F_WCA + F_bend + F_wall + F_drive - m gamma (v - u_i) + F_r,
//     v += dt F / m,  r~ = r + dt v,
//     SHAKE: Newton on the N-1 bond multipliers, the tridiagonal Jacobian
//            solved by parallel cyclic reduction in shared memory,
//     v = (r' - r) / dt,  r = r',
//     RATTLE: one tridiagonal solve removes the bond-parallel relative
//             velocities,
//     J_i += dt (F_drag + F_r);
//   then the translocation bookkeeping.  k_spread hands -J_i to the fluid with
//   the gather weights (warp-aggregated atomics into the post-collision
//   populations, Eq. 10 with the reaction sign).
#include "lb_pull.cuh"

namespace lbmd {

constexpr float kTwoSixth = 1.122462048309373f;  // 2^(1/6)

struct F3 {
  float x, y, z;
};
__device__ __forceinline__ F3 f3(float4 v) { return F3{v.x, v.y, v.z}; }
__device__ __forceinline__ float4 f4(F3 v) { return make_float4(v.x, v.y, v.z, 0.f); }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return F3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return F3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return F3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Threads of the MD block for a chain of N beads: enough to give every
// (bead, corner) pair of the gather its own thread and to split the pair-force
// loop, at most 1024.
int md_threads(int N) {
  const int n32 = (N + 31) / 32 * 32;
  return n32 >= 256 ? 1024 : (4 * n32 < 128 ? 128 : 4 * n32);
}

size_t md_smem_bytes(int N) {
  const int T = md_threads(N);
  const int n32 = (N + 31) / 32 * 32;
  const int nsplit = T / n32;
  // s_rh, s_rl, s_ui, s_t, s_b, s_v (float4), PCR (8 floats), x, partial forces
  return (size_t)N * (6 * sizeof(float4) + 9 * sizeof(float)) +
         (size_t)(nsplit - 1) * n32 * sizeof(float4);
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
// Wrapped node index and fraction of global = origin + hi + lo.
__device__ __forceinline__ void cell_frac_hl(float hi, float lo, int origin, int n, int &cell,
                                             float &frac) {
  const float fl = floorf(hi);
  frac = (hi - fl) + lo;
  cell = wrapi(origin + (int)fl, n);
}

// Tridiagonal solve by parallel cyclic reduction over rows 0..n-1 (one row
// per thread, a_0 = c_{n-1} = 0).  Every thread of the block must call it.
__device__ float pcr_solve(int n, float a, float b, float c, float d, float *tri, int N) {
  const int i = threadIdx.x;
  float *buf[2] = {tri, tri + 4 * N};
  if (i < n) {
    buf[0][i] = a;
    buf[0][N + i] = b;
    buf[0][2 * N + i] = c;
    buf[0][3 * N + i] = d;
  }
  __syncthreads();
  int cur = 0;
  for (int s = 1; s < n; s <<= 1) {
    const float *A = buf[cur], *B = buf[cur] + N, *C = buf[cur] + 2 * N, *D = buf[cur] + 3 * N;
    float *An = buf[cur ^ 1], *Bn = An + N, *Cn = An + 2 * N, *Dn = An + 3 * N;
    if (i < n) {
      float ai = A[i], bi = B[i], ci = C[i], di = D[i];
      float an = 0.f, cn = 0.f;
      if (i - s >= 0) {
        const float k1 = ai / B[i - s];
        bi -= k1 * C[i - s];
        di -= k1 * D[i - s];
        an = -k1 * A[i - s];
      }
      if (i + s < n) {
        const float k2 = ci / B[i + s];
        bi -= k2 * A[i + s];
        di -= k2 * D[i + s];
        cn = -k2 * C[i + s];
      }
      An[i] = an;
      Bn[i] = bi;
      Cn[i] = cn;
      Dn[i] = di;
    }
    __syncthreads();
    cur ^= 1;
  }
  return i < n ? buf[cur][3 * N + i] / buf[cur][N + i] : 0.f;
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

// Stage (1) for (bead, corner) pair e = 8 i + k handled by one thread; the
// eight lanes of a bead are consecutive, so the weight normalisation and the
// sum over corners are lane shuffles.  Writes the transfer weights for the
// spread and returns the bead's interpolated u on the corner-0 lane.
template <int S>
__device__ F3 gather_pair(const ChainArgs &a, int e, bool valid, const float4 *s_rh,
                          const float4 *s_rl) {
  using T = typename Store<S>::T;
  const LbGeom &g = a.geo;
  const int i = e >> 3, k = e & 7;
  int node = -1;
  float w = 0.f;
  if (valid) {
    const float4 rh = s_rh[i], rl = s_rl[i];
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
      const int x = node % g.nx, yz = node / g.nx;
      float h[kQ];
      pull19<S, true>(g, (const T *)a.f, x, yz % g.ny, yz / g.ny, h);
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

// WCA pair forces on bead i from beads j in [j0, j1) (non-bonded pairs,
// minimum image), with separations from the double-float positions.
__device__ __forceinline__ F3 pair_forces(const ChainArgs &a, int i, int j0, int j1,
                                          const float4 *s_rh, const float4 *s_rl) {
  const LbGeom &g = a.geo;
  const float sig2 = a.sigma * a.sigma;
  const float rc = kTwoSixth * a.sigma, rc2 = rc * rc;
  const float eps24 = 24.0f * a.eps;
  const float Lx = (float)g.nx, Ly = (float)g.ny, Lz = (float)g.nz;
  const float iLx = 1.0f / Lx, iLy = 1.0f / Ly, iLz = 1.0f / Lz;
  const float4 rh = s_rh[i], rl = s_rl[i];
  F3 F{0.f, 0.f, 0.f};
  for (int j = j0; j < j1; ++j) {
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

// Bending, wall and drive forces on bead i.
__device__ F3 local_forces(const ChainArgs &a, int i, const float4 *s_rh, const float4 *s_rl) {
  const LbGeom &g = a.geo;
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
  const float4 rh = s_rh[i], rl = s_rl[i];
  int c[3];
  float s[3];
  cell_frac_hl(rh.x, rl.x, a.ox, g.nx, c[0], s[0]);
  cell_frac_hl(rh.y, rl.y, a.oy, g.ny, c[1], s[1]);
  cell_frac_hl(rh.z, rl.z, a.oz, g.nz, c[2], s[2]);
  if (a.eps != 0.f) {
    // wall: Eq. 2 between the bead and every solid node closer than the cutoff;
    // node offsets n with |n - s| < rc: n in [ceil(s - rc), floor(s + rc)]
    const float sig2 = a.sigma * a.sigma;
    const float rc = kTwoSixth * a.sigma, rc2 = rc * rc;
    const float eps24 = 24.0f * a.eps;
    const int lo0 = (int)ceilf(s[0] - rc), hi0 = (int)floorf(s[0] + rc);
    const int lo1 = (int)ceilf(s[1] - rc), hi1 = (int)floorf(s[1] + rc);
    const int lo2 = (int)ceilf(s[2] - rc), hi2 = (int)floorf(s[2] + rc);
    for (int ox = lo0; ox <= hi0; ++ox) {
      const int x = wrapi(c[0] + ox, g.nx);
      if (!__ldg(&a.xslab[x])) continue;
      const float dx = s[0] - (float)ox;
      for (int oy = lo1; oy <= hi1; ++oy) {
        const int y = wrapi(c[1] + oy, g.ny);
        const float dy = s[1] - (float)oy;
        for (int oz = lo2; oz <= hi2; ++oz) {
          const int z = wrapi(c[2] + oz, g.nz);
          if (!solid_at(g.solid, g.ntx, g.ny, x, y, z)) continue;
          wca_add(F3{dx, dy, s[2] - (float)oz}, sig2, rc2, eps24, F);
        }
      }
    }
  }
  // pulling force of Sec. III inside the channel through the pore
  if (a.has_wall && a.pore_d > 0 && a.fdrive != 0.f) {
    const int di = wrapi(c[0] - a.wall_x + g.nx / 2, g.nx) - g.nx / 2;
    const float dx = (float)di + s[0] - 0.5f * (float)(a.wall_t - 1);
    const float half = 0.5f * (float)(a.wall_t - 1) + 1.5f;
    const float ry = (float)c[1] + s[1], rz = (float)c[2] + s[2];
    if (fabsf(dx) <= half && ry >= a.pore_y0 - 0.5f && ry < a.pore_y0 + a.pore_d - 0.5f &&
        rz >= a.pore_z0 - 0.5f && rz < a.pore_z0 + a.pore_d - 0.5f)
      F.x -= a.fdrive;
  }
  return F;
}

template <int S>
__global__ void __launch_bounds__(1024) k_md_cycle(ChainArgs a) {
  extern __shared__ float4 smem4[];
  const int N = a.N;
  const int T = blockDim.x;
  const int t = threadIdx.x;
  const int i = t;  // bead of this thread in the per-bead phases
  const bool bead = i < N;
  const int n32 = (N + 31) / 32 * 32;
  const int nsplit = T / n32;
  float4 *s_rh = smem4;      // positions, hi part (start of the substep)
  float4 *s_rl = s_rh + N;   // positions, lo part
  float4 *s_ui = s_rl + N;   // interpolated fluid velocity
  float4 *s_t = s_ui + N;    // displacement of the substep
  float4 *s_b = s_t + N;     // bond vectors
  float4 *s_v = s_b + N;     // velocities (RATTLE)
  float4 *s_fp = s_v + N;    // partial pair forces of splits 1..nsplit-1
  float *tri = (float *)(s_fp + (nsplit - 1) * n32);  // 8N: two PCR buffers
  float *s_x = tri + 8 * N;                             // N: PCR solution

  const long long step = a.status->step;
  float4 rh = make_float4(0, 0, 0, 0), rl = rh;
  F3 v{0.f, 0.f, 0.f};
  if (bead) {
    rh = a.pos[i];
    rl = a.pos_lo[i];
    v = f3(a.vel[i]);
    s_rh[i] = rh;
    s_rl[i] = rl;
  }
  __syncthreads();
  // (1) interpolation of the fluid velocity, frozen for the M substeps
  for (int e0 = 0; e0 < 8 * N; e0 += T) {
    const int e = e0 + t;
    const F3 u = gather_pair<S>(a, e, e < 8 * N, s_rh, s_rl);
    if (e < 8 * N && (e & 7) == 0) s_ui[e >> 3] = f4(u);
  }
  __syncthreads();
  const F3 ui = bead ? f3(s_ui[i]) : F3{0.f, 0.f, 0.f};
  F3 J{0.f, 0.f, 0.f};
  const float dt = a.dt, m = a.mass, im = 1.0f / a.mass, idt = 1.0f / a.dt;
  const float sig_r = sqrtf(2.0f * m * a.gamma * a.kT / dt);
  const float b0 = (bead && i < N - 1 && a.has_bonds) ? a.b0[i] : 1.f;
  const float tol = fmaxf(a.shake_tol, 1e-6f);
  int shake_bad = 0, newton_total = 0;
  const int fsplit = t / n32, fi = t - fsplit * n32;  // pair-force split of this thread
  const int chunk = (N + nsplit - 1) / nsplit;

  for (int k = 0; k < a.M; ++k) {  // (2) M MD substeps
    // pair forces, the j-range split over nsplit groups of threads
    F3 Fp{0.f, 0.f, 0.f};
    if (a.eps != 0.f && fi < N && fsplit < nsplit)
      Fp = pair_forces(a, fi, fsplit * chunk, min(N, (fsplit + 1) * chunk), s_rh, s_rl);
    if (fsplit >= 1 && fsplit < nsplit && fi < N) s_fp[(fsplit - 1) * n32 + fi] = f4(Fp);
    __syncthreads();
    F3 D{0.f, 0.f, 0.f};
    if (bead) {
      F3 Fc = Fp;
      for (int q = 1; q < nsplit; ++q) Fc = Fc + f3(s_fp[(q - 1) * n32 + i]);
      Fc = Fc + local_forces(a, i, s_rh, s_rl);
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
      if (bead) {
        s_t[i] = f4(D);
        if (i < N - 1) s_b[i] = f4(diff_hl(s_rh[i + 1], s_rl[i + 1], rh, rl));
      }
      __syncthreads();
      for (int it = 0;; ++it) {
        float G = 0.f, diag = 1.f, sub = 0.f, sup = 0.f;
        bool ok = true;
        if (i < N - 1) {
          const F3 sb = f3(s_b[i]);
          const F3 d = sb + (f3(s_t[i + 1]) - f3(s_t[i]));
          G = dot(d, d) - b0 * b0;
          ok = fabsf(G) <= tol * b0 * b0;
          diag = -4.0f * im * dot(d, sb);
          if (i > 0) sub = 2.0f * im * dot(d, f3(s_b[i - 1]));
          if (i < N - 2) sup = 2.0f * im * dot(d, f3(s_b[i + 1]));
        }
        if (__syncthreads_and(ok)) break;
        if (it >= a.shake_maxit) {
          const bool bad = (i < N - 1) && !(fabsf(G) <= 1e-3f * b0 * b0);
          if (__syncthreads_or(bad)) shake_bad = 1;
          break;
        }
        ++newton_total;
        const float x = pcr_solve(N - 1, sub, diag, sup, -G, tri, N);
        if (i < N - 1) s_x[i] = x;
        __syncthreads();
        if (bead) {
          F3 dd = f3(s_t[i]);
          if (i < N - 1) dd = dd + (s_x[i] * im) * f3(s_b[i]);
          if (i > 0) dd = dd - (s_x[i - 1] * im) * f3(s_b[i - 1]);
          s_t[i] = f4(dd);
        }
        __syncthreads();
      }
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
      const float mu = pcr_solve(N - 1, sub, diag, sup, -rhs, tri, N);
      if (i < N - 1) s_x[i] = mu;
      __syncthreads();
      if (bead) {
        if (i < N - 1) v = v + (s_x[i] * im) * f3(s_b[i]);
        if (i > 0) v = v - (s_x[i - 1] * im) * f3(s_b[i - 1]);
      }
    }
    __syncthreads();  // every read of s_rh / s_rl of this substep is done
    if (bead) {
      s_rh[i] = rh;
      s_rl[i] = rl;
    }
    __syncthreads();
  }

  if (bead) {
    a.pos[i] = rh;
    a.pos_lo[i] = rl;
    a.vel[i] = f4(v);
    a.ui[i] = f4(ui);
    a.J[i] = f4(J);
  }
  // Translocation bookkeeping (Sec. III): unwrapped x = origin + hi + lo
  const float xrel = bead ? ((float)(a.ox - a.wall_x) + rh.x) + rl.x : 0.f;
  const bool finite = isfinite(rh.x) && isfinite(rh.y) && isfinite(rh.z) && isfinite(v.x) &&
                      isfinite(v.y) && isfinite(v.z);
  const int nt = __syncthreads_count(bead && a.has_wall && xrel < 0.f);
  const int nan = __syncthreads_or(bead && !finite);
  const int out = __syncthreads_and(!bead || xrel > (float)(a.wall_t - 1) + 1.5f);
  const int bad = __syncthreads_or(shake_bad);
  if (t == 0) {
    DevStatus *st = a.status;
    st->n_trans = nt;
    if (nt > st->max_trans) st->max_trans = nt;
    if (bad) st->shake_fail += 1;
    st->newton_iters = newton_total;
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
}

cudaError_t md_prepare(int storage, int N) {
  const int smem = (int)md_smem_bytes(N);
  switch (storage) {
    case LBMD_STORE_F32:
      return cudaFuncSetAttribute(k_md_cycle<LBMD_STORE_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case LBMD_STORE_F16:
      return cudaFuncSetAttribute(k_md_cycle<LBMD_STORE_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case LBMD_STORE_BF16:
      return cudaFuncSetAttribute(k_md_cycle<LBMD_STORE_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_md_cycle(int storage, const ChainArgs &a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const int threads = md_threads(a.N);
  const size_t smem = md_smem_bytes(a.N);
  switch (storage) {
    case LBMD_STORE_F32: k_md_cycle<LBMD_STORE_F32><<<1, threads, smem, s>>>(a); break;
    case LBMD_STORE_F16: k_md_cycle<LBMD_STORE_F16><<<1, threads, smem, s>>>(a); break;
    case LBMD_STORE_BF16: k_md_cycle<LBMD_STORE_BF16><<<1, threads, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// (3) extrapolation of the forces: node x_k receives -w_ik J_i as the source
// S_p = 3 w_p c_p . F (Eq. 10, reaction sign) added to the post-collision
// populations.  Lanes of a warp that hit the same node sum their vectors
// first (in lane order), and one lane issues the 18 atomic adds.
// ---------------------------------------------------------------------------
template <int S>
__global__ void k_spread(LbGeom g, const int *__restrict__ sp_node, const float *__restrict__ sp_w,
                         const float4 *__restrict__ J, int nw, typename Store<S>::T *dst,
                         DevStatus *bump) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (bump != nullptr && e == 0) bump->step += 1;
  if (blockIdx.x * blockDim.x >= nw) return;  // whole warp out of range
  const int lane = threadIdx.x & 31;
  int node = -1;
  F3 F{0.f, 0.f, 0.f};
  if (e < nw) {
    node = sp_node[e];
    if (node >= 0) {
      const float w = sp_w[e];
      const float4 j = J[e >> 3];
      F = F3{-w * j.x, -w * j.y, -w * j.z};
    }
  }
  const unsigned peers = __match_any_sync(0xffffffffu, node);
  F3 sum{0.f, 0.f, 0.f};
#pragma unroll 4
  for (int l = 0; l < 32; ++l) {
    const float vx = __shfl_sync(0xffffffffu, F.x, l);
    const float vy = __shfl_sync(0xffffffffu, F.y, l);
    const float vz = __shfl_sync(0xffffffffu, F.z, l);
    if ((peers >> l) & 1u) sum = sum + F3{vx, vy, vz};
  }
  const int leader = __ffs(peers) - 1;
  if (node >= 0 && lane == leader) {
    using St = Store<S>;
    const size_t Vp = (size_t)g.Vp;
#pragma unroll
    for (int p = 1; p < kQ; ++p) {
      const float cf = cx(p) * sum.x + cy(p) * sum.y + cz(p) * sum.z;
      St::add(dst + (size_t)p * Vp + node, 3.0f * wq(p) * cf);
    }
  }
}

cudaError_t launch_spread(int storage, const LbGeom &g, const int *sp_node, const float *sp_w,
                          const float4 *J, int N, int nw, void *dst, DevStatus *bump,
                          cudaStream_t s) {
  (void)N;
  const int threads = 256;
  const int blocks = nw > 0 ? (nw + threads - 1) / threads : 1;
  switch (storage) {
    case LBMD_STORE_F32:
      k_spread<LBMD_STORE_F32><<<blocks, threads, 0, s>>>(g, sp_node, sp_w, J, nw, (float *)dst, bump);
      break;
    case LBMD_STORE_F16:
      k_spread<LBMD_STORE_F16><<<blocks, threads, 0, s>>>(g, sp_node, sp_w, J, nw, (__half *)dst, bump);
      break;
    case LBMD_STORE_BF16:
      k_spread<LBMD_STORE_BF16><<<blocks, threads, 0, s>>>(g, sp_node, sp_w, J, nw, (__nv_bfloat16 *)dst, bump);
      break;
    default:
      return cudaErrorInvalidValue;
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

cudaError_t launch_read_bead_aux(const float4 *ui, const float4 *J, int N, double *dui,
                                 double *dJ, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_read_beads<<<(N + 255) / 256, 256, 0, s>>>(ui, nullptr, J, N, 0, 0, 0, dui, dJ);
  return cudaGetLastError();
}

}  // namespace lbmd
