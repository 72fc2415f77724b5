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

size_t md_smem_bytes(int N) {
  // s_r, s_t, s_b, s_v (float4 each), two PCR buffers of (a, b, c, d), x
  return (size_t)N * (4 * sizeof(float4) + 9 * sizeof(float));
}

// Split an unwrapped local coordinate into a wrapped node index and the
// fraction in [0, 1): global = origin + local.
__device__ __forceinline__ void cell_frac(float local, int origin, int n, int &cell, float &frac) {
  const float fl = floorf(local);
  frac = local - fl;
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

// Eq. 3 bending at the angle of beads (a, b, c): returns the force on the
// bead at position `which` (0 = a, 1 = b, 2 = c).
__device__ __forceinline__ F3 bend_force(F3 ra, F3 rb, F3 rc, float kappa, int which) {
  const F3 b1 = rb - ra, b2 = rc - rb;
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

template <int S>
__device__ void gather_bead(const ChainArgs &a, F3 r, int i, F3 &ui) {
  using T = typename Store<S>::T;
  const LbGeom &g = a.geo;
  int c0[3];
  float s[3];
  cell_frac(r.x, a.ox, g.nx, c0[0], s[0]);
  cell_frac(r.y, a.oy, g.ny, c0[1], s[1]);
  cell_frac(r.z, a.oz, g.nz, c0[2], s[2]);
  int node[8];
  float w[8];
  float wsum = 0.f;
  if (a.coupling == LBMD_COUPLING_NGP) {
    const int x = s[0] >= 0.5f ? wrap_p1(c0[0], g.nx) : c0[0];
    const int y = s[1] >= 0.5f ? wrap_p1(c0[1], g.ny) : c0[1];
    const int z = s[2] >= 0.5f ? wrap_p1(c0[2], g.nz) : c0[2];
    const bool sol = solid_at(g.solid, g.ntx, g.ny, x, y, z);
    node[0] = sol ? -1 : (int)(((size_t)z * g.ny + y) * g.nx + x);
    w[0] = sol ? 0.f : 1.f;
    wsum = w[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      node[k] = -1;
      w[k] = 0.f;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ox = k & 1, oy = (k >> 1) & 1, oz = (k >> 2) & 1;
      const int x = ox ? wrap_p1(c0[0], g.nx) : c0[0];
      const int y = oy ? wrap_p1(c0[1], g.ny) : c0[1];
      const int z = oz ? wrap_p1(c0[2], g.nz) : c0[2];
      const bool sol = solid_at(g.solid, g.ntx, g.ny, x, y, z);
      const float wk = (ox ? s[0] : 1.f - s[0]) * (oy ? s[1] : 1.f - s[1]) * (oz ? s[2] : 1.f - s[2]);
      node[k] = sol ? -1 : (int)(((size_t)z * g.ny + y) * g.nx + x);
      w[k] = sol ? 0.f : wk;
      wsum += w[k];
    }
  }
  ui = F3{0.f, 0.f, 0.f};
  const float inv = wsum > 0.f ? 1.0f / wsum : 0.f;
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const float wk = w[k] * inv;
    a.sp_node[8 * i + k] = node[k];
    a.sp_w[8 * i + k] = wk;
    if (node[k] < 0) continue;
    const int x = node[k] % g.nx, yz = node[k] / g.nx;
    const int y = yz % g.ny, z = yz / g.ny;
    float h[kQ];
    pull19<S, true>(g, (const T *)a.f, x, y, z, h);
    float drho, jx, jy, jz;
    moments19(h, drho, jx, jy, jz);
    if (a.forcing == LBMD_FORCING_GUO) {
      jx += 0.5f * a.g[0];
      jy += 0.5f * a.g[1];
      jz += 0.5f * a.g[2];
    }
    const float rinv = wk / (a.rho0 + drho);
    ui = ui + F3{jx * rinv, jy * rinv, jz * rinv};
  }
}

// Conservative + external forces on bead i (WCA pairs, bending, wall, drive).
__device__ F3 bead_forces(const ChainArgs &a, int i, F3 r, const float4 *s_r) {
  const LbGeom &g = a.geo;
  const int N = a.N;
  const float sig2 = a.sigma * a.sigma;
  const float rc = kTwoSixth * a.sigma, rc2 = rc * rc;
  const float eps24 = 24.0f * a.eps;
  const float Lx = (float)g.nx, Ly = (float)g.ny, Lz = (float)g.nz;
  F3 F{0.f, 0.f, 0.f};
  if (a.eps != 0.f) {
    for (int j = 0; j < N; ++j) {
      const int dij = j - i;
      if (dij == 0 || (a.has_bonds && (dij == 1 || dij == -1))) continue;
      F3 d = r - f3(s_r[j]);
      d.x -= Lx * floorf(d.x / Lx + 0.5f);
      d.y -= Ly * floorf(d.y / Ly + 0.5f);
      d.z -= Lz * floorf(d.z / Lz + 0.5f);
      wca_add(d, sig2, rc2, eps24, F);
    }
  }
  if (a.kappa != 0.f && a.has_bonds) {
    if (i >= 2) F = F + bend_force(f3(s_r[i - 2]), f3(s_r[i - 1]), r, a.kappa, 2);
    if (i >= 1 && i + 1 < N) F = F + bend_force(f3(s_r[i - 1]), r, f3(s_r[i + 1]), a.kappa, 1);
    if (i + 2 < N) F = F + bend_force(r, f3(s_r[i + 1]), f3(s_r[i + 2]), a.kappa, 0);
  }
  // wall: Eq. 2 between the bead and every solid node within the cutoff
  int c[3];
  float s[3];
  cell_frac(r.x, a.ox, g.nx, c[0], s[0]);
  cell_frac(r.y, a.oy, g.ny, c[1], s[1]);
  cell_frac(r.z, a.oz, g.nz, c[2], s[2]);
  if (a.eps != 0.f) {
    // node offsets n with |n - s| < rc along each axis: n in [ceil(s - rc), floor(s + rc)]
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
    int di = wrapi(c[0] - a.wall_x + g.nx / 2, g.nx) - g.nx / 2;
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
  const int i = threadIdx.x;
  const bool bead = i < N;
  float4 *s_r = smem4;       // positions at the start of the substep
  float4 *s_t = s_r + N;     // trial / constrained positions
  float4 *s_b = s_t + N;     // bond vectors
  float4 *s_v = s_b + N;     // velocities (RATTLE)
  float *tri = (float *)(s_v + N);  // 8N: two PCR buffers
  float *s_x = tri + 8 * N;         // N: PCR solution

  const long long step = a.status->step;
  F3 r{0.f, 0.f, 0.f}, v{0.f, 0.f, 0.f}, ui{0.f, 0.f, 0.f}, J{0.f, 0.f, 0.f};
  if (bead) {
    r = f3(a.pos[i]);
    v = f3(a.vel[i]);
    // (1) interpolation of the fluid velocity, frozen for the M substeps
    gather_bead<S>(a, r, i, ui);
  }
  const float dt = a.dt, m = a.mass, im = 1.0f / a.mass;
  const float sig_r = sqrtf(2.0f * m * a.gamma * a.kT / dt);
  const float b0 = (bead && i < N - 1 && a.has_bonds) ? a.b0[i] : 1.f;
  const float tol = fmaxf(a.shake_tol, 2e-5f);
  int shake_bad = 0;

  for (int k = 0; k < a.M; ++k) {  // (2) M MD substeps
    if (bead) s_r[i] = f4(r);
    __syncthreads();
    F3 rt{0.f, 0.f, 0.f};
    if (bead) {
      const F3 Fc = bead_forces(a, i, r, s_r);
      const float3 xi = gauss3(a.seed, (uint32_t)i, step, (uint32_t)k, 0u);
      const F3 fdrag = (-m * a.gamma) * (v - ui);
      const F3 fr = sig_r * F3{xi.x, xi.y, xi.z};
      v = v + (dt * im) * (Fc + fdrag + fr);
      J = J + dt * (fdrag + fr);
      rt = r + dt * v;
    }
    if (a.has_bonds) {
      // SHAKE: r'_i = r~_i + (lam_i s_i - lam_{i-1} s_{i-1}) / m with the old
      // bond vectors s_b; Newton on G_b = |d_b|^2 - b0^2 = 0.
      if (bead) {
        s_t[i] = f4(rt);
        if (i < N - 1) s_b[i] = f4(f3(s_r[i + 1]) - r);
      }
      __syncthreads();
      for (int it = 0;; ++it) {
        float G = 0.f, diag = 1.f, sub = 0.f, sup = 0.f;
        bool ok = true;
        if (i < N - 1) {
          const F3 d = f3(s_t[i + 1]) - f3(s_t[i]);
          G = dot(d, d) - b0 * b0;
          ok = fabsf(G) <= tol * b0 * b0;
          diag = -4.0f * im * dot(d, f3(s_b[i]));
          if (i > 0) sub = 2.0f * im * dot(d, f3(s_b[i - 1]));
          if (i < N - 2) sup = 2.0f * im * dot(d, f3(s_b[i + 1]));
        }
        if (__syncthreads_and(ok)) break;
        if (it >= a.shake_maxit) {
          const bool bad = (i < N - 1) && !(fabsf(G) <= 1e-3f * b0 * b0);
          if (__syncthreads_or(bad)) shake_bad = 1;
          break;
        }
        const float x = pcr_solve(N - 1, sub, diag, sup, -G, tri, N);
        if (i < N - 1) s_x[i] = x;
        __syncthreads();
        if (bead) {
          F3 t = f3(s_t[i]);
          if (i < N - 1) t = t + (s_x[i] * im) * f3(s_b[i]);
          if (i > 0) t = t - (s_x[i - 1] * im) * f3(s_b[i - 1]);
          s_t[i] = f4(t);
        }
        __syncthreads();
      }
      if (bead) rt = f3(s_t[i]);
    }
    if (bead) {
      v = (1.0f / dt) * (rt - r);
      r = rt;
    }
    if (a.has_bonds) {
      // RATTLE: v_i += (mu_i d_i - mu_{i-1} d_{i-1}) / m with d_b the new bonds,
      // chosen so that d_b . (v_{b+1} - v_b) = 0 for every bond.
      __syncthreads();  // every read of s_t / s_b above is done
      if (bead) {
        s_r[i] = f4(r);
        s_v[i] = f4(v);
      }
      __syncthreads();
      if (i < N - 1) s_b[i] = f4(f3(s_r[i + 1]) - r);
      __syncthreads();
      float rhs = 0.f, diag = 1.f, sub = 0.f, sup = 0.f;
      if (i < N - 1) {
        const F3 d = f3(s_b[i]);
        rhs = dot(d, f3(s_v[i + 1]) - v);
        diag = -2.0f * im * dot(d, d);
        if (i > 0) sub = im * dot(d, f3(s_b[i - 1]));
        if (i < N - 2) sup = im * dot(d, f3(s_b[i + 1]));
      }
      const float mu = pcr_solve(N - 1, sub, diag, sup, -rhs, tri, N);
      if (i < N - 1) s_x[i] = mu;
      __syncthreads();
      if (bead) {
        if (i < N - 1) v = v + (s_x[i] * im) * f3(s_b[i]);
        if (i > 0) v = v - (s_x[i - 1] * im) * f3(s_b[i - 1]);
      }
    }
    __syncthreads();  // s_r is rewritten at the top of the next substep
  }

  if (bead) {
    a.pos[i] = f4(r);
    a.vel[i] = f4(v);
    a.ui[i] = f4(ui);
    a.J[i] = f4(J);
  }
  // Translocation bookkeeping (Sec. III)
  const float xrel = bead ? (float)(a.ox - a.wall_x) + r.x : 0.f;
  const bool finite = isfinite(r.x) && isfinite(r.y) && isfinite(r.z) && isfinite(v.x) &&
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
  const int threads = ((a.N + 31) / 32) * 32;
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

__global__ void k_read_beads(const float4 *pos, const float4 *vel, int N, int ox, int oy, int oz,
                             double *dpos, double *dvel) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (dpos) {
    const float4 r = pos[i];
    dpos[3 * i] = (double)ox + (double)r.x;
    dpos[3 * i + 1] = (double)oy + (double)r.y;
    dpos[3 * i + 2] = (double)oz + (double)r.z;
  }
  if (dvel) {
    const float4 v = vel[i];
    dvel[3 * i] = v.x;
    dvel[3 * i + 1] = v.y;
    dvel[3 * i + 2] = v.z;
  }
}

cudaError_t launch_read_beads(const float4 *pos, const float4 *vel, int N, int ox, int oy, int oz,
                              double *dpos, double *dvel, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_read_beads<<<(N + 255) / 256, 256, 0, s>>>(pos, vel, N, ox, oy, oz, dpos, dvel);
  return cudaGetLastError();
}

cudaError_t launch_read_bead_aux(const float4 *ui, const float4 *J, int N, double *dui,
                                 double *dJ, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_read_beads<<<(N + 255) / 256, 256, 0, s>>>(ui, J, N, 0, 0, 0, dui, dJ);
  return cudaGetLastError();
}

}  // namespace lbmd
