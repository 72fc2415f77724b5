// lb_kernels.cu -- D3Q19 BGK stream-collide (Eq. 5 with the Eq. 6 equilibrium
// and the body-force source), population initialisation and field read-outs.
//
// Layout: structure of arrays, h[p][z][y][x] with population stride Vp, every
// entry the deviation h = f - w_p rho0 in the storage type.  One thread per
// node; a warp covers 32 consecutive x of one (y, z) row so that every one of
// the 19 loads and 19 stores of a warp is a contiguous 128-byte (fp32) or
// 64-byte (16-bit) segment; the loads for c_x = +-1 are shifted by one element
// and are served from L1/L2 for the neighbouring warp's sector.
#include "lb_collide.cuh"

namespace lbmd {

// Six 256-thread blocks per SM (40 registers): the occupancy that measured
// fastest for this kernel; it is HBM-bound and needs the loads of many warps
// in flight.
template <int S, int FORCING, typename I>
__global__ void __launch_bounds__(32 * kRowsPerBlock, 6)
    k_stream_collide(LbGeom g, LbPhys ph, const typename Store<S>::T *__restrict__ src,
                     typename Store<S>::T *__restrict__ dst, DevStatus *bump) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = blockIdx.z;
  if (bump != nullptr && x == 0 && y == 0 && z == 0) bump->step += 1;
  if (x >= g.nx || y >= g.ny) return;
  stream_collide_node<S, FORCING, I>(g, ph, src, dst, x, y, z, tile_is_near(g, x, y, z));
}

// Ensemble stream-collide: a persistent grid over the tiles of every live
// realisation.  A block takes `claim` consecutive tiles at a time from a
// global counter, so blocks that become resident late (after the MD blocks of
// the same step) simply take fewer tiles.  A tile is 32 x ROWS consecutive
// nodes of one z-plane, so a warp reads and writes one contiguous run of
// every population whatever the box width (no idle lanes for widths that are
// not a multiple of 32).  A warp takes the bounce-back checks if any of its
// nodes needs them.  WARPS is the occupancy the register budget is sized for:
// 48 warps per SM (40 registers, a little spilling) or 32 (64 registers,
// none); population offsets are 32-bit.
template <int S, int FORCING, int ROWS, int WARPS>
__global__ void __launch_bounds__(32 * ROWS, WARPS / ROWS)
    k_ens_stream_collide(const EnsLb *__restrict__ lbd, const EnsTile *__restrict__ tiles,
                         const int *__restrict__ n_tiles, int *__restrict__ counter,
                         const int *__restrict__ live, int cur, int claim) {
  using T = typename Store<S>::T;
  // two claim slots used alternately: a slot is rewritten two claims later,
  // after every thread has passed the barrier that follows its read
  __shared__ int s_first[2];
  const int n = *n_tiles;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int slot = 0;; slot ^= 1) {
    if (tid == 0) s_first[slot] = atomicAdd(counter, claim);
    __syncthreads();
    const int first = s_first[slot];
    if (first >= n) return;
    const int last = min(first + claim, n);
    for (int t = first; t < last; ++t) {
      const int4 w = __ldg(reinterpret_cast<const int4 *>(tiles) + t);  // (m, z, r0, -)
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
      // node of this thread: row-major index r in the plane, its row by a
      // float reciprocal with a one-step correction (exact for nx * ny < 2^22)
      const int plane = d.nx * d.ny;
      const int r = w.z + tid;
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
      const bool near = __any_sync(0xffffffffu, active && tile_is_near(g, x, y, w.y));
      const T *src = (const T *)(cur ? d.pop[1] : d.pop[0]);
      T *dst = (T *)(cur ? d.pop[0] : d.pop[1]);
      if (active) stream_collide_node<S, FORCING, int>(g, ph, src, dst, x, y, w.y, near);
    }
  }
}

template <int S, typename I>
static cudaError_t lb_launch(const LbGeom &g, const LbPhys &ph, const void *src, void *dst,
                             DevStatus *bump, cudaStream_t s) {
  using T = typename Store<S>::T;
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, g.nz);
  if (ph.g[0] == 0.f && ph.g[1] == 0.f && ph.g[2] == 0.f)
    k_stream_collide<S, kForcingNone, I><<<grid, block, 0, s>>>(g, ph, (const T *)src, (T *)dst, bump);
  else if (ph.forcing == LBMD_FORCING_GUO)
    k_stream_collide<S, LBMD_FORCING_GUO, I><<<grid, block, 0, s>>>(g, ph, (const T *)src, (T *)dst, bump);
  else
    k_stream_collide<S, LBMD_FORCING_PAPER, I><<<grid, block, 0, s>>>(g, ph, (const T *)src, (T *)dst, bump);
  return cudaGetLastError();
}

template <int S>
static cudaError_t lb_launch(const LbGeom &g, const LbPhys &ph, const void *src, void *dst,
                             DevStatus *bump, cudaStream_t s) {
  // 32-bit offsets when every population index fits
  if ((long long)kQ * g.Vp < 0x7fffffffLL) return lb_launch<S, int>(g, ph, src, dst, bump, s);
  return lb_launch<S, size_t>(g, ph, src, dst, bump, s);
}

cudaError_t launch_lb_stream_collide(int storage, const LbGeom &g, const LbPhys &ph,
                                     const void *src, void *dst, DevStatus *bump,
                                     cudaStream_t s) {
  switch (storage) {
    case LBMD_STORE_F32: return lb_launch<LBMD_STORE_F32>(g, ph, src, dst, bump, s);
    case LBMD_STORE_F16: return lb_launch<LBMD_STORE_F16>(g, ph, src, dst, bump, s);
    case LBMD_STORE_BF16: return lb_launch<LBMD_STORE_BF16>(g, ph, src, dst, bump, s);
  }
  return cudaErrorInvalidValue;
}

template <int S, int FORCING, int ROWS, int WARPS>
static cudaError_t ens_lb_launch(int claim, int grid, const EnsLb *lbd, const EnsTile *tiles,
                                 const int *n_tiles, int *counter, const int *live, int cur,
                                 cudaStream_t s) {
  k_ens_stream_collide<S, FORCING, ROWS, WARPS><<<grid, dim3(32, ROWS), 0, s>>>(
      lbd, tiles, n_tiles, counter, live, cur, claim);
  return cudaGetLastError();
}

template <int S, int FORCING, int ROWS, int WARPS>
static int ens_lb_occupancy() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_stream_collide<S, FORCING, ROWS, WARPS>,
                                                    32 * ROWS, 0) != cudaSuccess)
    return 0;
  return n;
}

// Dispatch on (storage, forcing, rows, warps per SM) to one instantiation.
struct EnsLbFns {
  cudaError_t (*launch)(int, int, const EnsLb *, const EnsTile *, const int *, int *,
                        const int *, int, cudaStream_t);
  int (*occupancy)();
};
template <int S, int F, int R>
static EnsLbFns ens_fns_warps(int warps) {
  if (warps == 32) return {&ens_lb_launch<S, F, R, 32>, &ens_lb_occupancy<S, F, R, 32>};
  return {&ens_lb_launch<S, F, R, 48>, &ens_lb_occupancy<S, F, R, 48>};
}
template <int S, int F>
static EnsLbFns ens_fns_rows(int rows, int warps) {
  if (rows == 4) return ens_fns_warps<S, F, 4>(warps);
  if (rows == 16) return ens_fns_warps<S, F, 16>(warps);
  return ens_fns_warps<S, F, 8>(warps);
}
template <int S>
static EnsLbFns ens_fns_store(int forcing, int rows, int warps) {
  if (forcing == kForcingNone) return ens_fns_rows<S, kForcingNone>(rows, warps);
  if (forcing == LBMD_FORCING_GUO) return ens_fns_rows<S, LBMD_FORCING_GUO>(rows, warps);
  return ens_fns_rows<S, LBMD_FORCING_PAPER>(rows, warps);
}
static EnsLbFns ens_fns(int storage, int forcing, int rows, int warps) {
  if (storage == LBMD_STORE_F16) return ens_fns_store<LBMD_STORE_F16>(forcing, rows, warps);
  if (storage == LBMD_STORE_BF16) return ens_fns_store<LBMD_STORE_BF16>(forcing, rows, warps);
  return ens_fns_store<LBMD_STORE_F32>(forcing, rows, warps);
}

cudaError_t launch_ens_stream_collide(int storage, int forcing, int rows, int warps, int claim,
                                      int grid, const EnsLb *lbd, const EnsTile *tiles,
                                      const int *n_tiles, int *counter, const int *live, int cur,
                                      cudaStream_t s) {
  if (storage < LBMD_STORE_F32 || storage > LBMD_STORE_BF16) return cudaErrorInvalidValue;
  return ens_fns(storage, forcing, rows, warps).launch(claim, grid, lbd, tiles, n_tiles, counter,
                                                       live, cur, s);
}

int ens_lb_blocks_per_sm(int storage, int forcing, int rows, int warps) {
  return ens_fns(storage, forcing, rows, warps).occupancy();
}

// Link mask of every node: bit 0 if the node is solid, bit p (1..18) if its
// pull source x - c_p (periodic wrap) is solid.
__global__ void k_link_mask(LbGeom g, uint32_t *__restrict__ mask) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  uint32_t bb = solid_at(g.solid, g.ntx, g.ny, x, y, z) ? 1u : 0u;
#pragma unroll
  for (int p = 1; p < kQ; ++p) {
    const int sx = wrapi(x - cx(p), g.nx), sy = wrapi(y - cy(p), g.ny), sz = wrapi(z - cz(p), g.nz);
    if (solid_at(g.solid, g.ntx, g.ny, sx, sy, sz)) bb |= 1u << p;
  }
  mask[((size_t)z * g.ny + y) * g.nx + x] = bb;
}

cudaError_t launch_link_mask(const LbGeom &g, uint32_t *mask, cudaStream_t s) {
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, g.nz);
  k_link_mask<<<grid, block, 0, s>>>(g, mask);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Initialisation: the pre-collision state f(x, 0) = f_eq(rho(x), u(x)) must be
// what the first pull produces, so the stored post-collision buffer holds
//   h*_q(y) = f_eq,q(y + c_q) - w_q rho0     if y + c_q is fluid,
//   h*_q(y) = f_eq,opp(q)(y) - w_q rho0      otherwise (bounce-back source),
// at fluid nodes y, and zero at solid nodes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void init_fields_at(int x, int y, int z, const LbGeom &g, float rho0,
                                               const float *rho, const float *u, float tg_amp,
                                               float &r, float &ux, float &uy, float &uz) {
  const size_t c = ((size_t)z * g.ny + y) * g.nx + x;
  r = rho ? rho[c] : rho0;
  if (u) {
    ux = u[c];
    uy = u[(size_t)g.V + c];
    uz = u[2 * (size_t)g.V + c];
  } else if (tg_amp != 0.f) {
    float sx, cxv, sy, cyv;
    sincospif(2.0f * (float)x / (float)g.nx, &sx, &cxv);
    sincospif(2.0f * (float)y / (float)g.ny, &sy, &cyv);
    ux = tg_amp * sx * cyv;
    uy = -tg_amp * cxv * sy;
    uz = 0.f;
  } else {
    ux = uy = uz = 0.f;
  }
}

__device__ __forceinline__ float feq_dev(int p, float r, float rho0, float ux, float uy, float uz) {
  const float cu = cx(p) * ux + cy(p) * uy + cz(p) * uz;
  const float usq = ux * ux + uy * uy + uz * uz;
  return wq(p) * ((r - rho0) + r * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
}

template <int S>
__global__ void k_init(LbGeom g, float rho0, const float *rho, const float *u, float tg_amp,
                       typename Store<S>::T *__restrict__ dst) {
  using St = Store<S>;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const size_t self = ((size_t)z * g.ny + y) * g.nx + x;
  const size_t Vp = (size_t)g.Vp;
  if (solid_at(g.solid, g.ntx, g.ny, x, y, z)) {
#pragma unroll
    for (int q = 0; q < kQ; ++q) St::store(dst + q * Vp + self, 0.f);
    return;
  }
  float r0, ux0, uy0, uz0;
  init_fields_at(x, y, z, g, rho0, rho, u, tg_amp, r0, ux0, uy0, uz0);
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int tx = wrapi(x + cx(q), g.nx), ty = wrapi(y + cy(q), g.ny), tz = wrapi(z + cz(q), g.nz);
    float v;
    if (q != 0 && !solid_at(g.solid, g.ntx, g.ny, tx, ty, tz)) {
      float r, ux, uy, uz;
      init_fields_at(tx, ty, tz, g, rho0, rho, u, tg_amp, r, ux, uy, uz);
      v = feq_dev(q, r, rho0, ux, uy, uz);
    } else if (q == 0) {
      v = feq_dev(0, r0, rho0, ux0, uy0, uz0);
    } else {
      v = feq_dev(opp(q), r0, rho0, ux0, uy0, uz0);
    }
    St::store(dst + q * Vp + self, v);
  }
}

cudaError_t launch_init_populations(int storage, const LbGeom &g, float rho0, const float *rho,
                                    const float *u, float tg_amp, void *dst, cudaStream_t s) {
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, g.nz);
  switch (storage) {
    case LBMD_STORE_F32:
      k_init<LBMD_STORE_F32><<<grid, block, 0, s>>>(g, rho0, rho, u, tg_amp, (float *)dst);
      break;
    case LBMD_STORE_F16:
      k_init<LBMD_STORE_F16><<<grid, block, 0, s>>>(g, rho0, rho, u, tg_amp, (__half *)dst);
      break;
    case LBMD_STORE_BF16:
      k_init<LBMD_STORE_BF16><<<grid, block, 0, s>>>(g, rho0, rho, u, tg_amp, (__nv_bfloat16 *)dst);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Read-outs over the z-slab [z0, z0 + nzc): moments (Eqs. 7-8) and the pulled
// pre-collision populations.  Solid nodes read zero.
// ---------------------------------------------------------------------------
template <int S>
__global__ void k_read_moments(LbGeom g, LbPhys ph, const typename Store<S>::T *__restrict__ src,
                               int z0, float *rho, float *u, long long ustride) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = z0 + blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const size_t o = ((size_t)blockIdx.z * g.ny + y) * g.nx + x;
  if (solid_at(g.solid, g.ntx, g.ny, x, y, z)) {
    if (rho) rho[o] = 0.f;
    if (u) u[o] = u[ustride + o] = u[2 * ustride + o] = 0.f;
    return;
  }
  float h[kQ];
  pull19<S, true>(g, src, x, y, z, h);
  float drho, jx, jy, jz;
  moments19(h, drho, jx, jy, jz);
  const float r = ph.rho0 + drho;
  if (ph.forcing == LBMD_FORCING_GUO) {
    jx += 0.5f * ph.g[0];
    jy += 0.5f * ph.g[1];
    jz += 0.5f * ph.g[2];
  }
  if (rho) rho[o] = r;
  if (u) {
    u[o] = jx / r;
    u[ustride + o] = jy / r;
    u[2 * ustride + o] = jz / r;
  }
}

template <int S>
__global__ void k_read_pulled(LbGeom g, float rho0, const typename Store<S>::T *__restrict__ src,
                              int z0, float *f, long long fstride) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = z0 + blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const size_t o = ((size_t)blockIdx.z * g.ny + y) * g.nx + x;
  if (solid_at(g.solid, g.ntx, g.ny, x, y, z)) {
#pragma unroll
    for (int p = 0; p < kQ; ++p) f[p * fstride + o] = 0.f;
    return;
  }
  float h[kQ];
  pull19<S, true>(g, src, x, y, z, h);
#pragma unroll
  for (int p = 0; p < kQ; ++p) f[p * fstride + o] = wq(p) * rho0 + h[p];
}

cudaError_t launch_read_moments(int storage, const LbGeom &g, const LbPhys &ph, const void *src,
                                long long z0, long long nzc, float *rho, float *u,
                                long long ustride, cudaStream_t s) {
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, (unsigned)nzc);
  switch (storage) {
    case LBMD_STORE_F32:
      k_read_moments<LBMD_STORE_F32><<<grid, block, 0, s>>>(g, ph, (const float *)src, (int)z0, rho, u, ustride);
      break;
    case LBMD_STORE_F16:
      k_read_moments<LBMD_STORE_F16><<<grid, block, 0, s>>>(g, ph, (const __half *)src, (int)z0, rho, u, ustride);
      break;
    case LBMD_STORE_BF16:
      k_read_moments<LBMD_STORE_BF16><<<grid, block, 0, s>>>(g, ph, (const __nv_bfloat16 *)src, (int)z0, rho, u, ustride);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_read_pulled(int storage, const LbGeom &g, float rho0, const void *src,
                               long long z0, long long nzc, float *f, long long fstride,
                               cudaStream_t s) {
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, (unsigned)nzc);
  switch (storage) {
    case LBMD_STORE_F32:
      k_read_pulled<LBMD_STORE_F32><<<grid, block, 0, s>>>(g, rho0, (const float *)src, (int)z0, f, fstride);
      break;
    case LBMD_STORE_F16:
      k_read_pulled<LBMD_STORE_F16><<<grid, block, 0, s>>>(g, rho0, (const __half *)src, (int)z0, f, fstride);
      break;
    case LBMD_STORE_BF16:
      k_read_pulled<LBMD_STORE_BF16><<<grid, block, 0, s>>>(g, rho0, (const __nv_bfloat16 *)src, (int)z0, f, fstride);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbmd
