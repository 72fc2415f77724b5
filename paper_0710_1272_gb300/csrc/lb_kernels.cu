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

// 16-bit storage: one thread per pair of x-adjacent nodes (pair_node).  A
// warp covers 64 nodes of one row, i.e. two 32-node tiles.  Register budget:
// 64 (four blocks per SM) for the benchmark's zero-force collision, 80 (three)
// for the forced variants, which would spill at 64.
template <typename T2, int FORCING>
__global__ void __launch_bounds__(32 * kRowsPerBlock, FORCING == kForcingNone ? 4 : 3)
    k_stream_collide_pair(LbGeom g, LbPhys ph, const uint32_t *__restrict__ src,
                          uint32_t *__restrict__ dst, DevStatus *bump) {
  const int xw = blockIdx.x * 32 + threadIdx.x;  // word: nodes 2 xw, 2 xw + 1
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = blockIdx.z;
  if (bump != nullptr && xw == 0 && y == 0 && z == 0) bump->step += 1;
  if (xw >= (g.nx >> 1) || y >= g.ny) return;
  pair_node<T2, FORCING>(g, ph, src, dst, xw, y, z, tile_is_near(g, 2 * xw, y, z));
}

template <typename T2>
static cudaError_t lb_launch_pair(const LbGeom &g, const LbPhys &ph, const void *src, void *dst,
                                  DevStatus *bump, cudaStream_t s) {
  dim3 block(32, kRowsPerBlock);
  dim3 grid((g.nx / 2 + 31) / 32, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, g.nz);
  const uint32_t *a = (const uint32_t *)src;
  uint32_t *b = (uint32_t *)dst;
  if (ph.g[0] == 0.f && ph.g[1] == 0.f && ph.g[2] == 0.f)
    k_stream_collide_pair<T2, kForcingNone><<<grid, block, 0, s>>>(g, ph, a, b, bump);
  else if (ph.forcing == LBMD_FORCING_GUO)
    k_stream_collide_pair<T2, LBMD_FORCING_GUO><<<grid, block, 0, s>>>(g, ph, a, b, bump);
  else
    k_stream_collide_pair<T2, LBMD_FORCING_PAPER><<<grid, block, 0, s>>>(g, ph, a, b, bump);
  return cudaGetLastError();
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
  const bool small = (long long)kQ * g.Vp < 0x7fffffffLL;
  // 16-bit storage with an even row length: two nodes per thread
  if (small && g.nx % 2 == 0) {
    if (S == LBMD_STORE_F16) return lb_launch_pair<__half2>(g, ph, src, dst, bump, s);
    if (S == LBMD_STORE_BF16) return lb_launch_pair<__nv_bfloat162>(g, ph, src, dst, bump, s);
  }
  if (small) return lb_launch<S, int>(g, ph, src, dst, bump, s);
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
// Initial (rho, u) of node (x, y): entry c of the given fields (component
// stride ustride), else rho0 and the Taylor-Green flow of amplitude tg_amp.
__device__ __forceinline__ void fields_at(int x, int y, size_t c, long long ustride,
                                          const LbGeom &g, float rho0, const float *rho,
                                          const float *u, float tg_amp, float &r, float &ux,
                                          float &uy, float &uz) {
  r = rho ? rho[c] : rho0;
  if (u) {
    ux = u[c];
    uy = u[(size_t)ustride + c];
    uz = u[2 * (size_t)ustride + c];
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

__device__ __forceinline__ void init_fields_at(int x, int y, int z, const LbGeom &g, float rho0,
                                               const float *rho, const float *u, float tg_amp,
                                               float &r, float &ux, float &uy, float &uz) {
  fields_at(x, y, ((size_t)z * g.ny + y) * g.nx + x, g.V, g, rho0, rho, u, tg_amp, r, ux, uy, uz);
}

// f_eq,p - w_p rho0 (Eq. 6), every operation rounded explicitly so that the
// pull and in-place initialisations produce the same bits.
__device__ __forceinline__ float feq_dev(int p, float r, float rho0, float ux, float uy, float uz) {
  const float cu = cx(p) * ux + cy(p) * uy + cz(p) * uz;  // +-u_a sums
  const float usq = fmaf(uz, uz, fmaf(uy, uy, __fmul_rn(ux, ux)));
  const float poly = fmaf(-1.5f, usq, fmaf(__fmul_rn(4.5f, cu), cu, __fmul_rn(3.0f, cu)));
  return __fmul_rn(wq(p), fmaf(r, poly, r - rho0));
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

// In-place streaming starts from the pre-collision state itself, stored
// locally (kPopAALocal): h_q(x, 0) = f_eq,q(rho(x), u(x)) - w_q rho0 at fluid
// nodes, zero at solid nodes.  One z-slab per launch; rho / u are the slab's.
template <int S>
__global__ void k_init_local(LbGeom g, float rho0, const float *rho, const float *u,
                             long long ustride, float tg_amp, int z0,
                             typename Store<S>::T *__restrict__ dst) {
  using St = Store<S>;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = z0 + blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const size_t self = ((size_t)z * g.ny + y) * g.nx + x;
  const size_t Vp = (size_t)g.Vp;
  float r = rho0, ux = 0.f, uy = 0.f, uz = 0.f;
  const bool solid = solid_at(g.solid, g.ntx, g.ny, x, y, z);
  if (!solid)
    fields_at(x, y, ((size_t)blockIdx.z * g.ny + y) * g.nx + x, ustride, g, rho0, rho, u, tg_amp, r,
              ux, uy, uz);
#pragma unroll
  for (int q = 0; q < kQ; ++q) St::store(dst + q * Vp + self, solid ? 0.f : feq_dev(q, r, rho0, ux, uy, uz));
}

cudaError_t launch_init_local(int storage, const LbGeom &g, float rho0, const float *rho,
                              const float *u, long long ustride, float tg_amp, long long z0,
                              long long nzc, void *dst, cudaStream_t s) {
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, (unsigned)nzc);
  switch (storage) {
    case LBMD_STORE_F32:
      k_init_local<LBMD_STORE_F32><<<grid, block, 0, s>>>(g, rho0, rho, u, ustride, tg_amp, (int)z0, (float *)dst);
      break;
    case LBMD_STORE_F16:
      k_init_local<LBMD_STORE_F16><<<grid, block, 0, s>>>(g, rho0, rho, u, ustride, tg_amp, (int)z0, (__half *)dst);
      break;
    case LBMD_STORE_BF16:
      k_init_local<LBMD_STORE_BF16><<<grid, block, 0, s>>>(g, rho0, rho, u, ustride, tg_amp, (int)z0, (__nv_bfloat16 *)dst);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Read-outs over the z-slab [z0, z0 + nzc): moments (Eqs. 7-8) and the
// pre-collision populations, fetched for the layout `mode` (kPop*).  Solid
// nodes read zero.
// ---------------------------------------------------------------------------
template <int S>
__global__ void k_read_moments(LbGeom g, LbPhys ph, const typename Store<S>::T *__restrict__ src,
                               int mode, int z0, float *rho, float *u, long long ustride) {
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
  fetch19<S>(g, src, x, y, z, mode, h);
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
                              int mode, int z0, float *f, long long fstride) {
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
  fetch19<S>(g, src, x, y, z, mode, h);
#pragma unroll
  for (int p = 0; p < kQ; ++p) f[p * fstride + o] = __fadd_rn(__fmul_rn(wq(p), rho0), h[p]);
}

cudaError_t launch_read_moments(int storage, const LbGeom &g, const LbPhys &ph, const void *src,
                                int mode, long long z0, long long nzc, float *rho, float *u,
                                long long ustride, cudaStream_t s) {
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, (unsigned)nzc);
  switch (storage) {
    case LBMD_STORE_F32:
      k_read_moments<LBMD_STORE_F32><<<grid, block, 0, s>>>(g, ph, (const float *)src, mode, (int)z0, rho, u, ustride);
      break;
    case LBMD_STORE_F16:
      k_read_moments<LBMD_STORE_F16><<<grid, block, 0, s>>>(g, ph, (const __half *)src, mode, (int)z0, rho, u, ustride);
      break;
    case LBMD_STORE_BF16:
      k_read_moments<LBMD_STORE_BF16><<<grid, block, 0, s>>>(g, ph, (const __nv_bfloat16 *)src, mode, (int)z0, rho, u, ustride);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_read_pulled(int storage, const LbGeom &g, float rho0, const void *src,
                               int mode, long long z0, long long nzc, float *f,
                               long long fstride, cudaStream_t s) {
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, (unsigned)nzc);
  switch (storage) {
    case LBMD_STORE_F32:
      k_read_pulled<LBMD_STORE_F32><<<grid, block, 0, s>>>(g, rho0, (const float *)src, mode, (int)z0, f, fstride);
      break;
    case LBMD_STORE_F16:
      k_read_pulled<LBMD_STORE_F16><<<grid, block, 0, s>>>(g, rho0, (const __half *)src, mode, (int)z0, f, fstride);
      break;
    case LBMD_STORE_BF16:
      k_read_pulled<LBMD_STORE_BF16><<<grid, block, 0, s>>>(g, rho0, (const __nv_bfloat16 *)src, mode, (int)z0, f, fstride);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbmd
