// lb_noalloc.cu -- one D3Q19 stream-collide step on caller-owned populations
// that allocates nothing: no context, no workspace, no cudaMalloc.
//
// Who needs it: code that cannot allocate device memory -- a caller whose
// device memory is entirely handed out by another framework's pool, code that
// runs while another thread captures a CUDA graph in global capture mode
// (where cudaMalloc is prohibited), or a real-time loop that must not touch
// the allocator -- but does own two population buffers and wants the solvent
// update of the coupled step (no beads).
//
// The only global memory besides the caller's input and output is the
// geometry scratch (solid bitfield and per-tile "solid nearby" flags), kept in
// a fixed file-scope device array.  Its size limits the box: ny * nz *
// ceil(nx / 32) <= 2^20 tiles (for example 256^3).  Every call rebuilds the
// scratch on the device from the parameters, so no state carries over from the
// previous call.  All calls share that one array: calls that overlap on the GPU
// (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "lbmd_common.cuh"

namespace lbmd {
namespace {

constexpr int kNoAllocMaxTiles = 1 << 20;  // words of the bitfield = tiles
constexpr int kMaxDevices = 64;

// [kNoAllocMaxTiles] uint32 solid words, then [kNoAllocMaxTiles] uint8 flags
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocMaxTiles + kNoAllocMaxTiles / 4];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch per device

struct GeoParams {
  int nx, ny, nz, ntx;
  int wall_x, wall_t, pore_d, pore_y0, pore_z0, y_walls;
};

__device__ __forceinline__ bool solid_node(const GeoParams &q, int x, int y, int z) {
  if (q.y_walls && (y == 0 || y == q.ny - 1)) return true;
  if (q.wall_x < 0) return false;
  int dx = x - q.wall_x;
  if (dx < 0) dx += q.nx;
  if (dx >= q.wall_t) return false;
  const bool in_pore = q.pore_d > 0 && y >= q.pore_y0 && y < q.pore_y0 + q.pore_d &&
                       z >= q.pore_z0 && z < q.pore_z0 + q.pore_d;
  return !in_pore;
}

// One thread per bitfield word: the solid bits of 32 consecutive x.
__global__ void k_noalloc_bits(GeoParams q, uint32_t *bits) {
  const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nwords = (long long)q.ny * q.nz * q.ntx;
  if (w >= nwords) return;
  const int t = (int)(w % q.ntx);
  const long long row = w / q.ntx;
  const int y = (int)(row % q.ny), z = (int)(row / q.ny);
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const int x = t * 32 + b;
    if (x < q.nx && solid_node(q, x, y, z)) word |= 1u << b;
  }
  bits[w] = word;
}

__device__ __forceinline__ bool bit_at(const uint32_t *bits, const GeoParams &q, int x, int y, int z) {
  return (bits[((long long)z * q.ny + y) * q.ntx + (x >> 5)] >> (x & 31)) & 1u;
}

// One thread per tile: 1 if a solid node lies within one node of the tile.
__global__ void k_noalloc_tiles(GeoParams q, const uint32_t *bits, uint8_t *tiles) {
  const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ntiles = (long long)q.ny * q.nz * q.ntx;
  if (w >= ntiles) return;
  const int t = (int)(w % q.ntx);
  const long long row = w / q.ntx;
  const int y = (int)(row % q.ny), z = (int)(row / q.ny);
  const int x0 = t * 32, x1 = min(q.nx - 1, x0 + 31);
  const int xl = wrapi(x0 - 1, q.nx), xr = wrapi(x1 + 1, q.nx);
  uint8_t near = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = wrapi(y + dy, q.ny), zz = wrapi(z + dz, q.nz);
      // the tile's own 32 cells (bits beyond nx are zero), then its two x-neighbours
      if (bits[((long long)zz * q.ny + yy) * q.ntx + t] != 0u || bit_at(bits, q, xl, yy, zz) ||
          bit_at(bits, q, xr, yy, zz))
        near = 1;
    }
  tiles[w] = near;
}

// Collide-then-push form of Eq. 5 on absolute populations:
//   f*_p(x) = f_p - (f_p - f_eq,p(rho, u)) / tau + S_p(g),
//   f_p(x + c_p, t+1) = f*_p(x) if x + c_p is fluid, else f_opp(p)(x, t+1) = f*_p(x).
// Solid nodes of the output are set to zero.
template <int FORCING>
__global__ void __launch_bounds__(256) k_noalloc_step(GeoParams q, float omega, float rho0,
                                                      float gx, float gy, float gz,
                                                      const uint32_t *__restrict__ bits,
                                                      const uint8_t *__restrict__ tiles,
                                                      const float *__restrict__ fin,
                                                      float *__restrict__ fout) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= q.nx || y >= q.ny) return;
  const long long V = (long long)q.nx * q.ny * q.nz;
  const long long self = ((long long)z * q.ny + y) * q.nx + x;
  const bool near = tiles[((long long)z * q.ny + y) * q.ntx + (x >> 5)] != 0;
  if (near && bit_at(bits, q, x, y, z)) {
#pragma unroll
    for (int p = 0; p < kQ; ++p) fout[p * V + self] = 0.f;
    return;
  }
  float f[kQ];
  float rho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int p = 0; p < kQ; ++p) {
    f[p] = fin[p * V + self];
    rho += f[p];
    jx += cx(p) * f[p];
    jy += cy(p) * f[p];
    jz += cz(p) * f[p];
  }
  if (FORCING == LBMD_FORCING_GUO) {
    jx += 0.5f * gx;
    jy += 0.5f * gy;
    jz += 0.5f * gz;
  }
  const float ux = jx / rho, uy = jy / rho, uz = jz / rho;
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  const float gu = gx * ux + gy * uy + gz * uz;
  const int nx = q.nx, ny = q.ny, nz = q.nz;
#pragma unroll
  for (int p = 0; p < kQ; ++p) {
    const float cu = cx(p) * ux + cy(p) * uy + cz(p) * uz;
    const float feq = wq(p) * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - usq15);
    const float cg = cx(p) * gx + cy(p) * gy + cz(p) * gz;
    const float src = FORCING == LBMD_FORCING_GUO
                          ? (1.0f - 0.5f * omega) * wq(p) * (3.0f * (cg - gu) + 9.0f * cu * cg)
                          : 3.0f * wq(p) * cg;
    const float fs = f[p] - omega * (f[p] - feq) + src;
    const int xd = cx(p) == 1 ? wrap_p1(x, nx) : (cx(p) == -1 ? wrap_m1(x, nx) : x);
    const int yd = cy(p) == 1 ? wrap_p1(y, ny) : (cy(p) == -1 ? wrap_m1(y, ny) : y);
    const int zd = cz(p) == 1 ? wrap_p1(z, nz) : (cz(p) == -1 ? wrap_m1(z, nz) : z);
    if (p != 0 && near && bit_at(bits, q, xd, yd, zd))
      fout[opp(p) * V + self] = fs;
    else
      fout[p * V + ((long long)zd * ny + yd) * nx + xd] = fs;
  }
}

// Device address of the scratch array on the current device, looked up once.
cudaError_t scratch_address(uint32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = (uint32_t *)g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lbmd

using namespace lbmd;

extern "C" int lbmd_lb_step_noalloc(const lbmd_params *p, const float *f_in, float *f_out,
                                    void *cuda_stream) {
  if (!p || !f_in || !f_out) return LBMD_EINVAL;
  if (f_in == f_out) return LBMD_EINVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nz > 65535) return LBMD_EINVAL;
  if (!(p->tau > 0.5) || !(p->rho0 > 0)) return LBMD_EINVAL;
  // FP32 solvent only: no bead state to keep, no step counter for the noise
  if (p->storage != LBMD_STORE_F32 || p->n_beads != 0 || p->kT_fluid != 0.0) return LBMD_EUNSUPPORTED;
  if (p->forcing != LBMD_FORCING_PAPER && p->forcing != LBMD_FORCING_GUO) return LBMD_EINVAL;
  if (p->wall_x < -1 || p->wall_x >= p->nx) return LBMD_EINVAL;
  if (p->y_walls != 0 && p->y_walls != 1) return LBMD_EINVAL;
  GeoParams q;
  q.nx = p->nx;
  q.ny = p->ny;
  q.nz = p->nz;
  q.ntx = (p->nx + 31) / 32;
  q.wall_x = p->wall_x;
  q.wall_t = p->wall_thickness;
  q.pore_d = p->pore_d;
  q.y_walls = p->y_walls;
  if (p->wall_x >= 0) {
    if (p->wall_thickness < 1 || p->wall_thickness >= p->nx) return LBMD_EINVAL;
    if (p->pore_d < 0 || p->pore_d > p->ny || p->pore_d > p->nz) return LBMD_EINVAL;
    q.pore_y0 = p->pore_y0 >= 0 ? p->pore_y0 : (p->ny - p->pore_d) / 2;
    q.pore_z0 = p->pore_z0 >= 0 ? p->pore_z0 : (p->nz - p->pore_d) / 2;
    if (q.pore_y0 + p->pore_d > p->ny || q.pore_z0 + p->pore_d > p->nz) return LBMD_EINVAL;
  } else {
    q.pore_y0 = q.pore_z0 = 0;
  }
  const long long tiles = (long long)q.ny * q.nz * q.ntx;
  if (tiles > kNoAllocMaxTiles) return LBMD_ESIZE;  // box larger than the fixed scratch
  if ((q.ny + 7) / 8 > 65535) return LBMD_EINVAL;   // grid y of the step kernel (ny <= 524280)

  uint32_t *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return LBMD_ECUDA;
  uint32_t *bits = scratch;
  uint8_t *tile = (uint8_t *)(scratch + kNoAllocMaxTiles);
  // launched with cudaLaunchKernelEx, whose return value is the status of
  // that launch alone (not an error left behind by unrelated earlier work)
  cudaLaunchConfig_t cfg = {};
  cfg.stream = (cudaStream_t)cuda_stream;
  cfg.blockDim = dim3(256);
  cfg.gridDim = dim3((unsigned)((tiles + 255) / 256));
  if (cudaLaunchKernelEx(&cfg, k_noalloc_bits, q, bits) != cudaSuccess) return LBMD_ECUDA;
  if (cudaLaunchKernelEx(&cfg, k_noalloc_tiles, q, (const uint32_t *)bits, tile) != cudaSuccess)
    return LBMD_ECUDA;
  cfg.blockDim = dim3(32, 8);
  cfg.gridDim = dim3(q.ntx, (q.ny + 7) / 8, q.nz);
  const float omega = (float)(1.0 / p->tau), rho0 = (float)p->rho0;
  const float gx = (float)p->body_force[0], gy = (float)p->body_force[1], gz = (float)p->body_force[2];
  const uint32_t *cbits = bits;
  const uint8_t *ctile = tile;
  const cudaError_t e =
      p->forcing == LBMD_FORCING_GUO
          ? cudaLaunchKernelEx(&cfg, k_noalloc_step<LBMD_FORCING_GUO>, q, omega, rho0, gx, gy, gz, cbits,
                               ctile, f_in, f_out)
          : cudaLaunchKernelEx(&cfg, k_noalloc_step<LBMD_FORCING_PAPER>, q, omega, rho0, gx, gy, gz, cbits,
                               ctile, f_in, f_out);
  return e == cudaSuccess ? LBMD_OK : LBMD_ECUDA;
}
