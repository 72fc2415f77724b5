// lbmd_common.cuh -- device-side constants and helpers shared by the kernels of
// the coupled LB / polymer-MD step (arXiv:0710.1272, Sec. II).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lbmd_internal.h"

namespace lbmd {

// ---------------------------------------------------------------------------
// D3Q19 lattice (Sec. II: "the standard three-dimensional 19-speed lattice").
// Order: rest, +-x, +-y, +-z, then the twelve edge speeds; opposite directions
// are adjacent, so opp(p) = p + 1 for odd p and p - 1 for even p > 0.
// ---------------------------------------------------------------------------
constexpr int kQ = 19;
__host__ __device__ constexpr int cx(int p) {
  return (p == 1 || p == 7 || p == 9 || p == 11 || p == 13) ? 1
       : (p == 2 || p == 8 || p == 10 || p == 12 || p == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int p) {
  return (p == 3 || p == 7 || p == 10 || p == 15 || p == 17) ? 1
       : (p == 4 || p == 8 || p == 9 || p == 16 || p == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int p) {
  return (p == 5 || p == 11 || p == 14 || p == 15 || p == 18) ? 1
       : (p == 6 || p == 12 || p == 13 || p == 16 || p == 17) ? -1 : 0;
}
__host__ __device__ constexpr float wq(int p) {
  return p == 0 ? (1.0f / 3.0f) : (p <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}
__host__ __device__ constexpr int opp(int p) {
  return p == 0 ? 0 : ((p & 1) ? p + 1 : p - 1);
}

// ---------------------------------------------------------------------------
// Population storage: every type stores the deviation h_p = f_p - w_p rho0.
// ---------------------------------------------------------------------------
template <int S> struct Store;
template <> struct Store<LBMD_STORE_F32> {
  using T = float;
  static __device__ __forceinline__ float load(const T *p) { return __ldg(p); }
  static __device__ __forceinline__ float load_plain(const T *p) { return *p; }
  static __device__ __forceinline__ void store(T *p, float v) { *p = v; }
  static __device__ __forceinline__ void add(T *p, float v) { atomicAdd(p, v); }
};
template <> struct Store<LBMD_STORE_F16> {
  using T = __half;
  static __device__ __forceinline__ float load(const T *p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ float load_plain(const T *p) { return __half2float(*p); }
  static __device__ __forceinline__ void store(T *p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ void add(T *p, float v) { atomicAdd(p, __float2half_rn(v)); }
};
template <> struct Store<LBMD_STORE_BF16> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float load(const T *p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ float load_plain(const T *p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void store(T *p, float v) { *p = __float2bfloat16_rn(v); }
  static __device__ __forceinline__ void add(T *p, float v) { atomicAdd(p, __float2bfloat16_rn(v)); }
};

// ---------------------------------------------------------------------------
// Geometry helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_m1(int a, int n) { return a == 0 ? n - 1 : a - 1; }
__device__ __forceinline__ int wrap_p1(int a, int n) { return a == n - 1 ? 0 : a + 1; }
__device__ __forceinline__ int wrapi(int a, int n) {
  int m = a % n;
  return m < 0 ? m + n : m;
}

// Solid bit of node (x, y, z), coordinates already inside the box.
__device__ __forceinline__ bool solid_at(const uint32_t *__restrict__ bits, int wpr, int ny,
                                         int x, int y, int z) {
  return (__ldg(&bits[((size_t)z * ny + y) * wpr + (x >> 5)]) >> (x & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32 -> 64-bit multiplies, key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Also compiled for the host: the library's seeded chain start draws from it.
__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = mulhi32(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = mulhi32(0xCD9E8D57u, c.z);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

// Uniform in (0, 1) from the top 23 bits, exact in float: ((x >> 9) + 1/2) 2^-23.
__device__ __forceinline__ float uniform23(uint32_t x) {
  return (float)(x >> 9) * (1.0f / 8388608.0f) + (0.5f / 8388608.0f);
}

// Three standard normals for (bead, LB step, substep, stream): Box-Muller on
// the four uniforms of one Philox block.
__device__ __forceinline__ float3 gauss3(uint64_t seed, uint32_t bead, int64_t step,
                                         uint32_t substep, uint32_t stream) {
  U4 c{bead, (uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32),
       (substep & 0xFFu) | (stream << 8)};
  U4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u1 = uniform23(r.x), u2 = uniform23(r.y);
  const float u3 = uniform23(r.z), u4 = uniform23(r.w);
  const float r1 = sqrtf(-2.0f * logf(u1)), r2 = sqrtf(-2.0f * logf(u3));
  float s2, c2, s4, c4;
  sincospif(2.0f * u2, &s2, &c2);
  sincospif(2.0f * u4, &s4, &c4);
  return make_float3(r1 * c2, r1 * s2, r2 * c4);
}

}  // namespace lbmd
