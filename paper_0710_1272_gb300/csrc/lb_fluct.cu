// lb_fluct.cu -- the stream-collide with the thermal source F_p of Eq. 5
// (fluctuating LB), in its own translation unit: the same node update as
// k_stream_collide (pull) or k_aa_stream_collide (in place) plus fifteen
// Philox normals per node.
#include <cmath>

#include "lb_aa.cuh"

namespace lbmd {

template <int S, int FORCING, typename I>
__global__ void __launch_bounds__(32 * kRowsPerBlock)
    k_stream_collide_fluct(LbGeom g, LbPhys ph, const typename Store<S>::T *__restrict__ src,
                           typename Store<S>::T *__restrict__ dst) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kRowsPerBlock + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  stream_collide_node<S, FORCING, I, true>(g, ph, src, dst, x, y, z, tile_is_near(g, x, y, z));
}

template <int S, typename I>
static cudaError_t fluct_launch(const LbGeom &g, const LbPhys &ph, const void *src, void *dst,
                                cudaStream_t s) {
  using T = typename Store<S>::T;
  dim3 block(32, kRowsPerBlock);
  dim3 grid(g.ntx, (g.ny + kRowsPerBlock - 1) / kRowsPerBlock, g.nz);
  if (ph.g[0] == 0.f && ph.g[1] == 0.f && ph.g[2] == 0.f)
    k_stream_collide_fluct<S, kForcingNone, I><<<grid, block, 0, s>>>(g, ph, (const T *)src, (T *)dst);
  else if (ph.forcing == LBMD_FORCING_GUO)
    k_stream_collide_fluct<S, LBMD_FORCING_GUO, I><<<grid, block, 0, s>>>(g, ph, (const T *)src, (T *)dst);
  else
    k_stream_collide_fluct<S, LBMD_FORCING_PAPER, I><<<grid, block, 0, s>>>(g, ph, (const T *)src, (T *)dst);
  return cudaGetLastError();
}

template <int S>
static cudaError_t fluct_launch(const LbGeom &g, const LbPhys &ph, const void *src, void *dst,
                                cudaStream_t s) {
  if ((long long)kQ * g.Vp < 0x7fffffffLL) return fluct_launch<S, int>(g, ph, src, dst, s);
  return fluct_launch<S, size_t>(g, ph, src, dst, s);
}

cudaError_t launch_lb_stream_collide_fluct(int storage, const LbGeom &g, const LbPhys &ph,
                                           const void *src, void *dst, cudaStream_t s) {
  switch (storage) {
    case LBMD_STORE_F32: return fluct_launch<LBMD_STORE_F32>(g, ph, src, dst, s);
    case LBMD_STORE_F16: return fluct_launch<LBMD_STORE_F16>(g, ph, src, dst, s);
    case LBMD_STORE_BF16: return fluct_launch<LBMD_STORE_BF16>(g, ph, src, dst, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_lb_aa_fluct(int storage, const LbGeom &g, const LbPhys &ph, void *buf,
                               int odd, cudaStream_t s) {
  return aa_launch_storage<true>(storage, g, ph, buf, odd, nullptr, s);
}

void fluct_amplitudes(double kT, double tau, float amp[15]) {
  const double g1 = 1.0 - 1.0 / tau;
  for (int k = 4; k < kQ; ++k) {
    double b = 0.0;  // b_k = sum_p w_p e_kp^2
    for (int p = 0; p < kQ; ++p) b += (double)wq(p) * mode_row(k, p) * mode_row(k, p);
    amp[k - 4] = (float)std::sqrt(3.0 * kT * (1.0 - g1 * g1) / b);
  }
}

__global__ void k_bump_step(DevStatus *status) { status->step += 1; }

cudaError_t launch_bump_step(DevStatus *status, cudaStream_t s) {
  k_bump_step<<<1, 1, 0, s>>>(status);
  return cudaGetLastError();
}

}  // namespace lbmd
