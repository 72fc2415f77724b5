// lb_aa.cu -- the in-place (AA-pattern) stream-collide kernels without the
// thermal source (the kernel template and its layout are in lb_aa.cuh).
#include "lb_aa.cuh"

namespace lbmd {

cudaError_t launch_lb_aa(int storage, const LbGeom &g, const LbPhys &ph, void *buf, int odd,
                         DevStatus *bump, cudaStream_t s) {
  return aa_launch_storage<false>(storage, g, ph, buf, odd, bump, s);
}

}  // namespace lbmd
