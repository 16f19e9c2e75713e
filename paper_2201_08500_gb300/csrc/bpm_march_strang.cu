// Strang-splitting instantiations of the resident march kernel (Eq. split-op
// with a = (0, 1), b = (1/2, 1/2)): a half coupling before and after each
// propagation.  Kept in their own translation unit so that the first-order
// kernels are compiled (and register-allocated) without the extra step.
#include "bpm_march_impl.cuh"

namespace bpm {

cudaError_t march_set_attributes_strang() {
  cudaError_t e = cudaSuccess;
  cudaError_t r[] = {attr_one<256, 1, 2>(),  attr_one<256, 16, 2>(),
                     attr_one<512, 1, 2>(),  attr_one<512, 8, 2>(),
                     attr_one<1024, 1, 2>(), attr_one<1024, 4, 2>(),
                     attr_one<2048, 1, 2>(), attr_one<2048, 2, 2>(),
                     attr_one<4096, 1, 2>(), attr_one<8192, 1, 2>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  return e;
}

cudaError_t launch_march_strang(int n, int group, int blocks, const MarchArgs& a, cudaStream_t s) {
#define BPM_STRANG_CASE(NN, GG) \
  if (n == NN && group == GG) return launch_one<NN, GG, 2>(blocks, a, s);
  BPM_STRANG_CASE(256, 1) BPM_STRANG_CASE(256, 16)
  BPM_STRANG_CASE(512, 1) BPM_STRANG_CASE(512, 8)
  BPM_STRANG_CASE(1024, 1) BPM_STRANG_CASE(1024, 4)
  BPM_STRANG_CASE(2048, 1) BPM_STRANG_CASE(2048, 2)
  BPM_STRANG_CASE(4096, 1) BPM_STRANG_CASE(8192, 1)
#undef BPM_STRANG_CASE
  return cudaErrorInvalidValue;
}

}  // namespace bpm
