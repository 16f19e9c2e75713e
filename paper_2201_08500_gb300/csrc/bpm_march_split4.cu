// Fourth-order splitting instantiations of the resident march kernel (Eq.
// split-op with t = 1/(2 - 2^(1/3)), a = (0, t, 1-2t, t), b = (t/2, (1-t)/2,
// (1-t)/2, t/2)): per z step three propagations and four couplings, the two
// propagator tables of each channel read from L2.  Own translation unit, like
// the Strang kernels.
#include "bpm_march_impl.cuh"

namespace bpm {

size_t march_split4_smem_bytes(int n, int group) {
#define BPM_S4_SMEM(NN, GG) \
  if (n == NN && group == GG) return MarchBody<NN, GG, 4, 0>::type::smem_bytes();
  BPM_S4_SMEM(256, 1) BPM_S4_SMEM(256, 16) BPM_S4_SMEM(512, 1) BPM_S4_SMEM(512, 8)
  BPM_S4_SMEM(1024, 1) BPM_S4_SMEM(1024, 4) BPM_S4_SMEM(2048, 1) BPM_S4_SMEM(2048, 2)
  BPM_S4_SMEM(4096, 1) BPM_S4_SMEM(8192, 1)
#undef BPM_S4_SMEM
  return 0;
}

cudaError_t march_set_attributes_split4() {
  cudaError_t e = cudaSuccess;
  cudaError_t r[] = {attr_one<256, 1, 4>(),  attr_one<256, 16, 4>(), attr_one<512, 1, 4>(),
                     attr_one<512, 8, 4>(),  attr_one<1024, 1, 4>(), attr_one<1024, 4, 4>(),
                     attr_one<2048, 1, 4>(), attr_one<2048, 2, 4>(), attr_one<4096, 1, 4>(),
                     attr_one<8192, 1, 4>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  return e;
}

cudaError_t launch_march_split4(int n, int group, int blocks, const MarchArgs& a, cudaStream_t s) {
#define BPM_S4_CASE(NN, GG) \
  if (n == NN && group == GG) return launch_one<NN, GG, 4>(blocks, a, s);
  BPM_S4_CASE(256, 1) BPM_S4_CASE(256, 16)
  BPM_S4_CASE(512, 1) BPM_S4_CASE(512, 8)
  BPM_S4_CASE(1024, 1) BPM_S4_CASE(1024, 4)
  BPM_S4_CASE(2048, 1) BPM_S4_CASE(2048, 2)
  BPM_S4_CASE(4096, 1) BPM_S4_CASE(8192, 1)
#undef BPM_S4_CASE
  return cudaErrorInvalidValue;
}

}  // namespace bpm
