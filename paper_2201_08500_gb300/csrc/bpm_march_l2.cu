// First-order resident march, L2-table form (Resident<..., L2TAB = true>): the
// same per-channel arithmetic as bpm_march.cu (bitwise identical results), with
// propagator tables and stage twiddles read from L2 and at most 128 registers,
// so that two blocks share an SM and their FFT exchanges overlap the other
// block's butterflies.
#include <cuda_runtime.h>

#include "bpm_march_impl.cuh"

namespace bpm {

bool march_l2_supported(int n, int group) {
  return (n == 4096 && group == 1) || (n == 2048 && group == 2) || (n == 1024 && group == 4) ||
         (n == 512 && group == 8) || (n == 256 && group == 16);
}

size_t march_l2_smem_bytes(int n, int group) {
#define BPM_L2_SMEM(NN, GG) \
  if (n == NN && group == GG) return Resident<NN, GG, 1, true>::smem_bytes();
  BPM_L2_SMEM(256, 16) BPM_L2_SMEM(512, 8) BPM_L2_SMEM(1024, 4) BPM_L2_SMEM(2048, 2)
  BPM_L2_SMEM(4096, 1)
#undef BPM_L2_SMEM
  return 0;
}

cudaError_t march_set_attributes_l2() {
  cudaError_t e = cudaSuccess;
  cudaError_t r[] = {attr_one<256, 16, 1, true>(), attr_one<512, 8, 1, true>(),
                     attr_one<1024, 4, 1, true>(), attr_one<2048, 2, 1, true>(),
                     attr_one<4096, 1, 1, true>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  return e;
}

cudaError_t launch_march_l2(int n, int group, int blocks, const MarchArgs& a, cudaStream_t s) {
#define BPM_L2_LAUNCH(NN, GG) \
  if (n == NN && group == GG) return launch_one<NN, GG, 1, true>(blocks, a, s);
  BPM_L2_LAUNCH(256, 16) BPM_L2_LAUNCH(512, 8) BPM_L2_LAUNCH(1024, 4) BPM_L2_LAUNCH(2048, 2)
  BPM_L2_LAUNCH(4096, 1)
#undef BPM_L2_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace bpm
