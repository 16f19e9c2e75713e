// Resident split-step march of the two-beam BPM (Eq. fov10, first-order
// splitting a1 = b1 = 1 of Eq. split-op), one frequency channel per group of
// T = N/16 threads.  Both envelopes stay in registers for the whole march; per
// step each thread
//   1. prefetches its 16 deformation factors c(x, z_n) = Pi exp(+i h u) for the
//      coupling at the end of the step (coalesced, latency hidden by the FFTs);
//   2. runs the forward FFT of E0 and Eh (radix-16 register butterflies with
//      shared-memory exchanges, see bpm_fft.cuh);
//   3. multiplies the digit-reversed spectra by the tilted propagators
//      p+- = exp(i dz [sqrt(k^2 - (q +- h/2)^2) - k]) (Eq. fov4 with the shifted
//      spectrum after Eq. fov10), stored as FP32 hi + lo pairs that also carry
//      1/N and the FFT round-trip gain correction;
//   4. runs the inverse FFT (exact adjoint of the forward);
//   5. couples the envelopes pointwise (Eq. fov10 with Eq. Authier):
//        E0 <- a E0 + b+ c Eh,   Eh <- a Eh + b- conj(c) E0   inside the crystal.
// At the end of the launch the fields are written back and the per-channel
// reflectivity / transmissivity sums are reduced in FP64.
#include <cuda_runtime.h>

#include "bpm_march_impl.cuh"

namespace bpm {

namespace {

}  // namespace

int march_threads_per_channel(int n) { return n / 16; }

int march_max_group(int n) {
  switch (n) {
    case 256: return 16;
    case 512: return 8;
    case 1024: return 4;
    case 2048: return 2;
    default: return 1;
  }
}

size_t march_smem_bytes(int n, int group) {
#define BPM_SMEM_CASE(NN, GG) \
  if (n == NN && group == GG) return MarchBody<NN, GG, 1, 0>::type::smem_bytes();
  BPM_SMEM_CASE(256, 1) BPM_SMEM_CASE(256, 16)
  BPM_SMEM_CASE(512, 1) BPM_SMEM_CASE(512, 8)
  BPM_SMEM_CASE(1024, 1) BPM_SMEM_CASE(1024, 4)
  BPM_SMEM_CASE(2048, 1) BPM_SMEM_CASE(2048, 2)
  BPM_SMEM_CASE(4096, 1) BPM_SMEM_CASE(8192, 1)
#undef BPM_SMEM_CASE
  return 0;
}

cudaError_t march_set_attributes() {
  cudaError_t e = march_set_attributes_strang();
  if (cudaError_t e4 = march_set_attributes_split4(); e4 != cudaSuccess) e = e4;
  cudaError_t r[] = {attr_one<256, 1, 1>(),  attr_one<256, 16, 1>(),
                     attr_one<512, 1, 1>(),  attr_one<512, 8, 1>(),
                     attr_one<1024, 1, 1>(), attr_one<1024, 4, 1>(),
                     attr_one<2048, 1, 1>(), attr_one<2048, 2, 1>(),
                     attr_one<4096, 1, 1>(), attr_one<8192, 1, 1>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  return e;
}

cudaError_t launch_march(int n, int group, int blocks, const MarchArgs& a, cudaStream_t s) {
  if (a.split_order == 2) return launch_march_strang(n, group, blocks, a, s);
  if (a.split_order == 4) return launch_march_split4(n, group, blocks, a, s);
#define BPM_LAUNCH_CASE(NN, GG) \
  if (n == NN && group == GG) return launch_one<NN, GG, 1>(blocks, a, s);
  BPM_LAUNCH_CASE(256, 1) BPM_LAUNCH_CASE(256, 16)
  BPM_LAUNCH_CASE(512, 1) BPM_LAUNCH_CASE(512, 8)
  BPM_LAUNCH_CASE(1024, 1) BPM_LAUNCH_CASE(1024, 4)
  BPM_LAUNCH_CASE(2048, 1) BPM_LAUNCH_CASE(2048, 2)
  BPM_LAUNCH_CASE(4096, 1) BPM_LAUNCH_CASE(8192, 1)
#undef BPM_LAUNCH_CASE
  return cudaErrorInvalidValue;
}

}  // namespace bpm
