// First-order resident march, parked forms (Parked<N>: one envelope in
// registers, the other in shared memory, at most 128 registers): one channel
// per block of N/16 threads and 512/(N/16) blocks per SM, each at its own FFT
// phase.  Form 2 (Nx = 1024, 2048, 4096, first or fourth order) reads the
// tables from L2; form 3 (Nx = 2048, 4096, 8192, first order or Strang) keeps
// them in tensor memory (Nx = 1024, first order: two channels per block).
// Same per-channel arithmetic as the other forms (bitwise the same fields).
#include <cuda_runtime.h>

#include "bpm_march_impl.cuh"

namespace bpm {

bool march_parked_supported(int n, int form) {
  return form == 2 ? (n == 1024 || n == 2048 || n == 4096)
                   : form == 3 && (n == 1024 || n == 2048 || n == 4096 || n == 8192);
}

int march_parked_group(int n, int form) { return form == 3 && n == 1024 ? 2 : 1; }

size_t march_parked_smem_bytes(int n, int form) {
  if (form == 3 && n == 1024) return MarchBody<1024, 2, 1, 3>::type::smem_bytes();
  if (n == 1024) return Parked<1024, 1>::smem_bytes();
  if (n == 2048) return Parked<2048, 1>::smem_bytes();
  if (n == 4096) return Parked<4096, 1>::smem_bytes();
  if (n == 8192) return Parked<8192, 1>::smem_bytes();
  return 0;
}

cudaError_t march_set_attributes_parked() {
  cudaError_t e = cudaSuccess;
  cudaError_t r[] = {attr_one<1024, 1, 1, 2>(), attr_one<2048, 1, 1, 2>(),
                     attr_one<4096, 1, 1, 2>(), attr_one<2048, 1, 1, 3>(),
                     attr_one<4096, 1, 1, 3>(), attr_one<8192, 1, 1, 3>(),
                     attr_one<2048, 1, 2, 3>(), attr_one<4096, 1, 2, 3>(),
                     attr_one<8192, 1, 2, 3>(), attr_one<1024, 1, 4, 2>(),
                     attr_one<2048, 1, 4, 2>(), attr_one<4096, 1, 4, 2>(),
                     attr_one<1024, 2, 1, 3>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  return e;
}

cudaError_t launch_march_parked(int n, int form, int blocks, const MarchArgs& a, cudaStream_t s) {
  if (form == 3 && a.split_order == 2) {  // Strang: a half coupling before each propagation
    if (n == 2048) return launch_one<2048, 1, 2, 3>(blocks, a, s);
    if (n == 4096) return launch_one<4096, 1, 2, 3>(blocks, a, s);
    if (n == 8192) return launch_one<8192, 1, 2, 3>(blocks, a, s);
    return cudaErrorInvalidValue;
  }
  if (form == 2 && a.split_order == 4) {  // fourth order: two table sets from L2
    if (n == 1024) return launch_one<1024, 1, 4, 2>(blocks, a, s);
    if (n == 2048) return launch_one<2048, 1, 4, 2>(blocks, a, s);
    if (n == 4096) return launch_one<4096, 1, 4, 2>(blocks, a, s);
    return cudaErrorInvalidValue;
  }
  if (a.split_order != 1) return cudaErrorInvalidValue;
  if (form == 2) {
    if (n == 1024) return launch_one<1024, 1, 1, 2>(blocks, a, s);
    if (n == 2048) return launch_one<2048, 1, 1, 2>(blocks, a, s);
    if (n == 4096) return launch_one<4096, 1, 1, 2>(blocks, a, s);
  } else if (form == 3) {
    if (n == 1024) return launch_one<1024, 2, 1, 3>(blocks, a, s);
    if (n == 2048) return launch_one<2048, 1, 1, 3>(blocks, a, s);
    if (n == 4096) return launch_one<4096, 1, 1, 3>(blocks, a, s);
    if (n == 8192) return launch_one<8192, 1, 1, 3>(blocks, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace bpm
