// Allocation-free entry point: the single-instance BPM path with its
// intermediate buffers in a fixed, file-scope device array.
//
// Why: some callers cannot call cudaMalloc while they run this code -- for
// example a process whose device memory is entirely handed out by a
// caller-side pool, or a real-time loop that must not take the allocator's
// lock or risk fragmentation.  They
// pass their own input and output buffers; everything else (the deformation
// factor, the propagator tables, the coupling coefficients, the FFT constants,
// per-channel norms) lives in g_static_scratch below.
//
// Limits (rejected with BPM_ERR_UNSUPPORTED beyond them): dims = 2,
// 256 <= nx <= 4096, n_channels <= 16, nz * nx <= 524288 cells.  The array
// holds 6.3 MB on every GPU that loads the library, until the process exits.
#include <cuda_runtime.h>

#include <cmath>

#include <map>
#include <mutex>
#include <string>

#include "../../include/bpm.h"
#include "bpm_internal.h"

namespace bpm {
namespace {

constexpr int kStaticMaxNx = 4096;
constexpr int kStaticMaxChannels = 16;
constexpr long long kStaticMaxCells = 1LL << 19;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Byte offsets of the regions of the static array.
constexpr size_t kOffCfield = 0;
constexpr size_t kOffTables = kOffCfield + align256(sizeof(float2) * kStaticMaxCells);
constexpr size_t kOffCoef =
    kOffTables + align256(sizeof(float4) * 2 * kStaticMaxNx * size_t(kStaticMaxChannels));
constexpr size_t kOffTwiddle = kOffCoef + align256(sizeof(ChannelCoef) * kStaticMaxChannels);
constexpr size_t kOffRev = kOffTwiddle + align256(sizeof(float2) * kStaticMaxNx);
constexpr size_t kOffGain = kOffRev + align256(sizeof(int) * kStaticMaxNx);
constexpr size_t kOffOmega = kOffGain + align256(sizeof(double) * kStaticMaxNx);
constexpr size_t kOffWeight = kOffOmega + align256(sizeof(double) * kStaticMaxChannels);
constexpr size_t kOffNorm = kOffWeight + align256(sizeof(double2) * kStaticMaxChannels);
constexpr size_t kOffTrans = kOffNorm + align256(sizeof(double) * kStaticMaxChannels);
constexpr size_t kOffFlag = kOffTrans + align256(sizeof(double) * kStaticMaxChannels);
constexpr size_t kStaticBytes = kOffFlag + 256;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch, looked up once per device (with that
// device current).  In host code the symbol is only a stand-in for the device
// array, so kernels receive this address instead.
std::mutex g_static_mu;
std::map<int, unsigned char*> g_static_addr;

cudaError_t static_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_static_mu);
  auto it = g_static_addr.find(dev);
  if (it != g_static_addr.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess) return e;
  g_static_addr[dev] = static_cast<unsigned char*>(ptr);
  *out = static_cast<unsigned char*>(ptr);
  return cudaSuccess;
}

thread_local std::string g_static_error = "no error";

bpm_status sfail(bpm_status s, const std::string& m) {
  g_static_error = m;
  return s;
}

#define BPM_SCUDA(call, what)                                                        \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return sfail(BPM_ERR_CUDA, std::string(what) + ": " +     \
                                                      cudaGetErrorString(e_));       \
  } while (0)

}  // namespace
}  // namespace bpm

using namespace bpm;

extern "C" {

BPM_API size_t bpm_noalloc_scratch_bytes(void) { return kStaticBytes; }

BPM_API const char* bpm_noalloc_last_error(void) { return g_static_error.c_str(); }

BPM_API bpm_status bpm_run_noalloc(const bpm_grid* grid, int n_channels,
                                   const bpm_crystal_params* crystal, const double* u_field_dev,
                                   const double* omega, const double* weight_re_im,
                                   const bpm_beam_params* beam, void* e0_dev, void* eh_dev,
                                   double* refl_dev, void* cuda_stream) {
  BPM_NVTX();
  if (!grid || !crystal || !beam || !omega || !weight_re_im || !e0_dev || !eh_dev || !refl_dev)
    return sfail(BPM_ERR_INVALID_ARG, "null argument");
  const bpm_grid& g = *grid;
  if (g.dims != 2 || g.ny != 1)
    return sfail(BPM_ERR_UNSUPPORTED, "the allocation-free entry point takes 2D grids (ny = 1)");
  if (g.nx < 256 || g.nx > kStaticMaxNx || (g.nx & (g.nx - 1)))
    return sfail(BPM_ERR_UNSUPPORTED, "nx must be a power of two in [256, 4096] here");
  if (n_channels < 1 || n_channels > kStaticMaxChannels)
    return sfail(BPM_ERR_UNSUPPORTED, "n_channels must lie in [1, 16] here");
  if (g.nz < 1 || (long long)g.nz * g.nx > kStaticMaxCells)
    return sfail(BPM_ERR_UNSUPPORTED, "nz * nx must lie in [1, 524288] here");
  if (!(g.dx > 0) || !(g.dz > 0) || g.split_order != 1)
    return sfail(BPM_ERR_INVALID_ARG, "dx, dz must be positive and split_order 1");
  const double kPiS = 3.14159265358979323846;
  if (!(crystal->theta_B >= 0.0) || crystal->theta_B >= 85.0 * kPiS / 180.0 ||
      !(crystal->lambda_B > 0.0) || !(crystal->thickness >= 0.0) || !(beam->w0 > 0.0))
    return sfail(BPM_ERR_INVALID_ARG, "crystal or beam parameters out of range");
  int sms = 0;
  if (!device_ready(&sms))
    return sfail(BPM_ERR_UNSUPPORTED, "libbpm needs a GB300 (sm_103a) device");
  unsigned char* base = nullptr;
  BPM_SCUDA(static_scratch(&base), "static scratch address");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  SetupArgs sa{};
  sa.nx = g.nx;
  sa.ny = 1;
  sa.nz = g.nz;
  sa.n_ch = n_channels;
  sa.dims = 2;
  sa.dx = g.dx;
  sa.dy = g.dy;
  sa.dz = g.dz;
  sa.h = 4.0 * kPiS * std::sin(crystal->theta_B) / crystal->lambda_B;
  sa.chi0_re = crystal->chi0_re;
  sa.chi0_im = crystal->chi0_im;
  sa.chih_re = crystal->chih_re;
  sa.chih_im = crystal->chih_im;
  sa.chihb_re = crystal->chihbar_re;
  sa.chihb_im = crystal->chihbar_im;
  sa.zassenhaus = g.zassenhaus ? 1 : 0;
  sa.coupling_frac = 1.0;
  sa.split_order = 1;
  sa.x_surface = crystal->x_surface;
  sa.x_end = crystal->x_surface + crystal->thickness;
  sa.tan_psi = 0.0;  // symmetric-Bragg slab only on this entry point
  sa.z_begin = -HUGE_VAL;
  sa.z_end = HUGE_VAL;
  sa.theta_i = beam->theta_i;
  sa.x0 = beam->x0;
  sa.w0 = beam->w0;
  sa.zx = beam->zx;
  sa.zR = beam->zR;
  for (int i = 0; i < n_channels; ++i)
    if (!(omega[i] / 299792458.0 > 0.5 * sa.h))
      return sfail(BPM_ERR_INVALID_ARG, "a channel has k <= h/2 (no Bragg solution)");

  float2* cfield = reinterpret_cast<float2*>(base + kOffCfield);
  float4* tables = reinterpret_cast<float4*>(base + kOffTables);
  ChannelCoef* coef = reinterpret_cast<ChannelCoef*>(base + kOffCoef);
  float2* twiddle = reinterpret_cast<float2*>(base + kOffTwiddle);
  int* rev = reinterpret_cast<int*>(base + kOffRev);
  double* gain = reinterpret_cast<double*>(base + kOffGain);
  double* d_omega = reinterpret_cast<double*>(base + kOffOmega);
  double2* d_weight = reinterpret_cast<double2*>(base + kOffWeight);
  double* inc_norm = reinterpret_cast<double*>(base + kOffNorm);
  double* trans = reinterpret_cast<double*>(base + kOffTrans);
  int* flag = reinterpret_cast<int*>(base + kOffFlag);

  const float2* h_tw;
  const int* h_rev;
  const double* h_gain;
  fft_host_constants(g.nx, &h_tw, &h_rev, &h_gain);
  // every region below is rewritten in full by this call; only the flag must start at zero
  BPM_SCUDA(cudaMemcpyAsync(twiddle, h_tw, sizeof(float2) * g.nx, cudaMemcpyHostToDevice, st),
            "upload twiddles");
  BPM_SCUDA(cudaMemcpyAsync(rev, h_rev, sizeof(int) * g.nx, cudaMemcpyHostToDevice, st),
            "upload spectrum order");
  BPM_SCUDA(cudaMemcpyAsync(gain, h_gain, sizeof(double) * g.nx, cudaMemcpyHostToDevice, st),
            "upload gain");
  BPM_SCUDA(cudaMemcpyAsync(d_omega, omega, sizeof(double) * n_channels, cudaMemcpyHostToDevice,
                            st),
            "upload omega");
  BPM_SCUDA(cudaMemcpyAsync(d_weight, weight_re_im, sizeof(double2) * n_channels,
                            cudaMemcpyHostToDevice, st),
            "upload weights");
  BPM_SCUDA(cudaMemsetAsync(flag, 0, sizeof(int), st), "clear flag");

  float2* e0 = static_cast<float2*>(e0_dev);
  float2* eh = static_cast<float2*>(eh_dev);
  BPM_SCUDA(launch_deformation(sa, u_field_dev, cfield, st), "deformation kernel");
  BPM_SCUDA(launch_tables(sa, d_omega, gain, rev, tables, coef, flag, st), "tables kernel");
  BPM_SCUDA(launch_incident(sa, d_omega, d_weight, e0, eh, inc_norm, st), "incident kernel");
  MarchArgs a;
  a.tables = tables;
  a.coef = coef;
  a.twiddle = twiddle;
  a.twiddle_t = nullptr;  // nx <= 4096: twiddles stay in registers
  a.twiddle_p = nullptr;
  a.cfield = cfield;
  a.e0 = e0;
  a.eh = eh;
  a.inc_norm = inc_norm;
  a.refl = refl_dev;
  a.trans = trans;
  a.n_ch = n_channels;
  a.z0 = 0;
  a.n_steps = g.nz;
  a.split_order = 1;
  BPM_SCUDA(launch_march(g.nx, 1, n_channels, a, st), "march kernel");
  return BPM_OK;
}

}  // extern "C"
