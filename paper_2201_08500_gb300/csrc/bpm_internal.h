// Internal declarations shared by the host runtime and the kernel translation
// units of libbpm.  Not part of the public ABI (include/bpm.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace bpm {

// One NVTX range per C-ABI call, named after the call (header-only NVTX 3: a
// no-op unless a profiler or tracing tool is attached to the process).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define BPM_NVTX() ::bpm::NvtxRange bpm_nvtx_range_(__func__)

// Number of complex elements each thread holds per envelope in the resident
// march kernel: one radix-16 butterfly group per thread per stage.
constexpr int kElemsPerThread = 16;

// exp(-2 pi i m / 32) for m = 1..15 in FP32: the correctly rounded cos and
// -sin of 2 pi m / 32 (m = 8: the FP32 value of cos(pi/2) in double, as the
// twiddle table holds it).  The 8192-point transform's third radix-16 stage
// multiplies by W_32^(j m) with j = t % 2, so these are its only twiddles; the
// kernels take them as immediates instead of loads (the loaded values kept
// ~30 registers live and made the 512-thread kernels spill), and the host
// twiddle table uses the same values at k = (n / 32) m.
__host__ __device__ constexpr float w32_re(int m) {
  return m == 1 ? 0x1.f6297cp-1f : m == 2 ? 0x1.d906bcp-1f : m == 3 ? 0x1.a9b662p-1f
       : m == 4 ? 0x1.6a09e6p-1f : m == 5 ? 0x1.1c73b4p-1f : m == 6 ? 0x1.87de2ap-2f
       : m == 7 ? 0x1.8f8b84p-3f : m == 8 ? 0x1.1a6264p-54f : m == 9 ? -0x1.8f8b84p-3f
       : m == 10 ? -0x1.87de2ap-2f : m == 11 ? -0x1.1c73b4p-1f : m == 12 ? -0x1.6a09e6p-1f
       : m == 13 ? -0x1.a9b662p-1f : m == 14 ? -0x1.d906bcp-1f : -0x1.f6297cp-1f;
}
__host__ __device__ constexpr float w32_im(int m) {
  return m == 1 ? -0x1.8f8b84p-3f : m == 2 ? -0x1.87de2ap-2f : m == 3 ? -0x1.1c73b4p-1f
       : m == 4 ? -0x1.6a09e6p-1f : m == 5 ? -0x1.a9b662p-1f : m == 6 ? -0x1.d906bcp-1f
       : m == 7 ? -0x1.f6297cp-1f : m == 8 ? -0x1.0p+0f : m == 9 ? -0x1.f6297cp-1f
       : m == 10 ? -0x1.d906bcp-1f : m == 11 ? -0x1.a9b662p-1f : m == 12 ? -0x1.6a09e6p-1f
       : m == 13 ? -0x1.1c73b4p-1f : m == 14 ? -0x1.87de2ap-2f : -0x1.8f8b84p-3f;
}

// Coupling coefficients of Eq. fov10 for one channel, FP32.  a is split into
// hi + lo parts so that its systematic rounding does not accumulate over the
// march; b+ (Eh -> E0) and b- (E0 -> Eh) are used once per step and stay FP32.
struct ChannelCoef {
  float2 a_hi, a_lo;
  float2 bp, bm;
};

// Arguments of the resident split-step march kernel (one 1D plan).
struct MarchArgs {
  const float4* tables;      // [n_ch][2][16][T] {hi.re, hi.im, lo.re, lo.im}; env 0 = E0, 1 = Eh
  const ChannelCoef* coef;   // [n_ch]
  const float2* twiddle;     // [N] exp(-2 pi i k / N), FP32 correctly rounded
  const float2* twiddle_t;   // stage twiddles in thread order (kernels that read them from memory)
  const float2* twiddle_p;   // the same in thread-ordered pairs (parked forms, 128-bit loads)
  const float2* cfield;      // [nz][N] Pi(x, z) exp(+i h u(x, z)); 0 outside the crystal
  float2* e0;                // [n_ch][N]
  float2* eh;                // [n_ch][N]
  const double* inc_norm;    // [n_ch] sum |A+(z=0)|^2
  double* refl;              // [n_ch] R
  double* trans;             // [n_ch] T
  int n_ch;
  int z0;
  int n_steps;
  int split_order;           // Eq. split-op: 1, 2 (Strang) or 4 (tables and coef then hold two sets)
};

// Arguments of the 3D row / column passes (bpm_3d.cu).
struct Pass3DArgs {
  float2* e0;                // [n_ch][ny][nx] natural order (x space)
  float2* eh;
  float2* s0;                // [n_ch][nx][ny] transposed x-spectrum (working buffers)
  float2* sh;
  const float2* cfield;      // [nz][ny][nx]
  const int2* cspan;         // [nz][ny] {first, end} x of the nonzero cells of each row
  const ChannelCoef* coef;   // [n_ch]
  const float2* twx;         // stage twiddles of the x transform in thread order (twiddle_order)
  const float2* twy;         // same for the y transform
  const float4* anchor;      // [n_ch][2][nx] FP32 hi + lo of exp(i dz (K - k)) / (nx ny g_x)
  const float* gcorr;        // [n_ch][2][nx] -dz / (2 K)
  const float2* qy;          // [16][ny/16] {qy^2, 1/g_y - 1}: entry k T + t is position 16 t + k
  int nx, ny, z;
};

// Per-plan device pointers used by the setup kernels.
struct SetupArgs {
  int nx, ny, nz, n_ch, dims;
  double dx, dy, dz;
  double h;                  // reciprocal-lattice vector
  double chi0_re, chi0_im, chih_re, chih_im, chihb_re, chihb_im;
  int zassenhaus;
  double coupling_frac;      // fraction of dz per coupling application (3D: 1)
  int split_order;           // 2D tables: Eq. split-op order 1, 2 or 4
  double x_surface, x_end;   // slab [x_surface, x_end) at z = 0
  double tan_psi;            // entrance surface x = x_surface + z tan_psi (asymmetric cut)
  double z_begin, z_end;     // crystal only for z_begin <= z < z_end (Laue slab)
  double theta_i, x0, w0, zx, zR;
  const unsigned char* mask;  // [nz][ny][nx] crystal cells (nonzero), replacing the bounds; or null
};

// One work-queue item: channels ch0 .. ch0 + G - 1 of plan `plan` (transform size n).
struct BatchItem {
  int plan;
  int ch0;
  int n;
  int reserved;
};

// Work-queue launchers (bpm_batch.cu).  A round sorts its items into these
// queues (longest items first within each) and launches the queues back to
// back, the Nx = 8192 queues of every order first, then 4096, 2048, 1024 and
// the resident small-N queues (enqueue_round in bpm_api.cu):
enum BatchQueue {
  kQueueTm8192 = 0,  // first order, Nx = 8192: parked form, TMEM tables
  kQueueTm4096,      // first order, Nx = 4096: parked form, TMEM tables, 2 blocks / SM
  kQueueTm2048,      // first order, Nx = 2048: parked form, TMEM tables, 4 blocks / SM
  kQueueSmall,       // first order, Nx <= 512: resident form, G channels per block
  kQueueSmall2,      // Strang, Nx <= 1024: resident form
  kQueueBig4,        // fourth order, Nx = 8192: parked form, L2 tables (two sets)
  kQueueSmall4,      // fourth order, Nx <= 512: resident form, L2 tables (two sets)
  kQueueTm8192s2,    // Strang, Nx = 8192: parked form, TMEM tables
  kQueueTm4096s2,    // Strang, Nx = 4096: parked form, TMEM tables, 2 blocks / SM
  kQueueTm2048s2,    // Strang, Nx = 2048: parked form, TMEM tables, 4 blocks / SM
  kQueuePk4096s4,    // fourth order, Nx = 4096: parked form, L2 tables, 2 blocks / SM
  kQueuePk2048s4,    // fourth order, Nx = 2048: parked form, L2 tables, 4 blocks / SM
  kQueuePk1024s4,    // fourth order, Nx = 1024: parked form, L2 tables, 8 blocks / SM
  kQueueTm1024,      // first order, Nx = 1024: parked form, TMEM tables, two channels a
                     // block, 4 blocks / SM
  kQueueCount
};
int batch_group(int n);                               // channels per block of the resident kernels
int batch_item_channels(int n, int split_order);      // channels per item
int batch_queue(int n, int split_order);
int batch_blocks_per_sm(int queue);
cudaError_t launch_batch(const MarchArgs* plans, const BatchItem* items, int n_items, int* counter,
                         int queue, int blocks, cudaStream_t s);

// Host runtime helpers (bpm_api.cu): FFT constants of size n (twiddles, spectrum
// order, round-trip gain; host memory owned by a process-wide cache) and a
// readiness check of the current device (sm_103, kernel attributes set).
void fft_host_constants(int n, const float2** tw, const int** rev, const double** gain);
bool device_ready(int* sm_count);

// One-time kernel attribute setup (dynamic shared memory limits); must run
// outside stream capture, before the first launch on the current device.
cudaError_t march_set_attributes();
cudaError_t batch_set_attributes();
cudaError_t setup_set_attributes();

// Launchers (bpm_march.cu).  Return cudaSuccess or the launch error.
int march_threads_per_channel(int n);
int march_max_group(int n);
size_t march_smem_bytes(int n, int group);
cudaError_t launch_march(int n, int group, int blocks, const MarchArgs& a, cudaStream_t s);
cudaError_t launch_march_strang(int n, int group, int blocks, const MarchArgs& a, cudaStream_t s);
// Second form of the first-order march: propagator tables and stage twiddles
// read from L2 instead of shared memory / registers, at most 128 registers, so
// that two blocks (two channel groups at independent FFT phases) share an SM.
bool march_l2_supported(int n, int group);
size_t march_l2_smem_bytes(int n, int group);
cudaError_t launch_march_l2(int n, int group, int blocks, const MarchArgs& a, cudaStream_t s);
cudaError_t march_set_attributes_l2();
// Parked form (one envelope in registers, one in shared memory) at Nx = 1024..4096:
// one channel per block, several blocks per SM.
// (form 2: tables from L2, Nx = 1024..4096; form 3: tables in tensor memory,
// Nx = 1024..8192, two channels per block at 1024).
bool march_parked_supported(int n, int form);
// Channels per block of a parked form (2 for form 3 at Nx = 1024, else 1).
int march_parked_group(int n, int form);
size_t march_parked_smem_bytes(int n, int form);
cudaError_t launch_march_parked(int n, int form, int blocks, const MarchArgs& a, cudaStream_t s);
cudaError_t march_set_attributes_parked();
cudaError_t march_set_attributes_strang();
// Fourth-order splitting (Eq. split-op, a = (0, t, 1-2t, t), b = (t/2, (1-t)/2, (1-t)/2, t/2)).
cudaError_t launch_march_split4(int n, int group, int blocks, const MarchArgs& a, cudaStream_t s);
cudaError_t march_set_attributes_split4();
size_t march_split4_smem_bytes(int n, int group);

// 3D passes (bpm_3d.cu).  mode: 0 forward x only, 1 inverse x + coupling +
// forward x, 2 inverse x + coupling.
bool pass3d_supported(int nx, int ny);
cudaError_t pass3d_set_attributes();
// row_threads: 256 or 512 (tile of 256/T or 512/T rows, T = nx/16)
cudaError_t launch_row_pass(int mode, int row_threads, const Pass3DArgs& a, int n_ch,
                            cudaStream_t s);
// form 0: one block per column group; form >= 1: the persistent column pass
// streamed by bulk copies (sms: the SM count; status: device word that a
// bounded wait which gave up sets to kStatusTmaTimeout)
cudaError_t launch_col_pass(int form, const Pass3DArgs& a, int n_ch, int sms, int* status,
                            cudaStream_t s);
// The MODE-1 row pass streamed by tensor copies (launch form 2): tiles of
// row_threads / (nx/16) rows, for (nx, row_threads) = (256, 128), (512, 128),
// (512, 256), (1024, 256); sms and status as for the column pass.
bool row_tma_supported(int nx, int row_threads);
cudaError_t launch_row_pass_tma(int row_threads, const Pass3DArgs& a, int n_ch, int sms,
                                int* status, cudaStream_t s);
cudaError_t launch_reduce3d(const float2* e0, const float2* eh, long long plane, int n_ch,
                            const double* inc, double* refl, double* trans, cudaStream_t s);

// Setup launchers (bpm_setup.cu).
cudaError_t launch_tables3d(const SetupArgs& sa, const double* omega, const double* gainx,
                            const int* revx, float4* anchor, float* gcorr, ChannelCoef* coef,
                            cudaStream_t s);
// Extent of the crystal in each of `rows` deformation rows of nx cells:
// span[r] = {first x with c != 0, last such x + 1}, {0, 0} for a row without
// crystal.  The 3D row pass loads a row's c only inside it (c = 0 outside).
// (The 1D marches load their rows unconditionally: guarding those loads by
// the extent measured slower there.)
cudaError_t launch_crystal_span(const float2* cfield, int nx, long long rows, int2* span,
                                cudaStream_t s);
cudaError_t launch_deformation(const SetupArgs& sa, const double* u_dev, float2* cfield,
                               cudaStream_t s);
cudaError_t launch_tables(const SetupArgs& sa, const double* omega, const double* gain,
                          const int* rev, float4* tables, ChannelCoef* coef, int* bad,
                          cudaStream_t s);
cudaError_t launch_incident(const SetupArgs& sa, const double* omega, const double2* weight,
                            float2* e0, float2* eh, double* inc_norm, cudaStream_t s);
// Time response of channels first .. first + n_local - 1 of n_total ([n_total]
// rows of plane values; the other channels count as zero).
cudaError_t launch_omega_to_t(int n_total, int first, int n_local, long long plane,
                              double domega, const float2* eh, double2* out, cudaStream_t s);

}  // namespace bpm
