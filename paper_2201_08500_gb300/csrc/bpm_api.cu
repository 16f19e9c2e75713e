// Host runtime of libbpm: the C ABI of include/bpm.h.
//
// A plan owns the device state of one BPM problem (one crystal, one pulse,
// n_channels frequency channels): the deformation factor c(x, z), the per
// channel propagator tables and coupling coefficients, the two envelopes, the
// reflectivities and the time response.  All device work is enqueued on the
// caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/bpm.h"
#include "bpm_internal.h"

using namespace bpm;

namespace {

constexpr double kPiHost = 3.14159265358979323846;

thread_local std::string g_thread_error = "no error";

// ---------------------------------------------------------------------------
// FFT constants of one transform size: FP32 twiddles exp(-2 pi i k / n), the
// position -> frequency map of the digit-reversed spectrum and the round-trip
// gain g(p) = (1/n) sum_j |F_pj|^2 of the FP32 transform (F built from the
// FP32 twiddle and butterfly constants).  Dividing the propagator by g removes
// the first-order systematic magnitude error of forward + inverse transform
// (the phase errors already cancel because the inverse is the exact adjoint).
// ---------------------------------------------------------------------------
struct FftConsts {
  std::vector<float2> tw;
  std::vector<int> rev;
  std::vector<double> gain;
};

int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

double mag2_butterfly(int radix, int k, int m) {
  const double c8 = double(0.70710678118654752440f);
  const double c16 = double(0.92387953251128675613f);
  const double s16 = double(0.38268343236508977173f);
  if (radix == 16) {
    const int e = (k % 4) * (m % 4);
    if (e == 0 || e == 4) return 1.0;
    if (e == 2 || e == 6) return 2.0 * c8 * c8;
    return c16 * c16 + s16 * s16;
  }
  if (radix == 8) {
    const int e = (k % 2) * (m % 4);
    if (e == 0 || e == 2) return 1.0;
    return 2.0 * c8 * c8;
  }
  return 1.0;
}

const FftConsts& fft_consts(int n) {
  static std::mutex mu;
  static std::map<int, std::unique_ptr<FftConsts>> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(n);
  if (it != cache.end()) return *it->second;
  auto f = std::make_unique<FftConsts>();
  f->tw.resize(n);
  for (int k = 0; k < n; ++k) {
    const double a = 2.0 * kPiHost * double(k) / double(n);
    f->tw[k] = make_float2(float(std::cos(a)), float(-std::sin(a)));
  }
  // the W_32 powers the kernels take as immediates (w32_re / w32_im): the same
  // correctly rounded values, written here so that kernel and table agree
  for (int m = 1; m < 16 && n >= 32; ++m)
    f->tw[size_t(n / 32) * m] = make_float2(w32_re(m), w32_im(m));
  const int logn = ilog2i(n);
  const int S = (logn + 3) / 4;
  const int rlast = n >> (4 * (S - 1));
  auto L = [&](int s) { return s < S ? (n >> (4 * s)) : 1; };
  auto radix = [&](int s) { return s < S - 1 ? 16 : rlast; };
  f->rev.resize(n);
  for (int p = 0; p < n; ++p) {
    int rem = p, freq = 0, mul = 1;
    for (int s = 0; s < S; ++s) {
      const int d = rem / L(s + 1);
      rem %= L(s + 1);
      freq += d * mul;
      mul *= radix(s);
    }
    f->rev[p] = freq;
  }
  std::vector<double> G(n, 1.0), in(16), out(16);
  std::vector<int> pos(16);
  for (int s = 0; s < S; ++s) {
    const int R = radix(s);
    if (s < S - 1) {
      const int ls = L(s), ln = L(s + 1), stride = n / ls;
      for (int b = 0; b < n / ls; ++b)
        for (int j = 0; j < ln; ++j) {
          for (int k = 0; k < 16; ++k) {
            pos[k] = b * ls + j + ln * k;
            in[k] = G[pos[k]];
          }
          for (int m = 0; m < 16; ++m) {
            const float2 w = f->tw[(size_t(stride) * j * m) % n];
            const double tw2 = double(w.x) * w.x + double(w.y) * w.y;
            double acc = 0.0;
            for (int k = 0; k < 16; ++k) acc += in[k] * mag2_butterfly(16, k, m);
            out[m] = acc * tw2;
          }
          for (int m = 0; m < 16; ++m) G[pos[m]] = out[m];
        }
    } else {
      for (int b = 0; b < n / R; ++b) {
        for (int k = 0; k < R; ++k) in[k] = G[b * R + k];
        for (int m = 0; m < R; ++m) {
          double acc = 0.0;
          for (int k = 0; k < R; ++k) acc += in[k] * mag2_butterfly(R, k, m);
          out[m] = acc;
        }
        for (int m = 0; m < R; ++m) G[b * R + m] = out[m];
      }
    }
  }
  f->gain.resize(n);
  for (int p = 0; p < n; ++p) f->gain[p] = G[p] / double(n);
  auto& ref = *f;
  cache[n] = std::move(f);
  return ref;
}

// Stage twiddles W_L(s)^(j m) of an n-point transform in the order the 3D pass
// kernels read them: for each stage s < S-1, m = 1..15, j = 0..L(s+1)-1.
std::vector<float2> twiddle_order(int n) {
  const FftConsts& f = fft_consts(n);
  const int logn = ilog2i(n);
  const int S = (logn + 3) / 4;
  std::vector<float2> out;
  for (int s = 0; s < S - 1; ++s) {
    const int ls = n >> (4 * s), ln = n >> (4 * (s + 1)), stride = n / ls;
    for (int m = 1; m < 16; ++m)
      for (int j = 0; j < ln; ++j) out.push_back(f.tw[(size_t(stride) * j * m) % n]);
  }
  return out;
}

// The same twiddles in pairs for 128-bit loads: stage s, outputs m = 2i+1 and
// 2i+2 (i = 0..7; the second half of pair 7 is padding) of thread index j < ln
// at float2 offset 2 (off(s) + i ln + j), off(s) = sum over earlier stages of
// 8 ln.  Same FP32 values as twiddle_order.
std::vector<float2> twiddle_pairs(int n) {
  const FftConsts& f = fft_consts(n);
  const int logn = ilog2i(n);
  const int S = (logn + 3) / 4;
  std::vector<float2> out;
  for (int s = 0; s < S - 1; ++s) {
    const int ls = n >> (4 * s), ln = n >> (4 * (s + 1)), stride = n / ls;
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < ln; ++j) {
        out.push_back(f.tw[(size_t(stride) * j * (2 * i + 1)) % n]);
        out.push_back(i < 7 ? f.tw[(size_t(stride) * j * (2 * i + 2)) % n] : make_float2(0.f, 0.f));
      }
  }
  return out;
}

struct DeviceInfo {
  int sm_count = 0;
  int cc = 0;
  bool ok = false;
};

const DeviceInfo& device_info() {
  static std::mutex mu;
  static std::map<int, DeviceInfo> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  DeviceInfo d;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
    d.sm_count = prop.multiProcessorCount;
    d.cc = prop.major * 10 + prop.minor;
    d.ok = true;
    if (d.cc == 103)
      d.ok = march_set_attributes() == cudaSuccess && march_set_attributes_l2() == cudaSuccess &&
             march_set_attributes_parked() == cudaSuccess &&
             batch_set_attributes() == cudaSuccess &&
             setup_set_attributes() == cudaSuccess && pass3d_set_attributes() == cudaSuccess;
  }
  cache[dev] = d;
  return cache[dev];
}

}  // namespace

namespace bpm {
void fft_host_constants(int n, const float2** tw, const int** rev, const double** gain) {
  const FftConsts& f = fft_consts(n);
  *tw = f.tw.data();
  *rev = f.rev.data();
  *gain = f.gain.data();
}
bool device_ready(int* sm_count) {
  const DeviceInfo& d = device_info();
  if (sm_count) *sm_count = d.sm_count;
  return d.ok && d.cc == 103;
}
}  // namespace bpm

struct bpm_plan_s {
  bpm_grid grid{};
  int n_ch = 0;
  cudaStream_t stream = nullptr;
  std::string err = "no error";
  int plane = 0;

  bool have_crystal = false, have_pulse = false, time_valid = false, have_geometry = false;
  int z = 0;
  SetupArgs sa{};
  double domega = 1.0;
  // channel shard: this plan holds channels shard_first .. + n_ch - 1 of
  // shard_total (all of them unless bpm_set_channel_shard says otherwise)
  bool sharded = false;
  int shard_first = 0, shard_total = 0;

  // device buffers
  float2* cfield = nullptr;
  int2* cspan = nullptr;  // 3D: [nz][ny] crystal extent of each deformation row
  float2* e0 = nullptr;
  float2* eh = nullptr;
  float4* tables = nullptr;
  ChannelCoef* coef = nullptr;
  float2* twiddle = nullptr;
  float2* twiddle_t = nullptr;   // 2D: stage twiddles in thread order
  float2* twiddle_p = nullptr;   // 2D: the same in thread-ordered pairs
  int* rev = nullptr;
  double* gain = nullptr;
  double* omega = nullptr;
  double2* weight = nullptr;
  double* inc_norm = nullptr;
  double* refl = nullptr;
  double* trans = nullptr;
  double2* eh_time = nullptr;
  int* dflag = nullptr;
  double* u_tmp = nullptr;
  float* gcorr = nullptr;        // 3D: curvature factor per column
  float2* spec = nullptr;        // 3D: transposed x-spectra of both envelopes [2][ch][nx][ny]
  float2* twy = nullptr;         // 3D: y twiddles (thread order)
  float2* twx3 = nullptr;        // 3D: x twiddles (thread order)
  float2* qy = nullptr;          // 3D: {qy^2, 1/g_y - 1} per y-spectrum position
  const double* u_dev = nullptr;  // displacement used by the deformation setup (may be null)
  unsigned char* mask = nullptr;  // caller's crystal shape [nz][ny][nx] (plan-owned copy) or null
  size_t bytes = 0;               // device bytes owned by the plan

  int group = 1, blocks = 0;
  int form = 0;  // march form: 0 tables in shared memory, 1 tables in L2 (two blocks / SM)
  int row_threads = 256;  // 3D row pass tile: 256 or 512 threads
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bpm_stats stats{};
};

namespace {
// Rows of the plan's time response: all channels of the shard's instance.
int time_rows(const bpm_plan_s* p) { return p->sharded ? p->shard_total : p->n_ch; }
}  // namespace

namespace {

bpm_status fail(bpm_plan p, bpm_status s, const std::string& msg) {
  if (p)
    p->err = msg;
  else
    g_thread_error = msg;
  return s;
}

bpm_status cuda_fail(bpm_plan p, cudaError_t e, const char* what) {
  return fail(p, BPM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BPM_CUDA(p, call, what)                   \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      if (e_ == cudaErrorMemoryAllocation)        \
        return fail((p), BPM_ERR_OOM, what);      \
      return cuda_fail((p), e_, what);            \
    }                                             \
  } while (0)

template <typename T>
cudaError_t dalloc(T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
}

void free_plan_buffers(bpm_plan p) {
  void* ptrs[] = {p->cfield, p->e0,      p->eh,    p->tables, p->coef,     p->twiddle,
                  p->rev,    p->gain,    p->omega, p->weight, p->inc_norm, p->refl,
                  p->trans,  p->eh_time, p->dflag, p->u_tmp,  p->gcorr,    p->twy,
                  p->qy,     p->spec,    p->twx3,  p->twiddle_t, p->twiddle_p, p->mask,
                  p->cspan};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Device bytes a 1D plan allocates (fields, tables, deformation factor, outputs).
// Launch forms chosen by the autotuner, per shape, for this process.
struct TuneEntry {
  int form = 0, group = 1, row_threads = 256;
  float ms = 0.f;
};
using TuneKey = std::tuple<int, int, int, int, int>;  // dims, nx, ny, split order, channels
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;

TuneKey tune_key(const bpm_grid& g, int n_ch) {
  return TuneKey(g.dims, g.nx, g.dims == 3 ? g.ny : 1, g.split_order, n_ch);
}

// Whether a plan of grid g can run launch form (form, group, row_threads).
bool launch_valid(const bpm_grid& g, int form, int group, int row_threads) {
  if (g.dims == 3)
    return group == 1 && (((form == 0 || form == 1) && (row_threads == 256 || row_threads == 512)) ||
                          (form == 2 && row_tma_supported(g.nx, row_threads)));
  const int maxg = march_max_group(g.nx);
  if (row_threads != 256) return false;
  if (form == 0) return group == 1 || group == maxg;
  if (form == 3 && g.nx == 1024)  // two channels per block, first order
    return group == march_parked_group(g.nx, form) && g.split_order == 1;
  if (form == 2 || form == 3)
    return group == 1 &&
           (g.split_order == 1 || (form == 3 && g.split_order == 2) ||
            (form == 2 && g.split_order == 4)) &&
           march_parked_supported(g.nx, form);
  return form == 1 && g.split_order == 1 && march_l2_supported(g.nx, group);
}

// Derived launch quantities of the plan's form (2D: the march kernel's
// geometry; 3D plans run two passes a step, whose grids the passes size
// themselves, so only channels_per_block is set).
void apply_launch(bpm_plan p) {
  p->blocks = (p->n_ch + p->group - 1) / p->group;
  p->stats.channels_per_block = p->group;
  if (p->grid.dims == 3) {
    p->stats.threads_per_channel = 0;
    p->stats.blocks = 0;
    p->stats.smem_bytes = 0;
    return;
  }
  p->stats.threads_per_channel = march_threads_per_channel(p->grid.nx);
  p->stats.blocks = p->blocks;
  p->stats.smem_bytes = int(p->form == 1   ? march_l2_smem_bytes(p->grid.nx, p->group)
                            : p->form >= 2 ? march_parked_smem_bytes(p->grid.nx, p->form)
                                           : march_smem_bytes(p->grid.nx, p->group));
}

size_t plan_bytes(const bpm_grid& g, int n_ch) {
  const size_t plane = size_t(g.nx) * (g.dims == 3 ? g.ny : 1);
  const size_t nf = size_t(n_ch) * plane;
  size_t b = 0;
  b += size_t(g.nz) * plane * sizeof(float2);      // deformation factor
  if (g.dims == 3) b += size_t(g.nz) * g.ny * sizeof(int2);  // its rows' crystal extents
  b += 2 * nf * sizeof(float2);                    // E0, Eh
  const size_t sets = g.split_order == 4 ? 2 : 1;   // table / coefficient sets per channel
  b += sets * n_ch * 2 * g.nx * sizeof(float4);     // propagator tables (3D: column anchors)
  if (g.dims == 3)
    b += size_t(n_ch) * 2 * g.nx * sizeof(float) + size_t(g.ny) * 2 * sizeof(float2) +
         2 * nf * sizeof(float2);
  b += sets * n_ch * sizeof(ChannelCoef);
  b += size_t(g.nx) * (sizeof(float2) + sizeof(int) + sizeof(double));
  if (g.dims == 2) b += 3 * size_t(g.nx) * sizeof(float2);  // thread-order twiddles, pairs
  b += size_t(n_ch) * (5 * sizeof(double) + sizeof(double2));
  b += nf * sizeof(double2);                       // time response
  return b;
}

// Re-derive the deformation factor of the plan from its stored displacement.
cudaError_t enqueue_crystal(bpm_plan p) {
  cudaError_t e = launch_deformation(p->sa, p->u_dev, p->cfield, p->stream);
  if (e != cudaSuccess || p->grid.dims != 3) return e;
  // 3D: the row pass loads each deformation row only inside its crystal extent
  return launch_crystal_span(p->cfield, p->grid.nx, (long long)p->grid.nz * p->grid.ny, p->cspan,
                             p->stream);
}

// Tables, coefficients and incident field from the stored pulse; march back to z = 0.
cudaError_t enqueue_pulse(bpm_plan p) {
  cudaError_t e = p->grid.dims == 3
                      ? launch_tables3d(p->sa, p->omega, p->gain, p->rev, p->tables, p->gcorr,
                                        p->coef, p->stream)
                      : launch_tables(p->sa, p->omega, p->gain, p->rev, p->tables, p->coef,
                                      p->dflag, p->stream);
  if (e != cudaSuccess) return e;
  e = launch_incident(p->sa, p->omega, p->weight, p->e0, p->eh, p->inc_norm, p->stream);
  p->z = 0;
  p->time_valid = false;
  return e;
}

}  // namespace

extern "C" {

BPM_API const char* bpm_version(void) { return "libbpm 0.1 (sm_103a, resident radix-16 march)"; }

BPM_API const char* bpm_last_error(bpm_plan plan) {
  return plan ? plan->err.c_str() : g_thread_error.c_str();
}

BPM_API bpm_status bpm_plan_create(const bpm_grid* grid, int n_channels, void* cuda_stream,
                                   bpm_plan* out) {
  BPM_NVTX();
  if (!grid || !out) return fail(nullptr, BPM_ERR_INVALID_ARG, "null grid or output pointer");
  *out = nullptr;
  const bpm_grid& g = *grid;
  if (n_channels < 1) return fail(nullptr, BPM_ERR_INVALID_ARG, "n_channels must be >= 1");
  if (g.nz < 1 || !(g.dx > 0) || !(g.dz > 0))
    return fail(nullptr, BPM_ERR_INVALID_ARG, "nz, dx and dz must be positive");
  if (g.split_order != 1 && g.split_order != 2 && g.split_order != 4)
    return fail(nullptr, BPM_ERR_UNSUPPORTED, "split_order must be 1, 2 or 4");
  if (g.split_order != 1 && g.dims != 2)
    return fail(nullptr, BPM_ERR_UNSUPPORTED, "Strang splitting is implemented for 2D plans");
  if (g.dims == 2) {
    if (g.ny != 1) return fail(nullptr, BPM_ERR_INVALID_ARG, "dims = 2 requires ny = 1");
    if (!is_pow2(g.nx) || g.nx < 256 || g.nx > 8192)
      return fail(nullptr, BPM_ERR_UNSUPPORTED, "nx must be a power of two in [256, 8192]");
  } else if (g.dims == 3) {
    if (!pass3d_supported(g.nx, g.ny))
      return fail(nullptr, BPM_ERR_UNSUPPORTED, "3D: nx and ny must be 256, 512 or 1024");
    if (!(g.dy > 0)) return fail(nullptr, BPM_ERR_INVALID_ARG, "3D: dy must be positive");
  } else {
    return fail(nullptr, BPM_ERR_INVALID_ARG, "dims must be 2 or 3");
  }
  const DeviceInfo& di = device_info();
  if (di.cc != 103 && di.sm_count > 0)
    return fail(nullptr, BPM_ERR_UNSUPPORTED, "libbpm is built for sm_103a (GB300) only");
  if (!di.ok) return fail(nullptr, BPM_ERR_CUDA, "no usable CUDA device");
  if (di.cc != 103)
    return fail(nullptr, BPM_ERR_UNSUPPORTED, "libbpm is built for sm_103a (GB300) only");

  auto p = std::make_unique<bpm_plan_s>();
  p->grid = g;
  p->n_ch = n_channels;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  p->plane = g.nx * g.ny;
  bpm_plan P = p.get();
  const size_t nf = size_t(n_channels) * p->plane;
  bpm_status st = BPM_OK;
  auto check = [&](cudaError_t e, const char* what) {
    if (st == BPM_OK && e != cudaSuccess) {
      st = (e == cudaErrorMemoryAllocation) ? fail(P, BPM_ERR_OOM, what) : cuda_fail(P, e, what);
      g_thread_error = P->err;
    }
  };
  check(dalloc(&p->cfield, size_t(g.nz) * p->plane), "alloc deformation field");
  if (g.dims == 3) check(dalloc(&p->cspan, size_t(g.nz) * g.ny), "alloc crystal extents");
  check(dalloc(&p->e0, nf), "alloc E0");
  check(dalloc(&p->eh, nf), "alloc Eh");
  const size_t sets = g.split_order == 4 ? 2 : 1;  // Eq. split-op order 4: two of each
  check(dalloc(&p->tables, sets * n_channels * 2 * g.nx), "alloc propagator tables");
  check(dalloc(&p->coef, sets * n_channels), "alloc coefficients");
  check(dalloc(&p->twiddle, size_t(g.nx)), "alloc twiddles");
  if (g.dims == 2) check(dalloc(&p->twiddle_t, size_t(g.nx)), "alloc thread-order twiddles");
  if (g.dims == 2) check(dalloc(&p->twiddle_p, 2 * size_t(g.nx)), "alloc paired twiddles");
  check(dalloc(&p->rev, size_t(g.nx)), "alloc spectrum order");
  check(dalloc(&p->gain, size_t(g.nx)), "alloc gain");
  check(dalloc(&p->omega, size_t(n_channels)), "alloc omega");
  check(dalloc(&p->weight, size_t(n_channels)), "alloc weights");
  check(dalloc(&p->inc_norm, size_t(n_channels)), "alloc norms");
  check(dalloc(&p->refl, size_t(n_channels)), "alloc R");
  check(dalloc(&p->trans, size_t(n_channels)), "alloc T");
  check(dalloc(&p->eh_time, nf), "alloc time response");
  check(dalloc(&p->dflag, size_t(4)), "alloc status");
  if (g.dims == 3) {
    check(dalloc(&p->gcorr, size_t(n_channels) * 2 * g.nx), "alloc curvature factors");
    check(dalloc(&p->spec, 2 * nf), "alloc spectrum buffers");
    check(dalloc(&p->twy, size_t(g.ny)), "alloc y twiddles");
    check(dalloc(&p->twx3, size_t(g.nx)), "alloc x twiddles");
    check(dalloc(&p->qy, size_t(g.ny)), "alloc qy table");
  }
  if (st != BPM_OK) {
    free_plan_buffers(P);
    return st;
  }
  const FftConsts& fc = fft_consts(g.nx);
  // The natural table feeds the kernels that keep twiddles in registers; the
  // thread-ordered one those that read them from memory (Nx = 8192, L2 form).
  check(cudaMemcpyAsync(p->twiddle, fc.tw.data(), sizeof(float2) * g.nx, cudaMemcpyHostToDevice,
                        p->stream),
        "upload twiddles");
  std::vector<float2> tw_ord, tw_pair;
  if (g.dims == 2) {
    tw_ord = twiddle_order(g.nx);
    check(cudaMemcpyAsync(p->twiddle_t, tw_ord.data(), sizeof(float2) * tw_ord.size(),
                          cudaMemcpyHostToDevice, p->stream),
          "upload thread-order twiddles");
    tw_pair = twiddle_pairs(g.nx);
    check(cudaMemcpyAsync(p->twiddle_p, tw_pair.data(), sizeof(float2) * tw_pair.size(),
                          cudaMemcpyHostToDevice, p->stream),
          "upload paired twiddles");
  }
  check(cudaMemcpyAsync(p->rev, fc.rev.data(), sizeof(int) * g.nx, cudaMemcpyHostToDevice,
                        p->stream),
        "upload spectrum order");
  check(cudaMemcpyAsync(p->gain, fc.gain.data(), sizeof(double) * g.nx, cudaMemcpyHostToDevice,
                        p->stream),
        "upload gain");
  check(cudaMemsetAsync(p->dflag, 0, sizeof(int) * 4, p->stream), "clear status");
  std::vector<float2> qyt;
  if (g.dims == 3) {
    const FftConsts& fy = fft_consts(g.ny);
    qyt.resize(g.ny);
    for (int py = 0; py < g.ny; ++py) {
      const int m = fy.rev[py];
      const int mm = m < g.ny / 2 ? m : m - g.ny;
      const double q = 2.0 * kPiHost * double(mm) / (double(g.ny) * g.dy);
      // stored at k T + t for position py = 16 t + k (coalesced in the column pass)
      const int Ty = g.ny / 16;
      qyt[(py % 16) * Ty + py / 16] = make_float2(float(q * q), float(1.0 / fy.gain[py] - 1.0));
    }
    const std::vector<float2> twy = twiddle_order(g.ny), twx = twiddle_order(g.nx);
    check(cudaMemcpyAsync(p->twy, twy.data(), sizeof(float2) * twy.size(), cudaMemcpyHostToDevice,
                          p->stream),
          "upload y twiddles");
    check(cudaMemcpyAsync(p->twx3, twx.data(), sizeof(float2) * twx.size(),
                          cudaMemcpyHostToDevice, p->stream),
          "upload x twiddles");
    check(cudaMemcpyAsync(p->qy, qyt.data(), sizeof(float2) * g.ny, cudaMemcpyHostToDevice,
                          p->stream),
          "upload qy table");
  }
  check(cudaStreamSynchronize(p->stream), "plan upload");
  if (st != BPM_OK) {
    free_plan_buffers(P);
    return st;
  }
  const int maxg = march_max_group(g.nx);
  const long long full = (n_channels + maxg - 1) / maxg;
  p->group = (maxg > 1 && full >= di.sm_count) ? maxg : 1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(g, n_channels));
    if (it != g_tune.end() &&
        launch_valid(g, it->second.form, it->second.group, it->second.row_threads)) {
      p->form = it->second.form;
      p->group = it->second.group;
      p->row_threads = it->second.row_threads;
    }
  }
  apply_launch(p.get());
  p->bytes = plan_bytes(g, n_channels);
  *out = p.release();
  return BPM_OK;
}

BPM_API bpm_status bpm_set_crystal(bpm_plan p, double chi0_re, double chi0_im, double chih_re,
                                   double chih_im, double chihbar_re, double chihbar_im,
                                   double theta_B, double lambda_B, double x_surface,
                                   double thickness, const double* u_field, int u_on_device) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!(theta_B >= 0.0) || theta_B >= 85.0 * kPiHost / 180.0)
    return fail(p, BPM_ERR_INVALID_ARG, "theta_B must lie in [0, 85) degrees");
  if (!(lambda_B > 0.0) || !(thickness >= 0.0))
    return fail(p, BPM_ERR_INVALID_ARG, "lambda_B must be positive, thickness non-negative");
  SetupArgs& sa = p->sa;
  sa.nx = p->grid.nx;
  sa.ny = p->grid.ny;
  sa.nz = p->grid.nz;
  sa.n_ch = p->n_ch;
  sa.dims = p->grid.dims;
  sa.dx = p->grid.dx;
  sa.dy = p->grid.dy;
  sa.dz = p->grid.dz;
  sa.h = 4.0 * kPiHost * std::sin(theta_B) / lambda_B;
  sa.chi0_re = chi0_re;
  sa.chi0_im = chi0_im;
  sa.chih_re = chih_re;
  sa.chih_im = chih_im;
  sa.chihb_re = chihbar_re;
  sa.chihb_im = chihbar_im;
  sa.zassenhaus = p->grid.zassenhaus ? 1 : 0;
  sa.coupling_frac = p->grid.split_order == 2 ? 0.5 : 1.0;
  sa.split_order = p->grid.split_order;
  sa.x_surface = x_surface;
  sa.x_end = x_surface + thickness;
  if (!p->have_geometry) {
    sa.tan_psi = 0.0;
    sa.z_begin = -HUGE_VAL;
    sa.z_end = HUGE_VAL;
  }
  const size_t cells = size_t(p->grid.nz) * p->plane;
  const double* u_dev = nullptr;
  if (u_field) {
    if (u_on_device) {
      u_dev = u_field;
    } else {
      if (!p->u_tmp) {
        BPM_CUDA(p, dalloc(&p->u_tmp, cells), "alloc displacement upload");
        p->bytes += cells * sizeof(double);
      }
      BPM_CUDA(p, cudaMemcpyAsync(p->u_tmp, u_field, cells * sizeof(double),
                                  cudaMemcpyHostToDevice, p->stream),
               "upload displacement");
      u_dev = p->u_tmp;
    }
  }
  p->u_dev = u_dev;
  BPM_CUDA(p, enqueue_crystal(p), "deformation kernel");
  p->have_crystal = true;
  p->have_pulse = false;
  p->time_valid = false;
  return BPM_OK;
}

BPM_API bpm_status bpm_set_geometry(bpm_plan p, double tan_psi, double z_begin, double z_end) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!(std::fabs(tan_psi) < 1e3) || !(z_begin < z_end))
    return fail(p, BPM_ERR_INVALID_ARG, "need |tan_psi| < 1e3 and z_begin < z_end");
  p->sa.tan_psi = tan_psi;
  p->sa.z_begin = z_begin;
  p->sa.z_end = z_end;
  p->have_geometry = true;
  if (p->have_crystal) BPM_CUDA(p, enqueue_crystal(p), "deformation kernel");
  return BPM_OK;
}

BPM_API bpm_status bpm_set_crystal_shape(bpm_plan p, const unsigned char* mask, int on_device) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!mask) {
    p->sa.mask = nullptr;  // back to the crystal's boundaries (the copy is kept for reuse)
  } else {
    const size_t cells = size_t(p->grid.nz) * p->plane;
    if (!p->mask) {
      BPM_CUDA(p, dalloc(&p->mask, cells), "alloc crystal mask");
      p->bytes += cells;
    }
    BPM_CUDA(p, cudaMemcpyAsync(p->mask, mask, cells,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                p->stream),
             "upload crystal mask");
    if (!on_device) BPM_CUDA(p, cudaStreamSynchronize(p->stream), "upload crystal mask");
    p->sa.mask = p->mask;
  }
  if (p->have_crystal) BPM_CUDA(p, enqueue_crystal(p), "deformation kernel");
  return BPM_OK;
}

BPM_API bpm_status bpm_set_pulse(bpm_plan p, const double* omega, const double* weight_re_im,
                                 double theta_i, double x0, double w0, double zx, double zR) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!omega || !weight_re_im) return fail(p, BPM_ERR_INVALID_ARG, "null omega or weights");
  if (!p->have_crystal) return fail(p, BPM_ERR_STATE, "bpm_set_crystal must come first");
  if (!(w0 > 0.0)) return fail(p, BPM_ERR_INVALID_ARG, "w0 must be positive");
  for (int i = 0; i < p->n_ch; ++i)
    if (!(omega[i] > 0.0)) return fail(p, BPM_ERR_INVALID_ARG, "omega must be positive");
  for (int i = 0; i < p->n_ch; ++i)
    if (!(omega[i] / 299792458.0 > 0.5 * p->sa.h))
      return fail(p, BPM_ERR_INVALID_ARG, "a channel has k <= h/2 (no Bragg solution)");
  if (p->grid.split_order == 4) {
    // the propagation 1-2t < 0 runs backwards: an evanescent mode would grow by
    // exp((2t-1) dz kappa) before the forward steps damp it; require every
    // mode of the grid to propagate, |q| + h/2 < k
    const double qmax = kPiHost / p->grid.dx + 0.5 * p->sa.h;
    for (int i = 0; i < p->n_ch; ++i)
      if (!(omega[i] / 299792458.0 > qmax))
        return fail(p, BPM_ERR_UNSUPPORTED, "fourth-order splitting needs propagating modes only");
  }
  if (p->grid.dims == 3) {
    // the column pass expands sqrt(K^2 - qy^2) - K to second order in
    // c = dz qy^2 / (2K): require every K^2 > 0 and c < 1e-3 (terms dropped < 2e-10)
    const double qxm = kPiHost / p->grid.dx + 0.5 * p->sa.h;
    const double qym = kPiHost / p->grid.dy;
    for (int i = 0; i < p->n_ch; ++i) {
      const double k = omega[i] / 299792458.0;
      const double K2 = k * k - qxm * qxm;
      if (!(K2 > 0.0) || p->grid.dz * qym * qym / (2.0 * std::sqrt(K2)) > 1e-3)
        return fail(p, BPM_ERR_UNSUPPORTED, "3D grid too fine for the paraxial y correction");
    }
  }
  p->sa.theta_i = theta_i;
  p->sa.x0 = x0;
  p->sa.w0 = w0;
  p->sa.zx = zx;
  p->sa.zR = zR;
  if (!p->sharded) p->domega = p->n_ch > 1 ? omega[1] - omega[0] : 1.0;
  BPM_CUDA(p, cudaMemcpyAsync(p->omega, omega, sizeof(double) * p->n_ch, cudaMemcpyHostToDevice,
                              p->stream),
           "upload omega");
  BPM_CUDA(p, cudaMemcpyAsync(p->weight, weight_re_im, sizeof(double2) * p->n_ch,
                              cudaMemcpyHostToDevice, p->stream),
           "upload weights");
  BPM_CUDA(p, enqueue_pulse(p), "pulse setup kernels");
  p->have_pulse = true;
  return BPM_OK;
}

BPM_API bpm_status bpm_set_channel_shard(bpm_plan p, int first, int n_total, double d_omega) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (first < 0 || n_total < p->n_ch || first + p->n_ch > n_total)
    return fail(p, BPM_ERR_INVALID_ARG, "shard must lie within [0, n_total)");
  if (!(d_omega > 0.0) || !std::isfinite(d_omega))
    return fail(p, BPM_ERR_INVALID_ARG, "d_omega must be positive and finite");
  if (p->z != 0) return fail(p, BPM_ERR_STATE, "set the shard before the march starts");
  const int rows = std::max(p->shard_total, p->n_ch);
  if (n_total > rows) {
    double2* t = nullptr;
    BPM_CUDA(p, dalloc(&t, size_t(n_total) * p->plane), "alloc time response");
    cudaFree(p->eh_time);
    p->eh_time = t;
    p->bytes += size_t(n_total - rows) * p->plane * sizeof(double2);
  }
  p->sharded = true;
  p->shard_first = first;
  p->shard_total = n_total;
  p->domega = d_omega;
  p->time_valid = false;
  return BPM_OK;
}

BPM_API bpm_status bpm_set_fields(bpm_plan p, const void* e0, const void* eh, int z_step,
                                  int on_device) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!e0 || !eh) return fail(p, BPM_ERR_INVALID_ARG, "null field pointer");
  if (!p->have_pulse) return fail(p, BPM_ERR_STATE, "bpm_set_pulse must come first");
  if (z_step < 0 || z_step > p->grid.nz) return fail(p, BPM_ERR_INVALID_ARG, "z_step out of range");
  const size_t bytes = sizeof(float2) * size_t(p->n_ch) * p->plane;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  BPM_CUDA(p, cudaMemcpyAsync(p->e0, e0, bytes, kind, p->stream), "set E0");
  BPM_CUDA(p, cudaMemcpyAsync(p->eh, eh, bytes, kind, p->stream), "set Eh");
  if (!on_device) BPM_CUDA(p, cudaStreamSynchronize(p->stream), "set fields");
  p->z = z_step;
  p->time_valid = false;
  return BPM_OK;
}

BPM_API bpm_status bpm_run(bpm_plan p, int n_steps) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!p->have_pulse) return fail(p, BPM_ERR_STATE, "bpm_set_pulse must come first");
  if (n_steps < 0 || p->z + n_steps > p->grid.nz)
    return fail(p, BPM_ERR_INVALID_ARG, "n_steps must keep z within [0, nz]");
  MarchArgs a;
  a.tables = p->tables;
  a.coef = p->coef;
  a.twiddle = p->twiddle;
  a.twiddle_t = p->twiddle_t;
  a.twiddle_p = p->twiddle_p;
  a.cfield = p->cfield;
  a.e0 = p->e0;
  a.eh = p->eh;
  a.inc_norm = p->inc_norm;
  a.refl = p->refl;
  a.trans = p->trans;
  a.n_ch = p->n_ch;
  a.z0 = p->z;
  a.n_steps = n_steps;
  a.split_order = p->grid.split_order;
  int launches = 0, march_launches = 0;
  if (p->timing) BPM_CUDA(p, cudaEventRecord(p->ev0, p->stream), "timing event");
  if (p->grid.dims == 2) {
    if (p->form == 1 && a.split_order == 1)
      BPM_CUDA(p, launch_march_l2(p->grid.nx, p->group, p->blocks, a, p->stream), "march kernel");
    else if ((p->form == 2 && a.split_order != 2) || (p->form == 3 && a.split_order <= 2))
      BPM_CUDA(p, launch_march_parked(p->grid.nx, p->form, p->blocks, a, p->stream),
               "march kernel");
    else
      BPM_CUDA(p, launch_march(p->grid.nx, p->group, p->blocks, a, p->stream), "march kernel");
    march_launches = 1;
  } else if (n_steps > 0) {
    Pass3DArgs pa;
    pa.e0 = p->e0;
    pa.eh = p->eh;
    pa.s0 = p->spec;
    pa.sh = p->spec + size_t(p->n_ch) * p->plane;
    pa.cfield = p->cfield;
    pa.cspan = p->cspan;
    pa.coef = p->coef;
    pa.twx = p->twx3;
    pa.twy = p->twy;
    pa.anchor = p->tables;
    pa.gcorr = p->gcorr;
    pa.qy = p->qy;
    pa.nx = p->grid.nx;
    pa.ny = p->grid.ny;
    pa.z = p->z;
    // form 2 streams the MODE-1 row passes; its first and last row passes
    // (once a run) are the plain ones with 256-thread tiles
    const int plain_rt = p->form == 2 ? 256 : p->row_threads;
    const int sms = device_info().sm_count;
    BPM_CUDA(p, launch_row_pass(0, plain_rt, pa, p->n_ch, p->stream), "row pass");
    march_launches = 1;
    for (int s = 0; s < n_steps; ++s) {
      pa.z = p->z + s;
      BPM_CUDA(p, launch_col_pass(p->form, pa, p->n_ch, sms, p->dflag + 1, p->stream),
               "column pass");
      if (s == n_steps - 1)
        BPM_CUDA(p, launch_row_pass(2, plain_rt, pa, p->n_ch, p->stream), "row pass");
      else if (p->form == 2)
        BPM_CUDA(p, launch_row_pass_tma(p->row_threads, pa, p->n_ch, sms, p->dflag + 1, p->stream),
                 "row pass");
      else
        BPM_CUDA(p, launch_row_pass(1, plain_rt, pa, p->n_ch, p->stream), "row pass");
      march_launches += 2;
    }
  }
  launches += march_launches;
  if (p->timing) BPM_CUDA(p, cudaEventRecord(p->ev1, p->stream), "timing event");
  if (p->grid.dims == 3) {
    BPM_CUDA(p, launch_reduce3d(p->e0, p->eh, p->plane, p->n_ch, p->inc_norm, p->refl, p->trans,
                                p->stream),
             "reflectivity");
    ++launches;
  }
  p->z += n_steps;
  p->time_valid = false;
  if (p->z == p->grid.nz) {
    BPM_CUDA(p, launch_omega_to_t(time_rows(p), p->shard_first, p->n_ch, p->plane, p->domega,
                                  p->eh, p->eh_time, p->stream),
             "omega-to-t kernel");
    ++launches;
    p->time_valid = true;
  }
  p->stats.launches = launches;
  p->stats.march_launches = march_launches;
  return BPM_OK;
}

BPM_API bpm_status bpm_set_stream(bpm_plan p, void* cuda_stream) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  cudaStream_t ns = static_cast<cudaStream_t>(cuda_stream);
  if (ns == p->stream) return BPM_OK;
  cudaEvent_t ev;
  BPM_CUDA(p, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
  cudaError_t e = cudaEventRecord(ev, p->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ns, ev, 0);
  cudaEventDestroy(ev);
  BPM_CUDA(p, e, "stream switch");
  p->stream = ns;
  return BPM_OK;
}

BPM_API bpm_status bpm_sync(bpm_plan p) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  BPM_CUDA(p, cudaStreamSynchronize(p->stream), "stream synchronize");
  if (p->grid.dims == 3 && p->form >= 1) {
    // status word of the streamed passes: a bounded wait that gave up
    int st = 0;
    BPM_CUDA(p, cudaMemcpy(&st, p->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost), "status");
    if (st != 0) {
      BPM_CUDA(p, cudaMemset(p->dflag + 1, 0, sizeof(int)), "clear status");
      return fail(p, BPM_ERR_TIMEOUT, "3D streamed pass: a bulk-copy wait gave up");
    }
  }
  return BPM_OK;
}

BPM_API bpm_status bpm_fetch_fields(bpm_plan p, int which, void* dst, size_t bytes,
                                    int dst_on_device) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!dst) return fail(p, BPM_ERR_INVALID_ARG, "null destination");
  const size_t n = size_t(p->n_ch) * p->plane;
  const void* src = nullptr;
  size_t need = 0;
  switch (which) {
    case BPM_FIELD_E0: src = p->e0; need = n * sizeof(float2); break;
    case BPM_FIELD_EH: src = p->eh; need = n * sizeof(float2); break;
    case BPM_FIELD_EH_TIME:
      if (!p->time_valid) return fail(p, BPM_ERR_STATE, "time response needs the march at nz");
      src = p->eh_time;
      need = size_t(time_rows(p)) * p->plane * sizeof(double2);
      break;
    default: return fail(p, BPM_ERR_INVALID_ARG, "unknown field selector");
  }
  if (bytes != need) return fail(p, BPM_ERR_INVALID_ARG, "destination size mismatch");
  BPM_CUDA(p, cudaMemcpyAsync(dst, src, need,
                              dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              p->stream),
           "fetch fields");
  BPM_CUDA(p, cudaStreamSynchronize(p->stream), "fetch fields");
  return BPM_OK;
}

BPM_API bpm_status bpm_fetch_reflectivity(bpm_plan p, double* R, double* T, double* R_int) {
  BPM_NVTX();
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!p->have_pulse) return fail(p, BPM_ERR_STATE, "no pulse set");
  std::vector<double> r(p->n_ch), t(p->n_ch);
  BPM_CUDA(p, cudaMemcpyAsync(r.data(), p->refl, sizeof(double) * p->n_ch, cudaMemcpyDeviceToHost,
                              p->stream),
           "fetch R");
  BPM_CUDA(p, cudaMemcpyAsync(t.data(), p->trans, sizeof(double) * p->n_ch,
                              cudaMemcpyDeviceToHost, p->stream),
           "fetch T");
  BPM_CUDA(p, cudaStreamSynchronize(p->stream), "fetch reflectivity");
  if (R) std::memcpy(R, r.data(), sizeof(double) * p->n_ch);
  if (T) std::memcpy(T, t.data(), sizeof(double) * p->n_ch);
  if (R_int) {
    double s = 0.0;
    for (double v : r) s += v;
    *R_int = p->domega * s;
  }
  return BPM_OK;
}

BPM_API bpm_status bpm_set_timing(bpm_plan p, int enable) {
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (enable && !p->ev0) {
    BPM_CUDA(p, cudaEventCreate(&p->ev0), "create event");
    BPM_CUDA(p, cudaEventCreate(&p->ev1), "create event");
  }
  p->timing = enable != 0;
  return BPM_OK;
}

BPM_API bpm_status bpm_get_stats(bpm_plan p, bpm_stats* out) {
  if (!p || !out) return fail(p, BPM_ERR_INVALID_ARG, "null argument");
  p->stats.march_ms = 0.0;
  if (p->timing && p->ev0) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, p->ev0, p->ev1);
    if (e == cudaErrorNotReady) return fail(p, BPM_ERR_STATE, "call bpm_sync before bpm_get_stats");
    if (e == cudaSuccess) p->stats.march_ms = ms;
  }
  *out = p->stats;
  return BPM_OK;
}

BPM_API bpm_status bpm_get_launch(bpm_plan p, bpm_launch* out) {
  if (!p || !out) return fail(p, BPM_ERR_INVALID_ARG, "null argument");
  out->form = p->form;
  out->channels_per_block = p->group;
  out->row_threads = p->row_threads;
  out->ms = 0.f;
  return BPM_OK;
}

BPM_API bpm_status bpm_set_launch(bpm_plan p, const bpm_launch* f) {
  BPM_NVTX();
  if (!p || !f) return fail(p, BPM_ERR_INVALID_ARG, "null argument");
  if (!launch_valid(p->grid, f->form, f->channels_per_block, f->row_threads))
    return fail(p, BPM_ERR_INVALID_ARG, "launch form not available for this plan");
  p->form = f->form;
  p->group = f->channels_per_block;
  p->row_threads = f->row_threads;
  apply_launch(p);
  return BPM_OK;
}

namespace {

std::string device_tag() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return "unknown";
  std::string name(prop.name);
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  return name + "/" + std::to_string(prop.multiProcessorCount);
}

// Times `steps` steps of plan p in its current form: one warm-up, median of three.
bpm_status time_form(bpm_plan p, int steps, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  float t[3];
  for (int r = -1; r < 3; ++r) {
    p->z = 0;
    BPM_CUDA(p, cudaEventRecord(e0, p->stream), "tune event");
    const bpm_status st = bpm_run(p, steps);
    if (st != BPM_OK) return st;
    BPM_CUDA(p, cudaEventRecord(e1, p->stream), "tune event");
    BPM_CUDA(p, cudaEventSynchronize(e1), "tune sync");
    if (r >= 0) BPM_CUDA(p, cudaEventElapsedTime(&t[r], e0, e1), "tune time");
  }
  std::sort(t, t + 3);
  *ms = t[1];
  return BPM_OK;
}

}  // namespace

BPM_API bpm_status bpm_tune(const bpm_grid* grid, int n_channels, int steps, bpm_launch* best,
                            bpm_launch* all, int max_all, int* n_all) {
  BPM_NVTX();
  if (!grid || !best || n_channels < 1 || steps < 1 || (all && max_all < 0))
    return fail(nullptr, BPM_ERR_INVALID_ARG, "bpm_tune: bad arguments");
  bpm_grid g = *grid;
  g.nz = steps;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(nullptr, BPM_ERR_CUDA, "bpm_tune: stream");
  bpm_plan p = nullptr;
  bpm_status st = bpm_plan_create(&g, n_channels, s, &p);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<bpm_launch> meas;
  if (st == BPM_OK) {
    // synthetic content: a slab over the second quarter of x (vacuum elsewhere,
    // as in Bragg geometry) and a Gaussian beam in front of it, channels around
    // the Bragg condition of the 45-degree reflection at lambda = 1.26116 A
    const double lam = 1.26116e-10, thb = 0.25 * kPiHost, width = g.nx * g.dx;
    st = bpm_set_crystal(p, -1.0e-5, 1.0e-8, -4.0e-6, 5.0e-9, -4.0e-6, 5.0e-9, thb, lam,
                         0.25 * width + 0.5 * g.dx, 0.25 * width, nullptr, 0);
    std::vector<double> omega(n_channels), wgt(2 * size_t(n_channels), 0.0);
    const double wb = 2.0 * kPiHost * 299792458.0 / lam;
    for (int i = 0; i < n_channels; ++i) {
      omega[i] = wb * (1.0 + 1.0e-5 + 8.0e-5 * (double(i) / n_channels - 0.5));
      wgt[2 * size_t(i)] = 1.0;
    }
    const double w0 = width / 32.0;
    if (st == BPM_OK)
      st = bpm_set_pulse(p, omega.data(), wgt.data(), thb, width / 8.0, w0, 0.0,
                         kPiHost * w0 * w0 / lam);
    if (st == BPM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
      st = fail(nullptr, BPM_ERR_CUDA, "bpm_tune: events");
    std::vector<bpm_launch> cand;
    if (g.dims == 3) {
      cand.push_back(bpm_launch{0, 1, 256, 0.f});
      cand.push_back(bpm_launch{0, 1, 512, 0.f});
      cand.push_back(bpm_launch{1, 1, 256, 0.f});
      cand.push_back(bpm_launch{1, 1, 512, 0.f});
      for (int rt : {128, 256})
        if (launch_valid(g, 2, 1, rt)) cand.push_back(bpm_launch{2, 1, rt, 0.f});
    } else {
      const int maxg = march_max_group(g.nx);
      cand.push_back(bpm_launch{0, 1, 256, 0.f});
      if (maxg > 1) cand.push_back(bpm_launch{0, maxg, 256, 0.f});
      if (launch_valid(g, 1, maxg, 256)) cand.push_back(bpm_launch{1, maxg, 256, 0.f});
      if (launch_valid(g, 2, 1, 256)) cand.push_back(bpm_launch{2, 1, 256, 0.f});
      if (launch_valid(g, 3, 1, 256)) cand.push_back(bpm_launch{3, 1, 256, 0.f});
      if (launch_valid(g, 3, 2, 256)) cand.push_back(bpm_launch{3, 2, 256, 0.f});
    }
    for (size_t i = 0; st == BPM_OK && i < cand.size(); ++i) {
      st = bpm_set_launch(p, &cand[i]);
      if (st == BPM_OK) st = time_form(p, steps, e0, e1, &cand[i].ms);
      if (st == BPM_OK) meas.push_back(cand[i]);
    }
  }
  const std::string err = st == BPM_OK ? std::string() : std::string(bpm_last_error(p));
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  bpm_plan_destroy(p);
  cudaStreamDestroy(s);
  if (st != BPM_OK) return fail(nullptr, st, "bpm_tune: " + err);
  size_t b = 0;
  for (size_t i = 1; i < meas.size(); ++i)
    if (meas[i].ms < meas[b].ms) b = i;
  *best = meas[b];
  if (all)
    for (int i = 0; i < int(meas.size()) && i < max_all; ++i) all[i] = meas[size_t(i)];
  if (n_all) *n_all = int(meas.size());
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TuneEntry te;
  te.form = best->form;
  te.group = best->channels_per_block;
  te.row_threads = best->row_threads;
  te.ms = best->ms;
  g_tune[tune_key(*grid, n_channels)] = te;
  return BPM_OK;
}

BPM_API bpm_status bpm_tune_save(const char* path) {
  BPM_NVTX();
  if (!path) return fail(nullptr, BPM_ERR_INVALID_ARG, "null path");
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(nullptr, BPM_ERR_INVALID_ARG, std::string("cannot write ") + path);
  const std::string tag = device_tag();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::fprintf(f, "# libbpm launch forms: device dims nx ny split_order channels form "
                  "channels_per_block row_threads ms\n");
  for (const auto& kv : g_tune) {
    const TuneKey& k = kv.first;
    const TuneEntry& e = kv.second;
    std::fprintf(f, "%s %d %d %d %d %d %d %d %d %.6f\n", tag.c_str(), std::get<0>(k),
                 std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), e.form, e.group,
                 e.row_threads, double(e.ms));
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? BPM_OK : fail(nullptr, BPM_ERR_INVALID_ARG, std::string("cannot write ") + path);
}

BPM_API bpm_status bpm_tune_load(const char* path, int* n_loaded) {
  BPM_NVTX();
  if (!path) return fail(nullptr, BPM_ERR_INVALID_ARG, "null path");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(nullptr, BPM_ERR_INVALID_ARG, std::string("cannot read ") + path);
  const std::string tag = device_tag();
  std::map<TuneKey, TuneEntry> add;
  char line[512];
  bool bad = false;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    char dev[256];
    int d, nx, ny, so, nch, form, grp, rt;
    double ms;
    if (std::sscanf(line, "%255s %d %d %d %d %d %d %d %d %lf", dev, &d, &nx, &ny, &so, &nch, &form,
                    &grp, &rt, &ms) != 10) {
      bad = true;
      break;
    }
    if (tag != dev) continue;
    bpm_grid g{};
    g.dims = d;
    g.nx = nx;
    g.ny = ny;
    g.split_order = so;
    if (!launch_valid(g, form, grp, rt)) {
      bad = true;
      break;
    }
    TuneEntry e;
    e.form = form;
    e.group = grp;
    e.row_threads = rt;
    e.ms = float(ms);
    add[TuneKey(d, nx, ny, so, nch)] = e;
  }
  std::fclose(f);
  if (bad) return fail(nullptr, BPM_ERR_INVALID_ARG, std::string("malformed tune file ") + path);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : add) g_tune[kv.first] = kv.second;
  if (n_loaded) *n_loaded = int(add.size());
  return BPM_OK;
}

BPM_API void bpm_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

BPM_API void bpm_plan_destroy(bpm_plan p) {
  BPM_NVTX();
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  free_plan_buffers(p);
  delete p;
}

}  // extern "C"

// ===========================================================================
// Batches: many plans marched by one persistent work-queue launch per round.
// ===========================================================================
namespace {

struct BatchEntry {
  bpm_plan plan = nullptr;
  cudaStream_t orig_stream = nullptr;  // restored when the ticket completes or is cancelled
  uint64_t ticket = 0;
  bool finishing = false;  // finalize enqueued, done event recorded
  bool cancelled = false;
  cudaEvent_t done = nullptr;
};

// Host staging of one round's descriptors (pinned) and its device copy.
struct RoundSlot {
  MarchArgs* h_plans = nullptr;
  BatchItem* h_items = nullptr;
  MarchArgs* d_plans = nullptr;
  BatchItem* d_items = nullptr;
  int* d_counter = nullptr;  // [kQueueCount]: one counter per queue
  int cap_plans = 0, cap_items = 0;
  cudaEvent_t free_ev = nullptr;  // recorded after the round's kernels
  bool used = false;
};

}  // namespace

struct bpm_batch_s {
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // Nx = 8192 kernel runs here, forked from stream
  cudaStream_t cap = nullptr;   // graph capture stream (the caller's may be the legacy stream)
  cudaEvent_t fork = nullptr, join = nullptr;
  size_t budget = 0, used = 0;
  uint64_t next_ticket = 1;
  std::vector<BatchEntry> entries;
  std::map<uint64_t, int> finished;  // ticket -> 1 done, 2 cancelled
  RoundSlot slots[3];
  int next_slot = 0;
  RoundSlot graph_slot;
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_key = 0;
  std::string err = "no error";
  int rounds = 0;
  int last_items[2] = {0, 0};
  int max_blocks = 0;  // SM cap of the persistent launches (0: every SM)
  int graph_kernels = 0;  // kernel nodes of the captured graph
};

namespace {

bpm_status bfail(bpm_batch b, bpm_status s, const std::string& msg) {
  if (b) b->err = msg;
  g_thread_error = msg;
  return s;
}

#define BPM_BCUDA(b, call, what)                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? BPM_ERR_OOM : BPM_ERR_CUDA, \
                   std::string(what) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

// Growing a slot frees its old buffers, which synchronizes the device; the
// first reservation is sized (256 plans, 16384 items: ~0.3 MB) so that a
// server's rounds never grow one.
cudaError_t slot_reserve(RoundSlot& r, int n_plans, int n_items) {
  cudaError_t e = cudaSuccess;
  if (n_plans > r.cap_plans) {
    if (r.h_plans) cudaFreeHost(r.h_plans);
    if (r.d_plans) cudaFree(r.d_plans);
    r.cap_plans = std::max(n_plans * 2, 256);
    if ((e = cudaMallocHost(&r.h_plans, sizeof(MarchArgs) * r.cap_plans)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&r.d_plans, sizeof(MarchArgs) * r.cap_plans)) != cudaSuccess) return e;
  }
  if (n_items > r.cap_items) {
    if (r.h_items) cudaFreeHost(r.h_items);
    if (r.d_items) cudaFree(r.d_items);
    r.cap_items = std::max(n_items * 2, 16384);
    if ((e = cudaMallocHost(&r.h_items, sizeof(BatchItem) * r.cap_items)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&r.d_items, sizeof(BatchItem) * r.cap_items)) != cudaSuccess) return e;
  }
  if (!r.d_counter && (e = cudaMalloc(&r.d_counter, kQueueCount * sizeof(int))) != cudaSuccess)
    return e;
  if (!r.free_ev && (e = cudaEventCreateWithFlags(&r.free_ev, cudaEventDisableTiming)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

void slot_free(RoundSlot& r) {
  if (r.h_plans) cudaFreeHost(r.h_plans);
  if (r.h_items) cudaFreeHost(r.h_items);
  if (r.d_plans) cudaFree(r.d_plans);
  if (r.d_items) cudaFree(r.d_items);
  if (r.d_counter) cudaFree(r.d_counter);
  if (r.free_ev) cudaEventDestroy(r.free_ev);
  r = RoundSlot();
}

MarchArgs march_args(bpm_plan p, int n_steps) {
  MarchArgs a;
  a.tables = p->tables;
  a.coef = p->coef;
  a.twiddle = p->twiddle;
  a.twiddle_t = p->twiddle_t;
  a.twiddle_p = p->twiddle_p;
  a.cfield = p->cfield;
  a.e0 = p->e0;
  a.eh = p->eh;
  a.inc_norm = p->inc_norm;
  a.refl = p->refl;
  a.trans = p->trans;
  a.n_ch = p->n_ch;
  a.z0 = p->z;
  a.n_steps = n_steps;
  a.split_order = p->grid.split_order;
  return a;
}

// Enqueue one round on b->stream using slot r: every active entry advances
// min(chunk, nz - z) steps; entries that reach nz get their time response and
// a completion event.  Items are ordered longest-first within each queue.
bpm_status enqueue_round(bpm_batch b, RoundSlot& r, int chunk) {
  std::vector<int> act;
  for (int i = 0; i < int(b->entries.size()); ++i) {
    const BatchEntry& e = b->entries[i];
    if (!e.finishing && !e.cancelled && e.plan->z < e.plan->grid.nz) act.push_back(i);
  }
  if (act.empty()) return BPM_OK;
  // queues by transform size and splitting order (BatchQueue), each sorted longest first
  struct Tmp {
    BatchItem it;
    double cost;
    int q;
  };
  std::vector<Tmp> tmp;
  std::vector<int> steps(act.size());
  for (int k = 0; k < int(act.size()); ++k) {
    bpm_plan p = b->entries[act[k]].plan;
    const int n = p->grid.nx;
    steps[k] = std::min(chunk, p->grid.nz - p->z);
    const int G = batch_item_channels(n, p->grid.split_order);
    const int q = batch_queue(n, p->grid.split_order);
    for (int c0 = 0; c0 < p->n_ch; c0 += G) {
      Tmp t;
      t.it = BatchItem{k, c0, n, 0};
      t.cost = double(steps[k]) * n * std::min(G, p->n_ch - c0) * std::log2(double(n));
      t.q = q;
      tmp.push_back(t);
    }
  }
  // launch rank of each queue: the longest items (Nx = 8192, every order) first,
  // then 4096, 2048 and 1024, then the resident small-N queues
  static constexpr int kOrder[kQueueCount] = {
      kQueueTm8192,   kQueueTm8192s2, kQueueBig4,     kQueueTm4096,   kQueueTm4096s2,
      kQueuePk4096s4, kQueueTm2048,   kQueueTm2048s2, kQueuePk2048s4, kQueueTm1024,
      kQueuePk1024s4, kQueueSmall,    kQueueSmall2,   kQueueSmall4};
  int rank[kQueueCount];
  for (int i = 0; i < kQueueCount; ++i) rank[kOrder[i]] = i;
  std::stable_sort(tmp.begin(), tmp.end(), [&rank](const Tmp& x, const Tmp& y) {
    return x.q != y.q ? rank[x.q] < rank[y.q] : x.cost > y.cost;
  });
  int cnt[kQueueCount] = {};
  for (auto& t : tmp) cnt[t.q]++;
  BPM_BCUDA(b, slot_reserve(r, int(act.size()), int(tmp.size())), "batch staging");
  if (r.used) BPM_BCUDA(b, cudaEventSynchronize(r.free_ev), "staging reuse");
  for (int k = 0; k < int(act.size()); ++k) r.h_plans[k] = march_args(b->entries[act[k]].plan, steps[k]);
  for (size_t i = 0; i < tmp.size(); ++i) r.h_items[i] = tmp[i].it;
  const DeviceInfo& di = device_info();
  const int sms = b->max_blocks > 0 ? std::min(b->max_blocks, di.sm_count) : di.sm_count;
  BPM_BCUDA(b, cudaMemcpyAsync(r.d_plans, r.h_plans, sizeof(MarchArgs) * act.size(),
                               cudaMemcpyHostToDevice, b->stream), "upload round");
  BPM_BCUDA(b, cudaMemcpyAsync(r.d_items, r.h_items, sizeof(BatchItem) * tmp.size(),
                               cudaMemcpyHostToDevice, b->stream), "upload items");
  BPM_BCUDA(b, cudaMemsetAsync(r.d_counter, 0, kQueueCount * sizeof(int), b->stream),
            "clear queues");
  // Queues run back to back, each on every SM (or the batch's cap) with its
  // blocks per SM: the Nx = 8192 items (the longest) first, then the smaller
  // ones; the idle tail is one item per queue.
  int off = 0;
  for (int i = 0; i < kQueueCount; ++i) {
    const int q = kOrder[i];
    if (cnt[q] > 0)
      BPM_BCUDA(b, launch_batch(r.d_plans, r.d_items + off, cnt[q], r.d_counter + q, q,
                                std::min(cnt[q], sms * batch_blocks_per_sm(q)), b->stream),
                "batch kernel");
    off += cnt[q];
  }
  const int n_big = cnt[kQueueTm8192] + cnt[kQueueTm8192s2] + cnt[kQueueBig4];
  const int n_small = int(tmp.size()) - n_big;
  BPM_BCUDA(b, cudaEventRecord(r.free_ev, b->stream), "round event");
  r.used = true;
  b->last_items[0] = n_small;
  b->last_items[1] = n_big;
  ++b->rounds;
  for (int k = 0; k < int(act.size()); ++k) {
    BatchEntry& e = b->entries[act[k]];
    bpm_plan p = e.plan;
    p->z += steps[k];
    p->time_valid = false;
    if (p->z == p->grid.nz) {
      BPM_BCUDA(b, launch_omega_to_t(time_rows(p), p->shard_first, p->n_ch, p->plane, p->domega,
                                     p->eh, p->eh_time, b->stream),
                "omega-to-t kernel");
      p->time_valid = true;
      if (!e.done) BPM_BCUDA(b, cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming), "event");
      BPM_BCUDA(b, cudaEventRecord(e.done, b->stream), "completion event");
      e.finishing = true;
    }
  }
  return BPM_OK;
}

}  // namespace

extern "C" {

BPM_API size_t bpm_plan_bytes(const bpm_grid* grid, int n_channels, int host_u) {
  if (!grid || n_channels < 1) return 0;
  size_t b = plan_bytes(*grid, n_channels);
  if (host_u) b += size_t(grid->nz) * grid->nx * (grid->dims == 3 ? grid->ny : 1) * sizeof(double);
  return b;
}

BPM_API bpm_status bpm_batch_create(size_t hbm_budget_bytes, void* cuda_stream, bpm_batch* out) {
  BPM_NVTX();
  if (!out) return bfail(nullptr, BPM_ERR_INVALID_ARG, "null output");
  *out = nullptr;
  const DeviceInfo& di = device_info();
  if (!di.ok || di.cc != 103)
    return bfail(nullptr, BPM_ERR_UNSUPPORTED, "libbpm needs a GB300 (sm_103a) device");
  auto b = std::make_unique<bpm_batch_s>();
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->budget = hbm_budget_bytes;
  BPM_BCUDA(b.get(), cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking), "side stream");
  BPM_BCUDA(b.get(), cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "capture stream");
  BPM_BCUDA(b.get(), cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  BPM_BCUDA(b.get(), cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming), "event");
  *out = b.release();
  return BPM_OK;
}

BPM_API bpm_status bpm_batch_submit(bpm_batch b, bpm_plan p, uint64_t* ticket) {
  BPM_NVTX();
  if (!b || !p || !ticket) return bfail(b, BPM_ERR_INVALID_ARG, "null argument");
  if (!p->have_pulse) return bfail(b, BPM_ERR_STATE, "plan needs crystal and pulse first");
  if (p->grid.dims != 2) return bfail(b, BPM_ERR_UNSUPPORTED, "batches take 2D plans");
  for (const auto& e : b->entries)
    if (e.plan == p) return bfail(b, BPM_ERR_STATE, "plan already in the batch");
  if (b->budget && b->used + p->bytes > b->budget)
    return bfail(b, BPM_ERR_OOM, "not admitted: HBM budget exhausted");
  BatchEntry e;
  e.orig_stream = p->stream;
  if (p->stream != b->stream) {
    // order the plan's setup work before the batch's rounds, then adopt the batch stream
    cudaEvent_t ev;
    BPM_BCUDA(b, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    BPM_BCUDA(b, cudaEventRecord(ev, p->stream), "event");
    BPM_BCUDA(b, cudaStreamWaitEvent(b->stream, ev, 0), "event wait");
    cudaEventDestroy(ev);
    p->stream = b->stream;
  }
  e.plan = p;
  e.ticket = b->next_ticket++;
  b->entries.push_back(e);
  b->used += p->bytes;
  *ticket = e.ticket;
  return BPM_OK;
}

BPM_API bpm_status bpm_batch_step(bpm_batch b, int chunk_steps) {
  BPM_NVTX();
  if (!b) return bfail(nullptr, BPM_ERR_INVALID_ARG, "null batch");
  if (chunk_steps < 1) return bfail(b, BPM_ERR_INVALID_ARG, "chunk_steps must be >= 1");
  RoundSlot& r = b->slots[b->next_slot];
  b->next_slot = (b->next_slot + 1) % 3;
  return enqueue_round(b, r, chunk_steps);
}

BPM_API bpm_status bpm_batch_run(bpm_batch b) { return bpm_batch_step(b, 1 << 30); }

BPM_API bpm_status bpm_batch_poll(bpm_batch b, uint64_t ticket, int* done) {
  BPM_NVTX();
  if (!b || !done) return bfail(b, BPM_ERR_INVALID_ARG, "null argument");
  *done = 0;
  auto f = b->finished.find(ticket);
  if (f != b->finished.end()) {
    if (f->second == 2) return bfail(b, BPM_ERR_CANCELLED, "ticket was cancelled");
    *done = 1;
    return BPM_OK;
  }
  for (size_t i = 0; i < b->entries.size(); ++i) {
    BatchEntry& e = b->entries[i];
    if (e.ticket != ticket) continue;
    if (!e.finishing) return BPM_OK;
    cudaError_t q = cudaEventQuery(e.done);
    if (q == cudaErrorNotReady) return BPM_OK;
    if (q != cudaSuccess) return bfail(b, BPM_ERR_CUDA, cudaGetErrorString(q));
    cudaEventDestroy(e.done);
    e.done = nullptr;
    // no round enqueued after the completing one touches this plan
    e.plan->stream = e.orig_stream;
    b->used -= e.plan->bytes;
    b->finished[ticket] = 1;
    b->entries.erase(b->entries.begin() + long(i));
    *done = 1;
    return BPM_OK;
  }
  return bfail(b, BPM_ERR_INVALID_ARG, "unknown ticket");
}

BPM_API bpm_status bpm_batch_cancel(bpm_batch b, uint64_t ticket) {
  BPM_NVTX();
  if (!b) return bfail(nullptr, BPM_ERR_INVALID_ARG, "null batch");
  for (size_t i = 0; i < b->entries.size(); ++i) {
    BatchEntry& e = b->entries[i];
    if (e.ticket != ticket) continue;
    if (e.finishing) return bfail(b, BPM_ERR_STATE, "ticket already finishing");
    // rounds already enqueued may still touch the plan: wait for them
    BPM_BCUDA(b, cudaStreamSynchronize(b->stream), "cancel");
    if (b->side) BPM_BCUDA(b, cudaStreamSynchronize(b->side), "cancel");
    e.plan->stream = e.orig_stream;
    if (e.done) cudaEventDestroy(e.done);
    b->used -= e.plan->bytes;
    b->finished[ticket] = 2;
    b->entries.erase(b->entries.begin() + long(i));
    return BPM_OK;
  }
  return bfail(b, BPM_ERR_INVALID_ARG, "unknown or finished ticket");
}

BPM_API bpm_status bpm_batch_sync(bpm_batch b) {
  BPM_NVTX();
  if (!b) return bfail(nullptr, BPM_ERR_INVALID_ARG, "null batch");
  BPM_BCUDA(b, cudaStreamSynchronize(b->stream), "batch synchronize");
  return BPM_OK;
}

// Replays, as one CUDA graph, the whole hot path of every entry in the batch:
// deformation factor, tables and incident field from the stored inputs, one
// round to nz, time response.  The graph is captured on the first call and
// again whenever the set of entries changes.
BPM_API bpm_status bpm_batch_run_graph(bpm_batch b) {
  BPM_NVTX();
  if (!b) return bfail(nullptr, BPM_ERR_INVALID_ARG, "null batch");
  uint64_t key = 1469598103934665603ull;
  for (const auto& e : b->entries) key = (key ^ reinterpret_cast<uintptr_t>(e.plan)) * 1099511628211ull;
  if (!b->graph || key != b->graph_key) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    BPM_BCUDA(b, cudaStreamSynchronize(b->stream), "pre-capture sync");
    // allocations happen before the capture: staging for every item, completion events
    int n_items = 0;
    for (auto& e : b->entries) {
      const int G = batch_item_channels(e.plan->grid.nx, e.plan->grid.split_order);
      n_items += (e.plan->n_ch + G - 1) / G;
      if (!e.done) BPM_BCUDA(b, cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming), "event");
    }
    BPM_BCUDA(b, slot_reserve(b->graph_slot, int(b->entries.size()), n_items), "graph staging");
    // capture on the batch's own stream; the graph is launched on the caller's
    cudaStream_t user = b->stream;
    b->stream = b->cap;
    for (auto& e : b->entries) {
      e.finishing = false;
      e.plan->z = 0;
      e.plan->stream = b->cap;
    }
    bpm_status st = BPM_OK;
    cudaGraph_t g = nullptr;
    cudaError_t be = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (be != cudaSuccess) {
      st = bfail(b, BPM_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(be));
    } else {
      for (auto& e : b->entries) {
        if (enqueue_crystal(e.plan) != cudaSuccess || enqueue_pulse(e.plan) != cudaSuccess) {
          st = bfail(b, BPM_ERR_CUDA, "setup launch during capture");
          break;
        }
      }
      if (st == BPM_OK) st = enqueue_round(b, b->graph_slot, 1 << 30);
    }
    cudaError_t ce = be == cudaSuccess ? cudaStreamEndCapture(b->cap, &g) : cudaSuccess;
    b->stream = user;
    for (auto& e : b->entries) e.plan->stream = user;
    if (st != BPM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    BPM_BCUDA(b, ce, "end capture");
    size_t n_nodes = 0;
    BPM_BCUDA(b, cudaGraphGetNodes(g, nullptr, &n_nodes), "graph nodes");
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    BPM_BCUDA(b, cudaGraphGetNodes(g, nodes.data(), &n_nodes), "graph nodes");
    b->graph_kernels = 0;
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      BPM_BCUDA(b, cudaGraphNodeGetType(nd, &ty), "graph node type");
      if (ty == cudaGraphNodeTypeKernel) ++b->graph_kernels;
    }
    cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    BPM_BCUDA(b, ie, "graph instantiate");
    b->graph_key = key;
    b->graph_slot.used = false;  // the captured round has not run yet
  }
  for (auto& e : b->entries) {
    e.plan->z = e.plan->grid.nz;
    e.plan->time_valid = true;
  }
  BPM_BCUDA(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
  return BPM_OK;
}

BPM_API bpm_status bpm_batch_graph_kernels(bpm_batch b, int* kernels) {
  if (!b || !kernels) return bfail(b, BPM_ERR_INVALID_ARG, "null argument");
  *kernels = b->graph ? b->graph_kernels : 0;
  return BPM_OK;
}

BPM_API bpm_status bpm_batch_pending(bpm_batch b, int* rounds_in_flight) {
  if (!b || !rounds_in_flight) return bfail(b, BPM_ERR_INVALID_ARG, "null argument");
  int n = 0;
  for (const RoundSlot& r : b->slots) {
    if (!r.used) continue;
    const cudaError_t q = cudaEventQuery(r.free_ev);
    if (q == cudaErrorNotReady) ++n;
    else if (q != cudaSuccess) return bfail(b, BPM_ERR_CUDA, std::string("round: ") + cudaGetErrorString(q));
  }
  *rounds_in_flight = n;
  return BPM_OK;
}

BPM_API bpm_status bpm_batch_set_max_blocks(bpm_batch b, int max_blocks) {
  if (!b) return bfail(nullptr, BPM_ERR_INVALID_ARG, "null batch");
  b->max_blocks = max_blocks > 0 ? max_blocks : 0;
  return BPM_OK;
}

BPM_API bpm_status bpm_batch_info(bpm_batch b, int* active, size_t* used_bytes, int* rounds,
                                  int* last_items) {
  if (!b) return bfail(nullptr, BPM_ERR_INVALID_ARG, "null batch");
  if (active) *active = int(b->entries.size());
  if (used_bytes) *used_bytes = b->used;
  if (rounds) *rounds = b->rounds;
  if (last_items) {
    last_items[0] = b->last_items[0];
    last_items[1] = b->last_items[1];
  }
  return BPM_OK;
}

BPM_API const char* bpm_batch_last_error(bpm_batch b) {
  return b ? b->err.c_str() : g_thread_error.c_str();
}

BPM_API void bpm_batch_destroy(bpm_batch b) {
  BPM_NVTX();
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->side) cudaStreamSynchronize(b->side);
  for (auto& e : b->entries)
    if (e.done) cudaEventDestroy(e.done);
  for (auto& r : b->slots) slot_free(r);
  slot_free(b->graph_slot);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

}  // extern "C"
