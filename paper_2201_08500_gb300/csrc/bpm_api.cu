// Host runtime of libbpm: the C ABI of include/bpm.h.
//
// A plan owns the device state of one BPM problem (one crystal, one pulse,
// n_channels frequency channels): the deformation factor c(x, z), the per
// channel propagator tables and coupling coefficients, the two envelopes, the
// reflectivities and the time response.  All device work is enqueued on the
// caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
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
  }
  cache[dev] = d;
  return cache[dev];
}

}  // namespace

struct bpm_plan_s {
  bpm_grid grid{};
  int n_ch = 0;
  cudaStream_t stream = nullptr;
  std::string err = "no error";
  int plane = 0;

  bool have_crystal = false, have_pulse = false, time_valid = false;
  int z = 0;
  SetupArgs sa{};
  double domega = 1.0;

  // device buffers
  float2* cfield = nullptr;
  float2* e0 = nullptr;
  float2* eh = nullptr;
  float4* tables = nullptr;
  ChannelCoef* coef = nullptr;
  float2* twiddle = nullptr;
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

  int group = 1, blocks = 0;
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bpm_stats stats{};
};

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
  void* ptrs[] = {p->cfield, p->e0,     p->eh,       p->tables, p->coef,    p->twiddle,
                  p->rev,    p->gain,   p->omega,    p->weight, p->inc_norm, p->refl,
                  p->trans,  p->eh_time, p->dflag,   p->u_tmp};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" {

BPM_API const char* bpm_version(void) { return "libbpm 0.1 (sm_103a, resident radix-16 march)"; }

BPM_API const char* bpm_last_error(bpm_plan plan) {
  return plan ? plan->err.c_str() : g_thread_error.c_str();
}

BPM_API bpm_status bpm_plan_create(const bpm_grid* grid, int n_channels, void* cuda_stream,
                                   bpm_plan* out) {
  if (!grid || !out) return fail(nullptr, BPM_ERR_INVALID_ARG, "null grid or output pointer");
  *out = nullptr;
  const bpm_grid& g = *grid;
  if (n_channels < 1) return fail(nullptr, BPM_ERR_INVALID_ARG, "n_channels must be >= 1");
  if (g.nz < 1 || !(g.dx > 0) || !(g.dz > 0))
    return fail(nullptr, BPM_ERR_INVALID_ARG, "nz, dx and dz must be positive");
  if (g.split_order != 1)
    return fail(nullptr, BPM_ERR_UNSUPPORTED, "only first-order splitting is implemented");
  if (g.dims != 2)
    return fail(nullptr, BPM_ERR_UNSUPPORTED, "only dims = 2 is implemented in this build");
  if (g.ny != 1) return fail(nullptr, BPM_ERR_INVALID_ARG, "dims = 2 requires ny = 1");
  if (!is_pow2(g.nx) || g.nx < 256 || g.nx > 8192)
    return fail(nullptr, BPM_ERR_UNSUPPORTED, "nx must be a power of two in [256, 8192]");
  const DeviceInfo& di = device_info();
  if (!di.ok) return fail(nullptr, BPM_ERR_CUDA, "no CUDA device");
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
  check(dalloc(&p->e0, nf), "alloc E0");
  check(dalloc(&p->eh, nf), "alloc Eh");
  check(dalloc(&p->tables, size_t(n_channels) * 2 * g.nx), "alloc propagator tables");
  check(dalloc(&p->coef, size_t(n_channels)), "alloc coefficients");
  check(dalloc(&p->twiddle, size_t(g.nx)), "alloc twiddles");
  check(dalloc(&p->rev, size_t(g.nx)), "alloc spectrum order");
  check(dalloc(&p->gain, size_t(g.nx)), "alloc gain");
  check(dalloc(&p->omega, size_t(n_channels)), "alloc omega");
  check(dalloc(&p->weight, size_t(n_channels)), "alloc weights");
  check(dalloc(&p->inc_norm, size_t(n_channels)), "alloc norms");
  check(dalloc(&p->refl, size_t(n_channels)), "alloc R");
  check(dalloc(&p->trans, size_t(n_channels)), "alloc T");
  check(dalloc(&p->eh_time, nf), "alloc time response");
  check(dalloc(&p->dflag, size_t(4)), "alloc status");
  if (st != BPM_OK) {
    free_plan_buffers(P);
    return st;
  }
  const FftConsts& fc = fft_consts(g.nx);
  check(cudaMemcpyAsync(p->twiddle, fc.tw.data(), sizeof(float2) * g.nx, cudaMemcpyHostToDevice,
                        p->stream),
        "upload twiddles");
  check(cudaMemcpyAsync(p->rev, fc.rev.data(), sizeof(int) * g.nx, cudaMemcpyHostToDevice,
                        p->stream),
        "upload spectrum order");
  check(cudaMemcpyAsync(p->gain, fc.gain.data(), sizeof(double) * g.nx, cudaMemcpyHostToDevice,
                        p->stream),
        "upload gain");
  check(cudaMemsetAsync(p->dflag, 0, sizeof(int) * 4, p->stream), "clear status");
  check(cudaStreamSynchronize(p->stream), "plan upload");
  if (st != BPM_OK) {
    free_plan_buffers(P);
    return st;
  }
  const int maxg = march_max_group(g.nx);
  const long long full = (n_channels + maxg - 1) / maxg;
  p->group = (maxg > 1 && full >= di.sm_count) ? maxg : 1;
  p->blocks = (n_channels + p->group - 1) / p->group;
  p->stats.threads_per_channel = march_threads_per_channel(g.nx);
  p->stats.channels_per_block = p->group;
  p->stats.blocks = p->blocks;
  p->stats.smem_bytes = int(march_smem_bytes(g.nx, p->group));
  *out = p.release();
  return BPM_OK;
}

BPM_API bpm_status bpm_set_crystal(bpm_plan p, double chi0_re, double chi0_im, double chih_re,
                                   double chih_im, double chihbar_re, double chihbar_im,
                                   double theta_B, double lambda_B, double x_surface,
                                   double thickness, const double* u_field, int u_on_device) {
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
  sa.x_surface = x_surface;
  sa.x_end = x_surface + thickness;
  const size_t cells = size_t(p->grid.nz) * p->plane;
  const double* u_dev = nullptr;
  if (u_field) {
    if (u_on_device) {
      u_dev = u_field;
    } else {
      if (!p->u_tmp) BPM_CUDA(p, dalloc(&p->u_tmp, cells), "alloc displacement upload");
      BPM_CUDA(p, cudaMemcpyAsync(p->u_tmp, u_field, cells * sizeof(double),
                                  cudaMemcpyHostToDevice, p->stream),
               "upload displacement");
      u_dev = p->u_tmp;
    }
  }
  BPM_CUDA(p, launch_deformation(sa, u_dev, p->cfield, p->stream), "deformation kernel");
  p->have_crystal = true;
  p->have_pulse = false;
  p->time_valid = false;
  return BPM_OK;
}

BPM_API bpm_status bpm_set_pulse(bpm_plan p, const double* omega, const double* weight_re_im,
                                 double theta_i, double x0, double w0, double zx, double zR) {
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!omega || !weight_re_im) return fail(p, BPM_ERR_INVALID_ARG, "null omega or weights");
  if (!p->have_crystal) return fail(p, BPM_ERR_STATE, "bpm_set_crystal must come first");
  if (!(w0 > 0.0)) return fail(p, BPM_ERR_INVALID_ARG, "w0 must be positive");
  for (int i = 0; i < p->n_ch; ++i)
    if (!(omega[i] > 0.0)) return fail(p, BPM_ERR_INVALID_ARG, "omega must be positive");
  p->sa.theta_i = theta_i;
  p->sa.x0 = x0;
  p->sa.w0 = w0;
  p->sa.zx = zx;
  p->sa.zR = zR;
  p->domega = p->n_ch > 1 ? omega[1] - omega[0] : 1.0;
  BPM_CUDA(p, cudaMemcpyAsync(p->omega, omega, sizeof(double) * p->n_ch, cudaMemcpyHostToDevice,
                              p->stream),
           "upload omega");
  BPM_CUDA(p, cudaMemcpyAsync(p->weight, weight_re_im, sizeof(double2) * p->n_ch,
                              cudaMemcpyHostToDevice, p->stream),
           "upload weights");
  BPM_CUDA(p, cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream), "clear flag");
  BPM_CUDA(p, launch_tables(p->sa, p->omega, p->gain, p->rev, p->tables, p->coef, p->dflag,
                            p->stream),
           "tables kernel");
  BPM_CUDA(p, launch_incident(p->sa, p->omega, p->weight, p->e0, p->eh, p->inc_norm, p->stream),
           "incident kernel");
  int bad = 0;
  BPM_CUDA(p, cudaMemcpyAsync(&bad, p->dflag, sizeof(int), cudaMemcpyDeviceToHost, p->stream),
           "read setup flag");
  BPM_CUDA(p, cudaStreamSynchronize(p->stream), "pulse setup");
  if (bad) return fail(p, BPM_ERR_INVALID_ARG, "a channel has k <= h/2 (no Bragg solution)");
  p->z = 0;
  p->have_pulse = true;
  p->time_valid = false;
  return BPM_OK;
}

BPM_API bpm_status bpm_set_fields(bpm_plan p, const void* e0, const void* eh, int z_step,
                                  int on_device) {
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
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  if (!p->have_pulse) return fail(p, BPM_ERR_STATE, "bpm_set_pulse must come first");
  if (n_steps < 0 || p->z + n_steps > p->grid.nz)
    return fail(p, BPM_ERR_INVALID_ARG, "n_steps must keep z within [0, nz]");
  MarchArgs a;
  a.tables = p->tables;
  a.coef = p->coef;
  a.twiddle = p->twiddle;
  a.cfield = p->cfield;
  a.e0 = p->e0;
  a.eh = p->eh;
  a.inc_norm = p->inc_norm;
  a.refl = p->refl;
  a.trans = p->trans;
  a.n_ch = p->n_ch;
  a.z0 = p->z;
  a.n_steps = n_steps;
  int launches = 0;
  if (p->timing) BPM_CUDA(p, cudaEventRecord(p->ev0, p->stream), "timing event");
  BPM_CUDA(p, launch_march(p->grid.nx, p->group, p->blocks, a, p->stream), "march kernel");
  ++launches;
  if (p->timing) BPM_CUDA(p, cudaEventRecord(p->ev1, p->stream), "timing event");
  p->z += n_steps;
  p->time_valid = false;
  if (p->z == p->grid.nz) {
    BPM_CUDA(p, launch_omega_to_t(p->n_ch, p->plane, p->domega, p->eh, p->eh_time, p->stream),
             "omega-to-t kernel");
    ++launches;
    p->time_valid = true;
  }
  p->stats.launches = launches;
  p->stats.march_launches = 1;
  return BPM_OK;
}

BPM_API bpm_status bpm_sync(bpm_plan p) {
  if (!p) return fail(nullptr, BPM_ERR_INVALID_ARG, "null plan");
  BPM_CUDA(p, cudaStreamSynchronize(p->stream), "stream synchronize");
  return BPM_OK;
}

BPM_API bpm_status bpm_fetch_fields(bpm_plan p, int which, void* dst, size_t bytes,
                                    int dst_on_device) {
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
      need = n * sizeof(double2);
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

BPM_API void bpm_plan_destroy(bpm_plan p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  free_plan_buffers(p);
  delete p;
}

}  // extern "C"
