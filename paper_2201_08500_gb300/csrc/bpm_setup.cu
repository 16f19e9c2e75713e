// Per-plan setup kernels of the BPM (FP64 arithmetic, run once per crystal /
// pulse) and the frequency-to-time assembly.
//
//  deformation_kernel : c(x, z) = Pi(x, z) exp(+i h u(x, z))         (Eq. Authier);
//                       Pi from the crystal's boundaries or a caller's mask
//  tables_kernel      : tilted propagators p+- and coupling coefficients
//                       (Eqs. fov4, fov11, fov12, Zassenhaus-like factor)
//  incident_kernel    : A+ = S g(x, y) exp(i (k sin theta_i - h/2) x), A- = 0
//                       (beam of Section 3.1, spectral amplitude of Eq. ref:tdp)
//  omega_to_t kernels : psi_h(t_j) = d_omega sum_i A-(omega_i) exp(-2 pi i (i - n/2) j / n)
//                       (frequency reassembly after Eq. ref:tdp), FP64 accumulation
#include <cuda_runtime.h>
#include <math.h>

#include "bpm_internal.h"

namespace bpm {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kC = 299792458.0;

struct dc {
  double re, im;
};
__device__ __forceinline__ dc dmk(double r, double i) { return dc{r, i}; }
__device__ __forceinline__ dc dadd(dc a, dc b) { return dc{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ dc dmul(dc a, dc b) {
  return dc{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ dc dscale(dc a, double s) { return dc{a.re * s, a.im * s}; }
__device__ __forceinline__ dc ddiv_real(dc a, double s) { return dc{a.re / s, a.im / s}; }
__device__ __forceinline__ dc dexp(dc z) {
  double s, c;
  sincos(z.im, &s, &c);
  const double m = exp(z.re);
  return dc{m * c, m * s};
}
__device__ __forceinline__ dc drecip(dc z) {
  const double d = z.re * z.re + z.im * z.im;
  return dc{z.re / d, -z.im / d};
}
// principal square root
__device__ __forceinline__ dc dsqrt(dc z) {
  const double r = hypot(z.re, z.im);
  double re = sqrt(0.5 * (r + fabs(z.re)));
  double im = (re > 0.0) ? z.im / (2.0 * re) : 0.0;
  if (z.re < 0.0) {
    const double t = re;
    re = fabs(im);
    im = (z.im >= 0.0) ? t : -t;
  }
  return dc{re, im};
}

__device__ __forceinline__ float2 to_f2(dc z) { return make_float2(float(z.re), float(z.im)); }

// Spatial frequency of DFT bin m on an n-point grid of spacing d (Nyquist negative).
__device__ __forceinline__ double qbin(int m, int n, double d) {
  const int mm = (m < n / 2) ? m : m - n;
  return 2.0 * kPi * double(mm) / (double(n) * d);
}

// exp(i dz [sqrt(k^2 - Q^2) - k]) with the evanescent branch decaying.
__device__ __forceinline__ dc tilted_propagator(double k, double Q2, double dz) {
  const double arg = k * k - Q2;
  if (arg >= 0.0) {
    // sqrt(k^2 - Q^2) - k = -Q^2 / (sqrt(k^2 - Q^2) + k): no cancellation
    const double ph = -dz * Q2 / (sqrt(arg) + k);
    double s, c;
    sincos(ph, &s, &c);
    return dc{c, s};
  }
  const double m = exp(-dz * sqrt(-arg));
  double s, c;
  sincos(-dz * k, &s, &c);
  return dc{m * c, m * s};
}

// Crystal mask Pi(x_j, z_n) (the crystal's boundaries set the geometry, end of
// Section 2): x_surface + z tan_psi <= x_j < x_end + z tan_psi and
// z_begin <= z_n < z_end, with x_j = j dx, z_n = n dz.  Every product and sum is
// rounded explicitly (no contraction) so that the decision is reproducible.
__device__ __forceinline__ bool in_crystal(const SetupArgs& sa, int j, int n) {
  const double x = __dmul_rn(double(j), sa.dx);
  const double z = __dmul_rn(double(n), sa.dz);
  if (!(z >= sa.z_begin && z < sa.z_end)) return false;
  const double shift = __dmul_rn(z, sa.tan_psi);
  return x >= __dadd_rn(sa.x_surface, shift) && x < __dadd_rn(sa.x_end, shift);
}

__global__ void deformation_kernel(SetupArgs sa, const double* __restrict__ u, float2* cfield) {
  const long long plane = (long long)sa.nx * sa.ny;
  const long long total = plane * sa.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = int(i % sa.nx);
    const bool in = sa.mask ? sa.mask[i] != 0 : in_crystal(sa, j, int(i / plane));
    float2 c = make_float2(0.f, 0.f);
    if (in) {
      const double ph = u ? sa.h * u[i] : 0.0;
      double s, co;
      sincos(ph, &s, &co);
      c = make_float2(float(co), float(s));
    }
    cfield[i] = c;
  }
}

// Crystal extent of each deformation row (one block per row at a time).
__global__ void crystal_span_kernel(const float2* __restrict__ cfield, int nx, long long rows,
                                    int2* span) {
  __shared__ int slo[32], shi[32];
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const float2* row = cfield + r * nx;
    int lo = nx, hi = -1;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const float2 c = row[x];
      if (c.x != 0.f || c.y != 0.f) {
        lo = min(lo, x);
        hi = max(hi, x);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, off));
      hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, off));
    }
    if ((threadIdx.x & 31) == 0) {
      slo[threadIdx.x / 32] = lo;
      shi[threadIdx.x / 32] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < int(blockDim.x / 32); ++w) {
        lo = min(lo, slo[w]);
        hi = max(hi, shi[w]);
      }
      span[r] = hi < 0 ? make_int2(0, 0) : make_int2(lo, hi + 1);
    }
    __syncthreads();
  }
}

// Power series of J0(w) and G1(w) = 2 J1(w)/w in terms of w^2 (A&S 9.1.10).
__device__ void bessel_j0_g1(dc w2, dc* j0, dc* g1) {
  const dc z = dscale(w2, -0.25);
  dc t0 = dmk(1, 0), t1 = dmk(1, 0), s0 = dmk(1, 0), s1 = dmk(1, 0);
  for (int k = 1; k < 40; ++k) {
    t0 = ddiv_real(dmul(t0, z), double(k) * k);
    t1 = ddiv_real(dmul(t1, z), double(k) * (k + 1));
    s0 = dadd(s0, t0);
    s1 = dadd(s1, t1);
  }
  *j0 = s0;
  *g1 = s1;
}

// Coupling coefficients of Eq. fov10 for one channel: w^2 = (k dz / cos a)^2
// chi_h chi_hbar, a = J0 e^{i phi} e^{w^2/8} (Zassenhaus), b+ = i G1 e^{i phi}
// k dz chi_hbar / (2 cos a), b- likewise with chi_h; a split into hi + lo.
__device__ ChannelCoef channel_coef(const SetupArgs& sa, double kdz, double cos_a) {
  const dc chi0 = dmk(sa.chi0_re, sa.chi0_im);
  const dc chih = dmk(sa.chih_re, sa.chih_im);
  const dc chihb = dmk(sa.chihb_re, sa.chihb_im);
  const double r = kdz / cos_a;
  const dc w2 = dscale(dmul(chih, chihb), r * r);
  const dc phase0 = dexp(dmul(dmk(0, 1), dscale(chi0, kdz / (2.0 * cos_a))));
  dc j0, g1;
  bessel_j0_g1(w2, &j0, &g1);
  const dc zf = sa.zassenhaus ? dexp(dscale(w2, 0.125)) : dmk(1, 0);
  const dc a = dmul(dmul(j0, phase0), zf);
  const dc ig1p = dmul(dmk(0, 1), dmul(g1, phase0));
  const dc bp = dmul(ig1p, dscale(chihb, kdz / (2.0 * cos_a)));
  const dc bm = dmul(ig1p, dscale(chih, kdz / (2.0 * cos_a)));
  ChannelCoef c;
  c.a_hi = to_f2(a);
  c.a_lo = make_float2(float(a.re - double(c.a_hi.x)), float(a.im - double(c.a_hi.y)));
  c.bp = to_f2(bp);
  c.bm = to_f2(bm);
  return c;
}

// One block per channel.  Tables are written in the march kernel's order:
// [ch][env][k][t] for the spectrum position p = 16 t + k, env 0 = E0 (+h/2), 1 = Eh (-h/2).
__global__ void tables_kernel(SetupArgs sa, const double* __restrict__ omega,
                              const double* __restrict__ gain, const int* __restrict__ rev,
                              float4* tables, ChannelCoef* coef, int* bad) {
  const int ch = blockIdx.x;
  const int n = sa.nx;
  const int T = n / 16;
  const double k = omega[ch] / kC;
  const double half_h = 0.5 * sa.h;
  const double s_ratio = half_h / k;
  if (!(s_ratio < 1.0)) {
    if (threadIdx.x == 0) atomicExch(bad, 1);
    return;
  }
  const double cos_a = sqrt(1.0 - s_ratio * s_ratio);  // cos(alpha), Eq. fov3
  const double kdz = k * sa.dz;
  // fractions of dz of the propagations (tables) and couplings (coefficient
  // sets) of Eq. split-op: order 1: (1; 1); order 2: (1; 1/2); order 4:
  // (t, 1-2t; t/2, (1-t)/2) with t = 1/(2 - 2^(1/3))
  const double t4 = 1.0 / (2.0 - cbrt(2.0));
  const int n_sets = sa.split_order == 4 ? 2 : 1;
  const double pf[2] = {sa.split_order == 4 ? t4 : 1.0, 1.0 - 2.0 * t4};
  const double cfr[2] = {sa.split_order == 4 ? 0.5 * t4 : (sa.split_order == 2 ? 0.5 : 1.0),
                         0.5 * (1.0 - t4)};
  if (threadIdx.x < n_sets)
    coef[size_t(ch) * n_sets + threadIdx.x] = channel_coef(sa, kdz * cfr[threadIdx.x], cos_a);
  for (int set = 0; set < n_sets; ++set) {
    float4* out = tables + (size_t(ch) * n_sets + set) * 2 * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      const double q = qbin(rev[p], n, sa.dx);
      const double scale = 1.0 / (double(n) * gain[p]);
      const int t = p / 16, kk = p % 16;
      for (int env = 0; env < 2; ++env) {
        const double Q = env == 0 ? q + half_h : q - half_h;
        dc P = tilted_propagator(k, Q * Q, sa.dz * pf[set]);
        P = dscale(P, scale);
        const float2 hi = to_f2(P);
        const float2 lo = make_float2(float(P.re - double(hi.x)), float(P.im - double(hi.y)));
        out[size_t(env) * n + size_t(kk) * T + t] = make_float4(hi.x, hi.y, lo.x, lo.y);
      }
    }
  }
}

// 3D: per channel and stored x-frequency column cs (px = 16 (cs % T) + cs / T),
// the anchor exp(i dz (K - k)) / (nx ny g_x(px)), K = sqrt(k^2 - (qx +- h/2)^2),
// as FP32 hi + lo, and the curvature factor -dz / (2 K) of the qy correction.
__global__ void tables3d_kernel(SetupArgs sa, const double* __restrict__ omega,
                                const double* __restrict__ gainx, const int* __restrict__ revx,
                                float4* anchor, float* gcorr, ChannelCoef* coef) {
  const int ch = blockIdx.x;
  const int n = sa.nx;
  const int T = n / 16;
  const double k = omega[ch] / kC;
  const double half_h = 0.5 * sa.h;
  const double s_ratio = half_h / k;
  const double cos_a = sqrt(1.0 - s_ratio * s_ratio);
  if (threadIdx.x == 0) coef[ch] = channel_coef(sa, k * sa.dz * sa.coupling_frac, cos_a);
  for (int cs = threadIdx.x; cs < n; cs += blockDim.x) {
    const int px = 16 * (cs % T) + cs / T;
    const double qx = qbin(revx[px], n, sa.dx);
    const double scale = 1.0 / (double(n) * double(sa.ny) * gainx[px]);
    for (int env = 0; env < 2; ++env) {
      const double Q = env == 0 ? qx + half_h : qx - half_h;
      const double K2 = k * k - Q * Q;
      dc P = tilted_propagator(k, Q * Q, sa.dz);
      P = dscale(P, scale);
      const float2 hi = to_f2(P);
      const float2 lo = make_float2(float(P.re - double(hi.x)), float(P.im - double(hi.y)));
      const size_t o = (size_t(ch) * 2 + env) * n + cs;
      anchor[o] = make_float4(hi.x, hi.y, lo.x, lo.y);
      gcorr[o] = K2 > 0.0 ? float(-sa.dz / (2.0 * sqrt(K2))) : 0.f;
    }
  }
}

// One block per channel: incident field and its FP64 norm.
__global__ void incident_kernel(SetupArgs sa, const double* __restrict__ omega,
                                const double2* __restrict__ weight, float2* e0, float2* eh,
                                double* inc_norm) {
  const int ch = blockIdx.x;
  const long long plane = (long long)sa.nx * sa.ny;
  const double k = omega[ch] / kC;
  const double dq = k * sin(sa.theta_i) - 0.5 * sa.h;
  const dc den = dmk(1.0, sa.zR != 0.0 ? sa.zx / sa.zR : 0.0);
  const dc pref = (sa.dims == 3) ? drecip(den) : drecip(dsqrt(den));
  const dc inv_den = drecip(den);
  const dc S = dmk(weight[ch].x, weight[ch].y);
  const dc Spref = dmul(S, pref);
  double acc = 0.0;
  for (long long i = threadIdx.x; i < plane; i += blockDim.x) {
    const int j = int(i % sa.nx);
    const int r = int(i / sa.nx);
    const double x = double(j) * sa.dx;
    const double y = (sa.dims == 3) ? (double(r) - double(sa.ny / 2)) * sa.dy : 0.0;
    const double rr = ((x - sa.x0) * (x - sa.x0) + y * y) / (sa.w0 * sa.w0);
    const dc g = dexp(dscale(inv_den, -rr));
    double s, c;
    sincos(dq * x, &s, &c);
    const dc v = dmul(dmul(Spref, g), dmk(c, s));
    e0[size_t(ch) * plane + i] = to_f2(v);
    eh[size_t(ch) * plane + i] = make_float2(0.f, 0.f);
    acc += v.re * v.re + v.im * v.im;
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) s += red[w];
    inc_norm[ch] = s;
  }
}

// Frequency-to-time, n a power of two: per block COLS columns of the
// [n][plane] spectrum, FP64 radix-2 transform in shared memory (bit-reversed
// load, log2 n butterfly passes), output scaled by d_omega exp(2 pi i (n/2) j / n).
// The plan holds channels first .. first + n_local - 1 of the n (a channel
// shard, or all of them); the others enter as zeros, so the output is this
// shard's part of the sum.
// The n/2 twiddles W^m = exp(-2 pi i m / n) are computed once per block into
// shared memory; stage len uses W^(kk n / len) (the same double as
// exp(-2 pi i kk / len): both arguments are exact binary fractions).
constexpr int kCols = 8;
__global__ void omega_to_t_fft_kernel(int n, int logn, int first, int n_local, long long plane,
                                      double domega, const float2* __restrict__ eh, double2* out) {
  extern __shared__ double2 sm[];  // [n][kCols], then the twiddles [n/2]
  double2* tw = sm + size_t(n) * kCols;
  const long long x0 = (long long)blockIdx.x * kCols;
  const int cols = int(min((long long)kCols, plane - x0));
  for (int m = threadIdx.x; m < n / 2; m += blockDim.x) {
    double s, co;
    sincospi(-2.0 * double(m) / double(n), &s, &co);
    tw[m] = make_double2(co, s);
  }
  for (int idx = threadIdx.x; idx < n * kCols; idx += blockDim.x) {
    const int i = idx / kCols, c = idx % kCols;
    const int ri = logn ? int(__brev(unsigned(i)) >> (32 - logn)) : 0;
    double2 v = make_double2(0.0, 0.0);
    const int li = i - first;
    if (c < cols && li >= 0 && li < n_local) {
      const float2 f = eh[(long long)li * plane + x0 + c];
      v = make_double2(double(f.x), double(f.y));
    }
    sm[ri * kCols + c] = v;
  }
  __syncthreads();
  for (int half = 1; half < n; half <<= 1) {
    const int len = half * 2;
    const int step = n / len;
    for (int idx = threadIdx.x; idx < (n / 2) * kCols; idx += blockDim.x) {
      const int bf = idx / kCols, c = idx % kCols;
      const int grp = bf / half, kk = bf % half;
      const int ia = grp * len + kk, ib = ia + half;
      const double2 w = tw[kk * step];
      const double2 u = sm[ia * kCols + c], v = sm[ib * kCols + c];
      const double2 wv = make_double2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
      sm[ia * kCols + c] = make_double2(u.x + wv.x, u.y + wv.y);
      sm[ib * kCols + c] = make_double2(u.x - wv.x, u.y - wv.y);
    }
    __syncthreads();
  }
  const int ic = n / 2;
  for (int idx = threadIdx.x; idx < n * kCols; idx += blockDim.x) {
    const int j = idx / kCols, c = idx % kCols;
    if (c >= cols) continue;
    // exp(+2 pi i e / n) = conj(W^e), W^(e + n/2) = -W^e
    const int e = int(((long long)ic * j) % n);
    const double2 w0 = tw[e % ic];
    const double sg = e < ic ? 1.0 : -1.0;
    const double co = sg * w0.x, s = -sg * w0.y;
    const double2 v = sm[j * kCols + c];
    out[(long long)j * plane + x0 + c] =
        make_double2(domega * (v.x * co - v.y * s), domega * (v.x * s + v.y * co));
  }
}

// Direct FP64 sum for any n (used when n is not a power of two), over this
// plan's channels first .. first + n_local - 1 of the n.
__global__ void omega_to_t_direct_kernel(int n, int first, int n_local, long long plane,
                                         double domega, const float2* __restrict__ eh,
                                         double2* out) {
  const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (x >= plane) return;
  const int ic = n / 2;
  double re = 0.0, im = 0.0;
  for (int li = 0; li < n_local; ++li) {
    const int i = first + li;
    const long long e = (((long long)(i - ic) * j) % n + n) % n;
    double s, co;
    sincospi(-2.0 * double(e) / double(n), &s, &co);
    const float2 f = eh[(long long)li * plane + x];
    re += double(f.x) * co - double(f.y) * s;
    im += double(f.x) * s + double(f.y) * co;
  }
  out[(long long)j * plane + x] = make_double2(domega * re, domega * im);
}

}  // namespace

cudaError_t setup_set_attributes() {
  return cudaFuncSetAttribute(omega_to_t_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              200 * 1024);
}

cudaError_t launch_deformation(const SetupArgs& sa, const double* u_dev, float2* cfield,
                               cudaStream_t s) {
  const long long total = (long long)sa.nx * sa.ny * sa.nz;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  deformation_kernel<<<int(blocks), 256, 0, s>>>(sa, u_dev, cfield);
  return cudaGetLastError();
}

cudaError_t launch_crystal_span(const float2* cfield, int nx, long long rows, int2* span,
                                cudaStream_t s) {
  const long long blocks = rows < 152 * 16 ? rows : 152 * 16;
  crystal_span_kernel<<<int(blocks), 256, 0, s>>>(cfield, nx, rows, span);
  return cudaGetLastError();
}

cudaError_t launch_tables(const SetupArgs& sa, const double* omega, const double* gain,
                          const int* rev, float4* tables, ChannelCoef* coef, int* bad,
                          cudaStream_t s) {
  tables_kernel<<<sa.n_ch, 256, 0, s>>>(sa, omega, gain, rev, tables, coef, bad);
  return cudaGetLastError();
}

cudaError_t launch_tables3d(const SetupArgs& sa, const double* omega, const double* gainx,
                            const int* revx, float4* anchor, float* gcorr, ChannelCoef* coef,
                            cudaStream_t s) {
  tables3d_kernel<<<sa.n_ch, 256, 0, s>>>(sa, omega, gainx, revx, anchor, gcorr, coef);
  return cudaGetLastError();
}

cudaError_t launch_incident(const SetupArgs& sa, const double* omega, const double2* weight,
                            float2* e0, float2* eh, double* inc_norm, cudaStream_t s) {
  incident_kernel<<<sa.n_ch, 256, 0, s>>>(sa, omega, weight, e0, eh, inc_norm);
  return cudaGetLastError();
}

cudaError_t launch_omega_to_t(int n_total, int first, int n_local, long long plane,
                              double domega, const float2* eh, double2* out, cudaStream_t s) {
  if (first < 0 || n_local < 0 || first + n_local > n_total) return cudaErrorInvalidValue;
  const int n = n_total;
  const bool pow2 = n > 0 && (n & (n - 1)) == 0;
  const size_t smem = size_t(n) * kCols * sizeof(double2) + size_t(n / 2) * sizeof(double2);
  if (pow2 && n >= 2 && smem <= 200 * 1024) {
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    const long long blocks = (plane + kCols - 1) / kCols;
    omega_to_t_fft_kernel<<<int(blocks), 256, smem, s>>>(n, logn, first, n_local, plane, domega,
                                                        eh, out);
    return cudaGetLastError();
  }
  dim3 grid(unsigned((plane + 127) / 128), unsigned(n));
  omega_to_t_direct_kernel<<<grid, 128, 0, s>>>(n, first, n_local, plane, domega, eh, out);
  return cudaGetLastError();
}

}  // namespace bpm
