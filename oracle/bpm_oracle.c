/*
 * FP64 CPU oracle for the two-beam FFT beam propagation method (BPM) of
 * Krzywinski & Halavanau, "Time-dependent dynamical Bragg diffraction in
 * deformed crystals by beam propagation method" (arXiv:2201.08500).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no code,
 * header, table or constant with the CUDA library: every quantity is derived
 * here again from the paper.
 *
 * What it computes, per frequency channel (Section 2 of the paper):
 *   - tilted angular propagators p+- = exp(i dz [sqrt(k^2-(q +- h/2)^2) - k])
 *     (Eq. fov4 with the shifted spectrum described after Eq. fov10);
 *   - the first three Jacobi-Anger terms of the susceptibility step
 *     (Eqs. fov9, fov11, fov12) with the Zassenhaus-like factor on the
 *     zeroth term (the unnumbered equation after Eq. split-op);
 *   - the deformation phase exp(i n h u) (Eq. Authier);
 *   - the two-envelope split-step march (Eq. fov10) with the first-, second-
 *     or fourth-order operator splitting of Eq. split-op;
 *   - the incident Gaussian beam of the "Stationary problems" subsection.
 * Reflectivity and the frequency-to-time sum (Eq. ref:tdp and the text that
 * follows it) are plain sums and are written in oracle/oracle.py with numpy.
 *
 * Readings where the paper is silent or garbled (all listed in the design
 * notes): E0 (carrier +h/2) takes sqrt(k^2-(q+h/2)^2); the propagator carries
 * the "-k" of Eq. fov2; z-hat in Eqs. fov9/fov11/fov12 is the step dz-hat;
 * cos(alpha) = sqrt(1-(h/2k)^2) per channel; the Zassenhaus factor is
 * exp(+w^2/8) in normalised units; the deformation phase is exp(+i h u) on
 * the E0 update and its conjugate on the Eh update; Pi and u are sampled at
 * z_n = n dz before step n; chi_h != chi_hbar is handled by splitting the
 * harmonic term as chi_hbar e^{+ihx} + chi_h e^{-ihx}.
 *
 * Parity: pinned (FFT vs direct DFT, Bessel series vs independent routines,
 * free-space Gaussian beam closed form, Beer-Lambert absorption, per-mode
 * 2x2 matrix power, flux identity, textbook Bragg-slab rocking curve).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_C_LIGHT 299792458.0
#define ORC_PI 3.14159265358979323846

/* Problem description; the Python side mirrors this layout with ctypes. */
typedef struct {
  int32_t dims; /* 2: (x,z); 3: (x,y,z) */
  int32_t nx, ny, nz;
  double dx, dy, dz;
  double chi0_re, chi0_im, chih_re, chih_im, chihb_re, chihb_im;
  double theta_B, lambda_B, x_surface, thickness;
  int32_t zassenhaus, split_order; /* Eq. split-op: 1 (Eq. fov4), 2 (Strang) or 4 (see orc_split_coefficients) */
  double theta_i, x0, w0, zx, zR;
  /* crystal shape (geometries by the crystal's boundaries, Section 2 end):
   * entrance surface x = x_surface + z tan_psi (asymmetric cut), slab
   * thickness along x, and the crystal cut to z_begin <= z < z_end (Laue slab
   * when the x range is unbounded). */
  double tan_psi, z_begin, z_end;
  /* An arbitrary crystal shape (Introduction: the method takes crystals of
   * any shape): Pi(x_j, y_r, z_n) = mask[(n ny + r) nx + j] != 0, [nz][ny][nx]
   * bytes, replacing the boundaries above; NULL keeps them. */
  const uint8_t* mask;
} orc_problem;

/* ------------------------------------------------------------------------- */
/* Discrete Fourier transforms.  Forward: F_m = sum_j f_j exp(-2 pi i j m/N);  */
/* inverse: f_j = (1/N) sum_m F_m exp(+2 pi i j m/N).                           */
/* ------------------------------------------------------------------------- */

static cplx unit_root(long num, long n, int sign) {
  /* exp(sign * 2 pi i num / n) with the integer reduced first */
  long r = num % n;
  if (r < 0) r += n;
  double ang = 2.0 * ORC_PI * (double)r / (double)n;
  return cos(ang) + (double)sign * I * sin(ang);
}

/* Direct O(N^2) DFT. sign = -1 forward, +1 inverse (inverse scaled by 1/N). */
int orc_dft(const cplx* in, cplx* out, int n, int sign) {
  if (n <= 0 || (sign != 1 && sign != -1)) return 1;
  for (int m = 0; m < n; ++m) {
    cplx acc = 0;
    for (int j = 0; j < n; ++j) acc += in[j] * unit_root((long)j * m, n, sign);
    out[m] = (sign > 0) ? acc / n : acc;
  }
  return 0;
}

/* Iterative radix-2 Cooley-Tukey (bit-reversal permutation, then log2 N     */
/* butterfly passes).  Twiddles are evaluated directly from the exact angle. */
int orc_fft(cplx* a, int n, int sign) {
  if (n <= 0 || (n & (n - 1)) || (sign != 1 && sign != -1)) return 1;
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int half = len >> 1;
    for (int k = 0; k < half; ++k) {
      cplx w = unit_root(k, len, sign);
      for (int s = 0; s < n; s += len) {
        cplx u = a[s + k];
        cplx v = a[s + k + half] * w;
        a[s + k] = u + v;
        a[s + k + half] = u - v;
      }
    }
  }
  if (sign > 0)
    for (int i = 0; i < n; ++i) a[i] /= n;
  return 0;
}

/* 2D transform of a row-major [ny][nx] array: along x, then along y. */
int orc_fft2(cplx* a, int nx, int ny, int sign) {
  if (ny < 1) return 1;
  for (int r = 0; r < ny; ++r)
    if (orc_fft(a + (size_t)r * nx, nx, sign)) return 1;
  if (ny == 1) return 0;
  cplx* col = (cplx*)malloc(sizeof(cplx) * (size_t)ny);
  if (!col) return 2;
  for (int c = 0; c < nx; ++c) {
    for (int r = 0; r < ny; ++r) col[r] = a[(size_t)r * nx + c];
    if (orc_fft(col, ny, sign)) {
      free(col);
      return 1;
    }
    for (int r = 0; r < ny; ++r) a[(size_t)r * nx + c] = col[r];
  }
  free(col);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Bessel functions of complex argument, by their power series               */
/* (Abramowitz & Stegun 9.1.10):                                             */
/*   J0(w)        = sum_k (-1)^k (w^2/4)^k / (k!)^2                          */
/*   G1(w) = 2 J1(w)/w = sum_k (-1)^k (w^2/4)^k / (k! (k+1)!)                */
/* Both depend on w only through w^2, so no square-root branch is needed.    */
/* ------------------------------------------------------------------------- */
static int bessel_series(cplx w2, cplx* j0, cplx* g1) {
  if (cabs(w2) > 64.0) return 1; /* series used only for |w| <= 8 */
  cplx z = -w2 / 4.0;
  cplx t0 = 1.0, t1 = 1.0, s0 = 1.0, s1 = 1.0;
  for (int k = 1; k < 60; ++k) {
    t0 *= z / ((double)k * (double)k);
    t1 *= z / ((double)k * (double)(k + 1));
    s0 += t0;
    s1 += t1;
  }
  *j0 = s0;
  *g1 = s1;
  return 0;
}

/* w2: pointer to (Re, Im) of w^2. */
int orc_bessel_j0_g1(const double* w2, cplx* j0, cplx* g1) {
  return bessel_series(w2[0] + I * w2[1], j0, g1);
}

/* ------------------------------------------------------------------------- */
/* Per-channel quantities (Section 2).                                       */
/* ------------------------------------------------------------------------- */
typedef struct {
  double k, h, cos_alpha;
  cplx a, bp, bm; /* coupling coefficients of Eq. fov10 */
  cplx w2;        /* w^2, w = k dz sqrt(chih chihb)/cos(alpha) */
} orc_chan;

static double wavenumber_h(const orc_problem* p) {
  /* reciprocal-lattice vector of the reflecting planes, Bragg's law */
  return 4.0 * ORC_PI * sin(p->theta_B) / p->lambda_B;
}

/* Coefficients of the susceptibility step B(frac dz) of Eq. split-op for one
 * channel: the step length dz-hat is frac * k dz in Eqs. fov9, fov11, fov12. */
static int chan_setup_frac(const orc_problem* p, double omega, double frac, orc_chan* c);

static int chan_setup(const orc_problem* p, double omega, orc_chan* c) {
  return chan_setup_frac(p, omega, 1.0, c);
}

static int chan_setup_frac(const orc_problem* p, double omega, double frac, orc_chan* c) {
  double k = omega / ORC_C_LIGHT;
  double h = wavenumber_h(p);
  double s = h / (2.0 * k);
  if (!(s < 1.0)) return 1;
  double cos_a = sqrt(1.0 - s * s); /* cos(alpha) of Eq. fov3 */
  cplx chi0 = p->chi0_re + I * p->chi0_im;
  cplx chih = p->chih_re + I * p->chih_im;
  cplx chihb = p->chihb_re + I * p->chihb_im;
  double kdz = frac * k * p->dz; /* normalised (fractional) step dz-hat */
  /* Eq. fov9 with delta-eps = chi0 + chihb e^{+ihx} + chih e^{-ihx}: the   */
  /* Jacobi-Anger argument is w = dz-hat sqrt(chih chihb)/cos(alpha), the    */
  /* constant part gives exp(i dz-hat chi0 / (2 cos alpha)).                  */
  cplx w2 = (kdz / cos_a) * (kdz / cos_a) * chih * chihb;
  cplx phase0 = cexp(I * kdz * chi0 / (2.0 * cos_a));
  cplx j0, g1;
  if (bessel_series(w2, &j0, &g1)) return 2;
  /* Eq. fov11 with the Zassenhaus-like factor exp(D2 dz-hat^2/2),          */
  /* D2 = (chi_h/2/cos alpha)^2, i.e. exp(w^2/8).                            */
  cplx zfac = p->zassenhaus ? cexp(w2 / 8.0) : 1.0;
  c->a = j0 * phase0 * zfac;
  /* Eq. fov12: i J1(w) e^{i phi}; J1(w) times the split of the harmonic    */
  /* amplitude equals G1(w) * dz-hat * chi / (2 cos alpha).                  */
  c->bp = I * g1 * phase0 * (kdz * chihb / (2.0 * cos_a)); /* Eh -> E0 */
  c->bm = I * g1 * phase0 * (kdz * chih / (2.0 * cos_a));  /* E0 -> Eh */
  c->k = k;
  c->h = h;
  c->cos_alpha = cos_a;
  c->w2 = w2;
  return 0;
}

static double qfreq(int m, int n, double d) {
  /* spatial frequency of DFT bin m (fftfreq order, Nyquist negative) */
  int mm = (m < n / 2) ? m : m - n;
  return 2.0 * ORC_PI * (double)mm / ((double)n * d);
}

/* Tilted propagator exp(i dz [sqrt(k^2 - (qx + sgn h/2)^2 - qy^2) - k]);     */
/* the principal root gives evanescent decay for the imaginary branch.       */
static cplx propagator(double k, double qx_shift, double qy, double dz) {
  double arg = k * k - qx_shift * qx_shift - qy * qy;
  if (arg >= 0.0) {
    double ph = dz * (sqrt(arg) - k);
    return cos(ph) + I * sin(ph);
  }
  double decay = dz * sqrt(-arg);
  return exp(-decay) * (cos(-dz * k) + I * sin(-dz * k));
}

/* Expose channel setup for the pin tests.                                   */
/* out_scalars: k, h, cos_alpha, Re w2, Im w2; coef: a, bp, bm;              */
/* pp, pm: [ny][nx] propagators for E0 (+h/2) and Eh (-h/2), may be NULL.     */
int orc_channel(const orc_problem* p, double omega, double* out_scalars, cplx* coef, cplx* pp,
                cplx* pm) {
  orc_chan c;
  int rc = chan_setup(p, omega, &c);
  if (rc) return rc;
  if (out_scalars) {
    out_scalars[0] = c.k;
    out_scalars[1] = c.h;
    out_scalars[2] = c.cos_alpha;
    out_scalars[3] = creal(c.w2);
    out_scalars[4] = cimag(c.w2);
  }
  if (coef) {
    coef[0] = c.a;
    coef[1] = c.bp;
    coef[2] = c.bm;
  }
  int ny = (p->dims == 3) ? p->ny : 1;
  for (int r = 0; r < ny; ++r) {
    double qy = (p->dims == 3) ? qfreq(r, p->ny, p->dy) : 0.0;
    for (int m = 0; m < p->nx; ++m) {
      double qx = qfreq(m, p->nx, p->dx);
      if (pp) pp[(size_t)r * p->nx + m] = propagator(c.k, qx + 0.5 * c.h, qy, p->dz);
      if (pm) pm[(size_t)r * p->nx + m] = propagator(c.k, qx - 0.5 * c.h, qy, p->dz);
    }
  }
  return 0;
}

/* Crystal mask Pi(x_j, y_r, z_n): x_j = j dx, z_n = n dz,                    */
/*   x_surface + z tan_psi <= x_j < x_surface + z tan_psi + thickness           */
/*   and z_begin <= z_n < z_end, or the caller's mask when one is given.       */
/* tan_psi = 0 and an unbounded z range give the symmetric-Bragg slab.          */
static int inside(const orc_problem* p, int j, int r, int n) {
  if (p->mask) {
    int ny = (p->dims == 3) ? p->ny : 1;
    return p->mask[((size_t)n * ny + r) * p->nx + j] != 0;
  }
  double x = (double)j * p->dx;
  double z = (double)n * p->dz;
  if (!(z >= p->z_begin && z < p->z_end)) return 0;
  double shift = z * p->tan_psi;
  double lo = p->x_surface + shift;
  double hi = p->x_surface + p->thickness;
  hi = hi + shift;
  return (x >= lo) && (x < hi);
}

/* Deformation factor c(x, z_n) = exp(+i h u(x, z_n)) (Eq. Authier, n=+1);   */
/* written as 0 outside the crystal.  u: [nz][ny][nx] metres or NULL.         */
int orc_deformation(const orc_problem* p, const double* u, int z_index, cplx* c_out,
                    uint8_t* mask_out) {
  double h = wavenumber_h(p);
  int ny = (p->dims == 3) ? p->ny : 1;
  for (int r = 0; r < ny; ++r)
    for (int j = 0; j < p->nx; ++j) {
      size_t idx = (size_t)r * p->nx + j;
      int in = inside(p, j, r, z_index);
      cplx cv = 0;
      if (in) {
        double uu = u ? u[((size_t)z_index * ny + r) * p->nx + j] : 0.0;
        double ph = h * uu;
        cv = cos(ph) + I * sin(ph);
      }
      if (c_out) c_out[idx] = cv;
      if (mask_out) mask_out[idx] = (uint8_t)in;
    }
  return 0;
}

/* Incident field of the "Stationary problems" subsection, for one channel: */
/*   A+(x, y, 0) = S * g(x, y) * exp(i dq x),  dq = k sin(theta_i) - h/2,     */
/*   g = (1 + i zx/zR)^(-1/2 or -1) exp(-((x-x0)^2 + y^2)/(W0^2 (1+i zx/zR))) */
/* with y_r = (r - ny/2) dy in 3D.  A- = 0.                                    */
static void incident_field(const orc_problem* p, double omega, cplx S, cplx* e0, cplx* eh) {
  double k = omega / ORC_C_LIGHT;
  double h = wavenumber_h(p);
  double dq = k * sin(p->theta_i) - 0.5 * h;
  cplx den = 1.0 + I * (p->zR != 0.0 ? p->zx / p->zR : 0.0);
  cplx pref = (p->dims == 3) ? 1.0 / den : 1.0 / csqrt(den);
  int ny = (p->dims == 3) ? p->ny : 1;
  for (int r = 0; r < ny; ++r) {
    double y = (p->dims == 3) ? ((double)r - (double)(p->ny / 2)) * p->dy : 0.0;
    for (int j = 0; j < p->nx; ++j) {
      double x = (double)j * p->dx;
      double rr = (x - p->x0) * (x - p->x0) + y * y;
      cplx g = pref * cexp(-rr / (p->w0 * p->w0 * den));
      double ph = dq * x;
      size_t idx = (size_t)r * p->nx + j;
      e0[idx] = S * g * (cos(ph) + I * sin(ph));
      if (eh) eh[idx] = 0;
    }
  }
}

/* S: pointer to (Re, Im) of the channel's spectral amplitude. */
int orc_incident(const orc_problem* p, double omega, const double* S, cplx* e0, cplx* eh) {
  incident_field(p, omega, S[0] + I * S[1], e0, eh);
  return 0;
}

/* Pointwise two-beam coupling of Eq. fov10 in crystal cells, simultaneous update. */
static void coupling_step(const orc_chan* c, const cplx* cf, const uint8_t* mk, cplx* e0, cplx* eh,
                          size_t n) {
  for (size_t i = 0; i < n; ++i) {
    if (!mk[i]) continue;
    cplx ap = e0[i], am = eh[i];
    e0[i] = c->a * ap + c->bp * cf[i] * am;
    eh[i] = c->a * am + c->bm * conj(cf[i]) * ap;
  }
}

/* Coefficients (a_i, b_i) of the product in Eq. split-op, applied left to    */
/* right, psi <- A(a_m dz) B(b_m dz) ... A(a_1 dz) B(b_1 dz) psi read as: for  */
/* i = 1..m, propagate by a_i dz, then couple by b_i dz:                      */
/*   order 1: a = (1), b = (1)                      (reduces to Eq. fov4)      */
/*   order 2: a = (0, 1), b = (1/2, 1/2)            (Strang)                   */
/*   order 4: a = (0, t, 1-2t, t), b = (t/2, (1-t)/2, (1-t)/2, t/2), with t    */
/*            the root 1/(2 - 2^(1/3)) = 1.35120719... of 2t^3 + (1-2t)^3 = 0  */
/*            (printed rounded as 1.3512).                                     */
/* Returns m, or 0 for an unknown order.                                       */
int orc_split_coefficients(int order, double* a, double* b) {
  if (order == 0 || order == 1) {
    a[0] = 1.0;
    b[0] = 1.0;
    return 1;
  }
  if (order == 2) {
    a[0] = 0.0, a[1] = 1.0;
    b[0] = 0.5, b[1] = 0.5;
    return 2;
  }
  if (order == 4) {
    double t = 1.0 / (2.0 - cbrt(2.0));
    a[0] = 0.0, a[1] = t, a[2] = 1.0 - 2.0 * t, a[3] = t;
    b[0] = 0.5 * t, b[1] = 0.5 * (1.0 - t), b[2] = 0.5 * (1.0 - t), b[3] = 0.5 * t;
    return 4;
  }
  return 0;
}

/* Propagators of a fraction f of the step: exp(i f dz [sqrt(...) - k]).      */
static void propagators_frac(const orc_problem* p, const orc_chan* c, double f, cplx* pp,
                             cplx* pm) {
  int ny = (p->dims == 3) ? p->ny : 1;
  for (int r = 0; r < ny; ++r) {
    double qy = (p->dims == 3) ? qfreq(r, p->ny, p->dy) : 0.0;
    for (int m = 0; m < p->nx; ++m) {
      double qx = qfreq(m, p->nx, p->dx);
      pp[(size_t)r * p->nx + m] = propagator(c->k, qx + 0.5 * c->h, qy, f * p->dz);
      pm[(size_t)r * p->nx + m] = propagator(c->k, qx - 0.5 * c->h, qy, f * p->dz);
    }
  }
}

/* Split-step z-march of Eq. fov10 for one channel, steps z_begin ..        */
/* z_begin+n_steps-1, fields e0/eh ([ny][nx]) advanced in place.              */
/* Step n is the product of Eq. split-op: for i = 1..m,                       */
/*   A(a_i dz): A+- <- IFFT(FFT(A+-) p+-(a_i dz))       (skipped if a_i = 0)   */
/*   B(b_i dz): in crystal cells, with the step coefficients of b_i dz,        */
/*     A+ <- a A+ + bp c(x,z_n) A-,   A- <- a A- + bm conj(c(x,z_n)) A+        */
/*     using the values before the update.                                    */
/* Every B of step n takes Pi and u at z_n (the operator B of Eq. split-op is */
/* written with delta-eps at the start of the step).                          */
int orc_march(const orc_problem* p, const double* u, double omega, int z_begin, int n_steps,
              cplx* e0, cplx* eh) {
  double sa[4], sb[4];
  int m = orc_split_coefficients(p->split_order, sa, sb);
  if (m == 0) return 4;
  orc_chan c[4];
  for (int i = 0; i < m; ++i) {
    int rc = chan_setup_frac(p, omega, sb[i], &c[i]);
    if (rc) return rc;
  }
  int ny = (p->dims == 3) ? p->ny : 1;
  size_t n = (size_t)p->nx * ny;
  cplx* pp = (cplx*)malloc(sizeof(cplx) * n * (size_t)m);
  cplx* pm = (cplx*)malloc(sizeof(cplx) * n * (size_t)m);
  cplx* cf = (cplx*)malloc(sizeof(cplx) * n);
  uint8_t* mk = (uint8_t*)malloc(n);
  if (!pp || !pm || !cf || !mk) {
    free(pp);
    free(pm);
    free(cf);
    free(mk);
    return 2;
  }
  for (int i = 0; i < m; ++i) propagators_frac(p, &c[i], sa[i], pp + n * i, pm + n * i);
  int rc = 0;
  for (int s = 0; s < n_steps; ++s) {
    int zn = z_begin + s;
    if (zn < 0 || zn >= p->nz) {
      rc = 3;
      break;
    }
    orc_deformation(p, u, zn, cf, mk);
    for (int i = 0; i < m; ++i) {
      if (sa[i] != 0.0) {
        orc_fft2(e0, p->nx, ny, -1);
        orc_fft2(eh, p->nx, ny, -1);
        for (size_t j = 0; j < n; ++j) {
          e0[j] *= pp[n * i + j];
          eh[j] *= pm[n * i + j];
        }
        orc_fft2(e0, p->nx, ny, +1);
        orc_fft2(eh, p->nx, ny, +1);
      }
      coupling_step(&c[i], cf, mk, e0, eh, n);
    }
  }
  free(pp);
  free(pm);
  free(cf);
  free(mk);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Whole run over channels: incident field, then n_steps of the march.       */
/* e0/eh: [n_ch][ny][nx]; channels spread over n_threads POSIX threads.      */
/* ------------------------------------------------------------------------- */
typedef struct {
  const orc_problem* p;
  const double* u;
  const double* omega;
  const cplx* S;
  int n_ch, n_steps, next_worker, stride;
  cplx *e0, *eh;
  int rc;
  int worker;
} run_ctx;

static void* run_worker(void* arg) {
  run_ctx* ctx = (run_ctx*)arg;
  const orc_problem* p = ctx->p;
  size_t n = (size_t)p->nx * ((p->dims == 3) ? p->ny : 1);
  for (int ch = ctx->worker; ch < ctx->n_ch; ch += ctx->stride) {
    cplx* e0 = ctx->e0 + (size_t)ch * n;
    cplx* eh = ctx->eh + (size_t)ch * n;
    incident_field(p, ctx->omega[ch], ctx->S[ch], e0, eh);
    int rc = orc_march(p, ctx->u, ctx->omega[ch], 0, ctx->n_steps, e0, eh);
    if (rc) ctx->rc = rc;
  }
  return NULL;
}

int orc_run(const orc_problem* p, const double* u, int n_ch, const double* omega, const cplx* S,
            int n_steps, cplx* e0, cplx* eh, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_ch) n_threads = n_ch;
  if (n_threads < 1) return 0;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  run_ctx* ctx = (run_ctx*)malloc(sizeof(run_ctx) * (size_t)n_threads);
  if (!th || !ctx) {
    free(th);
    free(ctx);
    return 2;
  }
  for (int t = 0; t < n_threads; ++t) {
    ctx[t] = (run_ctx){p, u, omega, S, n_ch, n_steps, 0, n_threads, e0, eh, 0, t};
    pthread_create(&th[t], NULL, run_worker, &ctx[t]);
  }
  int rc = 0;
  for (int t = 0; t < n_threads; ++t) {
    pthread_join(th[t], NULL);
    if (ctx[t].rc) rc = ctx[t].rc;
  }
  free(th);
  free(ctx);
  return rc;
}
