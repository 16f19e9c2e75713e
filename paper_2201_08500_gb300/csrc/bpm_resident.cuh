// Resident split-step march of one channel (shared by the single-plan and the
// work-queue kernels).  See bpm_march.cu for the step structure.
#pragma once

#include <cuda_runtime.h>

#include "bpm_fft.cuh"
#include "bpm_internal.h"

namespace bpm {

// Pointwise two-beam coupling of Eq. fov10 at one crystal cell (|c| = 1):
//   E0 <- a E0 + b+ c Eh,   Eh <- a Eh + b- conj(c) E0   (pre-update values),
// with a as FP32 hi + lo.
BPM_DEV void couple_cell(float2& p, float2& m, float2 c, const ChannelCoef& cf) {
  const float ahx = cf.a_hi.x, ahy = cf.a_hi.y, alx = cf.a_lo.x, aly = cf.a_lo.y;
  const float2 bpc = c_mul(cf.bp, c);   // b+ c
  const float2 bmc = c_mulc(cf.bm, c);  // b- conj(c)
  const float px = fmaf(ahx, p.x, fmaf(-ahy, p.y, fmaf(bpc.x, m.x, fmaf(-bpc.y, m.y,
                                                                          fmaf(alx, p.x, -aly * p.y)))));
  const float py = fmaf(ahx, p.y, fmaf(ahy, p.x, fmaf(bpc.x, m.y, fmaf(bpc.y, m.x,
                                                                         fmaf(alx, p.y, aly * p.x)))));
  const float mx = fmaf(ahx, m.x, fmaf(-ahy, m.y, fmaf(bmc.x, p.x, fmaf(-bmc.y, p.y,
                                                                          fmaf(alx, m.x, -aly * m.y)))));
  const float my = fmaf(ahx, m.y, fmaf(ahy, m.x, fmaf(bmc.x, p.y, fmaf(bmc.y, p.x,
                                                                         fmaf(alx, m.y, aly * m.x)))));
  p = make_float2(px, py);
  m = make_float2(mx, my);
}

template <int T, int G>
BPM_DEV void group_sync(int g) {
  if constexpr (G == 1 && T >= 32) {
    __syncthreads();
  } else if constexpr (T >= 32) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(T) : "memory");
  } else if constexpr (T == 16) {
    const unsigned lane = threadIdx.x & 31u;
    __syncwarp(lane < 16 ? 0x0000FFFFu : 0xFFFF0000u);
  } else {
    static_assert(T == 16, "threads per channel");
  }
}

// L2TAB selects the form with propagator tables and stage twiddles read from
// L2 (thread-ordered, coalesced) and the deformation row loaded at the
// coupling instead of prefetched, which fits in 128 registers and no table
// shared memory: two blocks per SM then run their FFT exchanges and butterflies
// at independent phases.
//
// SPLIT is the order of the operator splitting of Eq. split-op: 1 (propagate,
// couple), 2 (Strang: half couple, propagate, half couple) or 4 (couple t/2,
// propagate t, couple (1-t)/2, propagate 1-2t, couple (1-t)/2, propagate t,
// couple t/2; two propagator tables and two coefficient sets per channel,
// tables read from L2).  Every coupling of step n uses c(x, z_n).
template <int N, int G, int SPLIT = 1, bool L2TAB = false>
struct Resident {
  static_assert(SPLIT == 1 || SPLIT == 2 || SPLIT == 4, "splitting order");
  static constexpr bool STRANG = (SPLIT == 2);
  static constexpr int kTabs = SPLIT == 4 ? 2 : 1;   // propagator tables per channel
  using Gm = Geom<N>;
  static constexpr int T = Gm::T;
  static constexpr int S = Gm::S;
  static constexpr int NTW = S - 1;                  // stages carrying inter-stage twiddles
  static constexpr bool kTabSmem = !L2TAB && SPLIT != 4 && (N <= 4096);  // tables resident in smem
  static constexpr bool kTwRegs = !L2TAB && (N <= 4096);   // twiddles resident in registers
  static constexpr bool kPrefetchC = !L2TAB;               // deformation row loaded a step ahead
  static constexpr int kTwSlots = kTwRegs ? (NTW > 0 ? NTW : 1) : 1;

  __host__ __device__ static constexpr size_t tab_bytes() { return kTabSmem ? size_t(2) * N * sizeof(float4) : 0; }
  static constexpr bool kPadX = L2TAB;  // padded exchange layout (see exchange)
  __host__ __device__ static constexpr size_t buf_bytes() {
    return size_t(kPadX ? Pad<N>::kSlots : N) * sizeof(float4);
  }
  __host__ __device__ static constexpr size_t red_bytes() { return 64 * sizeof(double); }
  __host__ __device__ static constexpr size_t slot_bytes() { return tab_bytes() + buf_bytes() + red_bytes(); }
  __host__ __device__ static constexpr size_t smem_bytes() { return G * slot_bytes(); }

  // Offset of stage s in the thread-ordered twiddle table used when the
  // twiddles do not stay in registers (N = 8192): stage s, output m and
  // j = t % L(s+1) at tw[off(s) + (m - 1) L(s+1) + j], so that consecutive
  // threads read adjacent entries.
  __host__ __device__ static constexpr int tw_off(int s) {
    return s == 0 ? 0 : tw_off(s - 1) + 15 * Gm::LN(s - 1);
  }

  // Inter-stage twiddle of stage s for this thread and output m.
  template <int s>
  static BPM_DEV float2 twiddle(const float2 (&twr)[kTwSlots][15], const float2* tw, int t, int m) {
    if constexpr (kTwRegs) {
      return twr[s][m - 1];
    } else {
      constexpr int ln = Gm::LN(s);
      return __ldg(tw + tw_off(s) + (m - 1) * ln + (t % ln));
    }
  }

  template <int s>
  static BPM_DEV void stage_fwd(float2 (&a)[16], float2 (&b)[16], const float2 (&twr)[kTwSlots][15],
                                const float2* tw, int t) {
    if constexpr (s < S - 1) {
      dft16_fwd(a);
      dft16_fwd(b);
#pragma unroll
      for (int m = 1; m < 16; ++m) {
        const float2 w = twiddle<s>(twr, tw, t, m);
        a[m] = c_mul(a[m], w);
        b[m] = c_mul(b[m], w);
      }
    } else {
      last_stage<Gm::RLAST, false>(a);
      last_stage<Gm::RLAST, false>(b);
    }
  }

  template <int s>
  static BPM_DEV void stage_inv(float2 (&a)[16], float2 (&b)[16], const float2 (&twr)[kTwSlots][15],
                                const float2* tw, int t) {
    if constexpr (s < S - 1) {
#pragma unroll
      for (int m = 1; m < 16; ++m) {
        const float2 w = twiddle<s>(twr, tw, t, m);
        a[m] = c_mulc(a[m], w);
        b[m] = c_mulc(b[m], w);
      }
      dft16_inv(a);
      dft16_inv(b);
    } else {
      last_stage<Gm::RLAST, true>(a);
      last_stage<Gm::RLAST, true>(b);
    }
  }

  // Move both envelopes from the layout of stage SF to that of stage ST.  The
  // two envelopes of a position share one 16-byte slot {E0, Eh}, so each
  // element costs one 128-bit store and one 128-bit load.  The 128-register
  // L2 form uses the padded layout (Pad<N>: one base register per pattern,
  // constant offsets); the shared-memory form, with registers to spare, the
  // XOR swizzle, which measured faster there.  Both are free of bank conflicts
  // for 8-thread 128-bit phases at every size and stage.
  template <int SF, int ST>
  static BPM_DEV void exchange(float2 (&a)[16], float2 (&b)[16], float2* buf, int t, int g) {
    float4* b4 = reinterpret_cast<float4*>(buf);
    if constexpr (kPadX) {
      using P = Pad<N>;
      float4* st = b4 + P::template base<SF>(t);
      const float4* ld = b4 + P::template base<ST>(t);
      group_sync<T, G>(g);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        st[P::template off<SF>(k)] = make_float4(a[k].x, a[k].y, b[k].x, b[k].y);
      group_sync<T, G>(g);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 v = ld[P::template off<ST>(k)];
        a[k] = make_float2(v.x, v.y);
        b[k] = make_float2(v.z, v.w);
      }
    } else {
      group_sync<T, G>(g);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        b4[swz(Gm::template pos<SF>(t, k))] = make_float4(a[k].x, a[k].y, b[k].x, b[k].y);
      group_sync<T, G>(g);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 v = b4[swz(Gm::template pos<ST>(t, k))];
        a[k] = make_float2(v.x, v.y);
        b[k] = make_float2(v.z, v.w);
      }
    }
  }

  static BPM_DEV void fft_fwd(float2 (&a)[16], float2 (&b)[16], float2* buf,
                              const float2 (&twr)[kTwSlots][15], const float2* tw, int t, int g) {
    stage_fwd<0>(a, b, twr, tw, t);
    if constexpr (S > 1) {
      exchange<0, 1>(a, b, buf, t, g);
      stage_fwd<1>(a, b, twr, tw, t);
    }
    if constexpr (S > 2) {
      exchange<1, 2>(a, b, buf, t, g);
      stage_fwd<2>(a, b, twr, tw, t);
    }
    if constexpr (S > 3) {
      exchange<2, 3>(a, b, buf, t, g);
      stage_fwd<3>(a, b, twr, tw, t);
    }
    static_assert(S <= 4, "N <= 65536");
  }

  static BPM_DEV void fft_inv(float2 (&a)[16], float2 (&b)[16], float2* buf,
                              const float2 (&twr)[kTwSlots][15], const float2* tw, int t, int g) {
    if constexpr (S > 3) {
      stage_inv<3>(a, b, twr, tw, t);
      exchange<3, 2>(a, b, buf, t, g);
    }
    if constexpr (S > 2) {
      stage_inv<2>(a, b, twr, tw, t);
      exchange<2, 1>(a, b, buf, t, g);
    }
    if constexpr (S > 1) {
      stage_inv<1>(a, b, twr, tw, t);
      exchange<1, 0>(a, b, buf, t, g);
    }
    stage_inv<0>(a, b, twr, tw, t);
  }

  // Pointwise two-beam coupling of Eq. fov10 at one crystal cell (|c| = 1).
  static BPM_DEV void couple_in(float2& p, float2& m, float2 c, const ChannelCoef& cf) {
    couple_cell(p, m, c, cf);
  }

  // Coupling of this thread's 16 cells.  c = 0 marks vacuum (Pi = 0), where the
  // coupling is the identity (a = 1, b = 0) and nothing is computed.  Register
  // k of a warp holds 32 consecutive x, so the test is warp-uniform except at
  // the crystal's surfaces.
  static BPM_DEV void couple_row(float2 (&a)[16], float2 (&b)[16], const float2 (&c)[16],
                                 const ChannelCoef& cf) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (c[k].x != 0.f || c[k].y != 0.f) couple_in(a[k], b[k], c[k], cf);
  }

  // Loads this thread's inter-stage twiddles (kept in registers for N <= 4096).
  static BPM_DEV void load_twiddles(float2 (&twr)[kTwSlots][15], const float2* tw, int t) {
    if constexpr (kTwRegs) {
#pragma unroll
      for (int s = 0; s < NTW; ++s) {
        const int ln = N >> (4 * (s + 1));
        const int stride = 1 << (4 * s);
        const int j = t % ln;
#pragma unroll
        for (int m = 1; m < 16; ++m) twr[s][m - 1] = __ldg(tw + stride * j * m);
      }
    }
  }

  // One propagation A of Eq. split-op: forward FFT, the digit-reversed spectra
  // times the tilted propagators (smem copy `tab` or table `gt` in L2), inverse FFT.
  static BPM_DEV void propagate(float2 (&a)[16], float2 (&b)[16], float2* buf, const float4* tab,
                                const float4* gt, const float2 (&twr)[kTwSlots][15],
                                const float2* tw, int t, int g) {
    fft_fwd(a, b, buf, twr, tw, t, g);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float4 pa, pb;
      if constexpr (kTabSmem) {
        pa = tab[k * T + t];
        pb = tab[N + k * T + t];
      } else {
        pa = __ldg(gt + k * T + t);
        pb = __ldg(gt + N + k * T + t);
      }
      a[k] = c_mul2(a[k], pa);
      b[k] = c_mul2(b[k], pb);
    }
    fft_inv(a, b, buf, twr, tw, t, g);
  }

  // March channel ch of plan A by A.n_steps steps from z = A.z0 (this thread's
  // channel group g; T threads).  Ends with the group barrier, so the group's
  // shared memory may be reused afterwards.
  static BPM_DEV void march_channel(const MarchArgs& A, int ch, const float2 (&twr)[kTwSlots][15],
                                    unsigned char* smem, int g, int t) {
    unsigned char* slot = smem + size_t(g) * slot_bytes();
    float4* tab = reinterpret_cast<float4*>(slot);
    float2* buf = reinterpret_cast<float2*>(slot + tab_bytes());
    double* red = reinterpret_cast<double*>(slot + tab_bytes() + buf_bytes());

    const float4* gtab = A.tables + size_t(ch) * kTabs * 2 * N;
    if constexpr (kTabSmem) {
      for (int i = t; i < 2 * N; i += T) tab[i] = __ldg(gtab + i);
    }
    const ChannelCoef cf = A.coef[size_t(ch) * kTabs];
    float2 a[16], b[16];
    float2* e0 = A.e0 + size_t(ch) * N;
    float2* eh = A.eh + size_t(ch) * N;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a[k] = e0[t + T * k];
      b[k] = eh[t + T * k];
    }
    group_sync<T, G>(g);

    const float2* tw = kTwRegs ? A.twiddle : A.twiddle_t;
    for (int step = 0; step < A.n_steps; ++step) {
      const float2* crow = A.cfield + size_t(A.z0 + step) * N;
      float2 c[16];
      if constexpr (kPrefetchC || SPLIT != 1) {
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = __ldg(crow + t + T * k);
      }
      if constexpr (SPLIT == 4) {
        // B(t/2) A(t) B((1-t)/2) A(1-2t) B((1-t)/2) A(t) B(t/2): sub-step j
        // couples with set 0 (t/2) or 1 ((1-t)/2), then propagates with
        // table 0 (t dz) or 1 ((1-2t) dz); one copy of the FFT code
        const ChannelCoef cf1 = A.coef[size_t(ch) * 2 + 1];
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
          couple_row(a, b, c, j == 0 ? cf : cf1);
          propagate(a, b, buf, tab, gtab + (j == 1 ? 2 * N : 0), twr, tw, t, g);
        }
        couple_row(a, b, c, cf);
      } else {
        if constexpr (STRANG) couple_row(a, b, c, cf);  // B(dz/2) A(dz) B(dz/2), half-step cf
        propagate(a, b, buf, tab, gtab, twr, tw, t, g);
        if constexpr (!kPrefetchC && SPLIT == 1) {
#pragma unroll
          for (int k = 0; k < 16; ++k) c[k] = __ldg(crow + t + T * k);
        }
        couple_row(a, b, c, cf);
      }
    }

    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      e0[t + T * k] = a[k];
      eh[t + T * k] = b[k];
      sa += double(a[k].x) * a[k].x + double(a[k].y) * a[k].y;
      sb += double(b[k].x) * b[k].x + double(b[k].y) * b[k].y;
    }
    // reduce over the T threads of this channel
    constexpr int W = T < 32 ? T : 32;
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
      const unsigned mask = (T < 32) ? ((threadIdx.x & 31u) < 16 ? 0x0000FFFFu : 0xFFFF0000u)
                                     : 0xFFFFFFFFu;
      sa += __shfl_xor_sync(mask, sa, off);
      sb += __shfl_xor_sync(mask, sb, off);
    }
    if constexpr (T > 32) {
      const int w = t / 32;
      if ((t & 31) == 0) {
        red[2 * w] = sa;
        red[2 * w + 1] = sb;
      }
      group_sync<T, G>(g);
      if (t == 0) {
        sa = 0.0;
        sb = 0.0;
        for (int i = 0; i < T / 32; ++i) {
          sa += red[2 * i];
          sb += red[2 * i + 1];
        }
      }
    }
    if (t == 0) {
      const double inc = A.inc_norm[ch];
      A.refl[ch] = sb / inc;
      A.trans[ch] = sa / inc;
    }
    group_sync<T, G>(g);  // tab / red reuse by the next channel
  }

  // Single-plan launch: channel groups strided over the grid.
  static BPM_DEV void run(const MarchArgs& A, unsigned char* smem) {
    const int g = threadIdx.x / T;
    const int t = threadIdx.x % T;
    float2 twr[kTwSlots][15];
    load_twiddles(twr, A.twiddle, t);
    for (int ch = blockIdx.x * G + g; ch < A.n_ch; ch += gridDim.x * G)
      march_channel(A, ch, twr, smem, g, t);
  }

  // Work-queue item: channels ch0 .. ch0 + G - 1 of plan A (those < n_ch).
  static BPM_DEV void run_item(const MarchArgs& A, int ch0, unsigned char* smem) {
    const int g = threadIdx.x / T;
    const int t = threadIdx.x % T;
    if (g >= G) return;
    float2 twr[kTwSlots][15];
    load_twiddles(twr, A.twiddle, t);
    if (ch0 + g < A.n_ch) march_channel(A, ch0 + g, twr, smem, g, t);
  }
};


}  // namespace bpm
