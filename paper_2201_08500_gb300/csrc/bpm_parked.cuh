// Resident march with one envelope parked in shared memory: the form of
// Nx = 8192, and the "parked" launch form of Nx = 1024..4096.
//
// One channel per block of T = N/16 threads (16 positions each).  At Nx = 8192
// both envelopes in registers need more than the 128 registers a 512-thread
// block allows, and the spills went to DRAM.  At Nx <= 4096, with tables and
// twiddles read from L2, the parked form needs at most 128 registers and
// N (1 + 1/16 + 2) complex64 of shared memory (98 KB at 4096), so that two or
// more channel blocks share an SM and run their exchanges and butterflies at
// independent phases.  Here only one
// envelope lives in registers at a time: the other is parked in shared memory
// at the thread's own x positions (thread-private, so parking needs no
// barrier), and the two envelopes run the same single-envelope transform one
// after the other through a 64 KB exchange buffer.  The arithmetic of every
// element is that of bpm_resident.cuh (same butterflies, twiddles, tables and
// coupling, in the same order), so the fields are bitwise the same.
//
// Shared memory: exchange buffer (padded, N + N/16 complex64), E0 park, Eh park
// (N complex64 each) and the reduction area: 196.5 KB.  Tables and stage twiddles are read from L2.
//
// States of a step: [E0 in v, Eh parked] -> propagate E0 -> park E0, take Eh
// -> propagate Eh -> [Eh in v, E0 parked] -> couple (reading E0 back) ->
// [E0 in v, Eh parked].  Strang adds a coupling in the first state; fourth
// order runs three (propagate both, couple) rounds after it.
#pragma once

#include <cuda_runtime.h>

#include "bpm_resident.cuh"
#include "bpm_tmem.cuh"

namespace bpm {

// TMEM = true keeps each thread's propagator-table slice in tensor memory
// (bpm_tmem.cuh, 128 columns per thread: 2 envelopes x 16 positions x hi/lo
// float4) instead of reading it from L2 every step (one table set: SPLIT 1, 2).
template <int N, int SPLIT = 1, bool TMEM = false>
struct Parked {
  static_assert(SPLIT == 1 || SPLIT == 2 || SPLIT == 4, "splitting order");
  static_assert(!TMEM || SPLIT != 4, "TMEM tables: one table set");
  using Gm = Geom<N>;
  static constexpr int T = Gm::T;
  static constexpr int S = Gm::S;
  static constexpr int kTabs = SPLIT == 4 ? 2 : 1;
  // TMEM columns of the block: warps w and w + 4 share lanes, so each group of
  // four warps takes its own 128 columns
  static constexpr int kCols = 128 * (T >= 128 ? T / 128 : 1);

  __host__ __device__ static constexpr size_t xbuf_bytes() { return size_t(Pad<N>::kSlots) * sizeof(float2); }
  __host__ __device__ static constexpr size_t vec_bytes() { return size_t(N) * sizeof(float2); }
  __host__ __device__ static constexpr size_t red_bytes() { return 64 * sizeof(double); }
  __host__ __device__ static constexpr size_t smem_bytes() {
    return xbuf_bytes() + 2 * vec_bytes() + red_bytes();
  }

  // Offset of stage s in the thread-ordered twiddle table (see twiddle_order).
  __host__ __device__ static constexpr int tw_off(int s) {
    return s == 0 ? 0 : tw_off(s - 1) + 15 * Gm::LN(s - 1);
  }
  template <int s>
  static BPM_DEV float2 twiddle(const float2* tw, int t, int m) {
    constexpr int ln = Gm::LN(s);
    return __ldg(tw + tw_off(s) + (m - 1) * ln + (t % ln));
  }

  template <int s>
  static BPM_DEV void stage_fwd(float2 (&v)[16], const float2* tw, int t) {
    if constexpr (s < S - 1) {
      dft16_fwd(v);
#pragma unroll
      for (int m = 1; m < 16; ++m) v[m] = c_mul(v[m], twiddle<s>(tw, t, m));
    } else {
      last_stage<Gm::RLAST, false>(v);
    }
  }

  template <int s>
  static BPM_DEV void stage_inv(float2 (&v)[16], const float2* tw, int t) {
    if constexpr (s < S - 1) {
#pragma unroll
      for (int m = 1; m < 16; ++m) v[m] = c_mulc(v[m], twiddle<s>(tw, t, m));
      dft16_inv(v);
    } else {
      last_stage<Gm::RLAST, true>(v);
    }
  }

  // Single-envelope exchange through the padded layout (Pad<N>, 64-bit slots).
  template <int SF, int ST>
  static BPM_DEV void exchange(float2 (&v)[16], float2* x, int t) {
    using P = Pad<N>;
    float2* st = x + P::template base<SF>(t);
    const float2* ld = x + P::template base<ST>(t);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) st[P::template off<SF>(k)] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = ld[P::template off<ST>(k)];
  }

  // One envelope: forward FFT, digit-reversed spectrum times the tilted
  // propagator (hi + lo table gt of this envelope), inverse FFT.
  // Table multiply of one envelope: 16 positions, hi/lo float4 each, from L2
  // (gt) or from this thread's TMEM columns (tcol).
  static BPM_DEV void multiply(float2 (&v)[16], const float4* gt, uint32_t tcol, int t) {
    if constexpr (TMEM) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float4 tv[4];
        tmem_ld16(tcol + uint32_t(16 * c), tv);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 4; ++i) v[4 * c + i] = c_mul2(v[4 * c + i], tv[i]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = c_mul2(v[k], __ldg(gt + k * T + t));
    }
  }

  static BPM_DEV void propagate(float2 (&v)[16], float2* x, const float4* gt, uint32_t tcol,
                                const float2* tw, int t) {
    static_assert(S == 3 || S == 4, "parked form: 1024 <= N <= 8192");
    stage_fwd<0>(v, tw, t);
    exchange<0, 1>(v, x, t);
    stage_fwd<1>(v, tw, t);
    exchange<1, 2>(v, x, t);
    stage_fwd<2>(v, tw, t);
    if constexpr (S == 4) {
      exchange<2, 3>(v, x, t);
      stage_fwd<3>(v, tw, t);
    }
    multiply(v, gt, tcol, t);
    if constexpr (S == 4) {
      stage_inv<3>(v, tw, t);
      exchange<3, 2>(v, x, t);
    }
    stage_inv<2>(v, tw, t);
    exchange<2, 1>(v, x, t);
    stage_inv<1>(v, tw, t);
    exchange<1, 0>(v, x, t);
    stage_inv<0>(v, tw, t);
  }

  // [E0 in v, Eh parked] -> [Eh in v, E0 parked], both propagated (table set gt).
  static BPM_DEV void propagate_both(float2 (&v)[16], float2* x, float2* p0, float2* ph,
                                     const float4* gt, uint32_t tcol, const float2* tw, int t) {
    propagate(v, x, gt, tcol, tw, t);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      p0[k * T + t] = v[k];
      v[k] = ph[k * T + t];
    }
    propagate(v, x, gt + N, tcol + 64u, tw, t);
  }

  // [Eh in v, E0 parked] -> coupling at z_n -> [E0 in v, Eh parked].
  static BPM_DEV void couple_back(float2 (&v)[16], const float2* p0, float2* ph,
                                  const float2* crow, const ChannelCoef& cf, int t) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 c = __ldg(crow + t + T * k);
      float2 e0 = p0[k * T + t], eh = v[k];
      if (c.x != 0.f || c.y != 0.f) couple_cell(e0, eh, c, cf);
      ph[k * T + t] = eh;
      v[k] = e0;
    }
  }

  // [E0 in v, Eh parked] -> coupling at z_n, same state.
  static BPM_DEV void couple_front(float2 (&v)[16], float2* ph, const float2* crow,
                                   const ChannelCoef& cf, int t) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 c = __ldg(crow + t + T * k);
      if (c.x != 0.f || c.y != 0.f) {
        float2 eh = ph[k * T + t];
        couple_cell(v[k], eh, c, cf);
        ph[k * T + t] = eh;
      }
    }
  }

  // This thread's TMEM address: lanes of its warp's quarter, its warp group's
  // 128 columns (envelope e, position k at columns 64 e + 4 k .. + 3).
  static BPM_DEV uint32_t tmem_thread(uint32_t tbase, int t) {
    const int w = t / 32;
    return tbase + (uint32_t(32 * (w % 4)) << 16) + uint32_t(128 * (w / 4));
  }

  // Copies channel ch's tables (one set) from L2 into this thread's columns.
  static BPM_DEV void tmem_fill(const float4* gtab, uint32_t tcol, int t) {
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float4 tv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) tv[i] = __ldg(gtab + e * N + (4 * c + i) * T + t);
        tmem_st16(tcol + uint32_t(64 * e + 16 * c), tv);
      }
    tmem_wait_st();
  }

  // March channel ch of plan A by A.n_steps steps (this block: T threads).
  static BPM_DEV void march_channel(const MarchArgs& A, int ch, unsigned char* smem, int t,
                                    uint32_t tcol = 0) {
    float2* x = reinterpret_cast<float2*>(smem);
    float2* p0 = x + Pad<N>::kSlots;
    float2* ph = p0 + N;
    double* red = reinterpret_cast<double*>(ph + N);
    const float4* gtab = A.tables + size_t(ch) * kTabs * 2 * N;
    const ChannelCoef cf = A.coef[size_t(ch) * kTabs];
    const float2* tw = A.twiddle_t;
    float2* e0 = A.e0 + size_t(ch) * N;
    float2* eh = A.eh + size_t(ch) * N;
    if constexpr (TMEM) tmem_fill(gtab, tcol, t);
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      v[k] = e0[t + T * k];
      ph[k * T + t] = eh[t + T * k];
    }
    for (int step = 0; step < A.n_steps; ++step) {
      const float2* crow = A.cfield + size_t(A.z0 + step) * N;
      if constexpr (SPLIT == 4) {
        const ChannelCoef cf1 = A.coef[size_t(ch) * 2 + 1];
        couple_front(v, ph, crow, cf, t);
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
          propagate_both(v, x, p0, ph, gtab + (j == 1 ? 2 * N : 0), tcol, tw, t);
          couple_back(v, p0, ph, crow, j == 2 ? cf : cf1, t);
        }
      } else {
        if constexpr (SPLIT == 2) couple_front(v, ph, crow, cf, t);
        propagate_both(v, x, p0, ph, gtab, tcol, tw, t);
        couple_back(v, p0, ph, crow, cf, t);
      }
    }
    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 m = ph[k * T + t];
      e0[t + T * k] = v[k];
      eh[t + T * k] = m;
      sa += double(v[k].x) * v[k].x + double(v[k].y) * v[k].y;
      sb += double(m.x) * m.x + double(m.y) * m.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sa += __shfl_xor_sync(0xFFFFFFFFu, sa, off);
      sb += __shfl_xor_sync(0xFFFFFFFFu, sb, off);
    }
    const int w = t / 32;
    if ((t & 31) == 0) {
      red[2 * w] = sa;
      red[2 * w + 1] = sb;
    }
    __syncthreads();
    if (t == 0) {
      sa = 0.0;
      sb = 0.0;
      for (int i = 0; i < T / 32; ++i) {
        sa += red[2 * i];
        sb += red[2 * i + 1];
      }
      const double inc = A.inc_norm[ch];
      A.refl[ch] = sb / inc;
      A.trans[ch] = sa / inc;
    }
    __syncthreads();  // smem reuse by the next channel
  }

  static BPM_DEV void run(const MarchArgs& A, unsigned char* smem) {
    const int t = threadIdx.x;
    if constexpr (TMEM) {
      __shared__ uint32_t s_tbase;
      if (t / 32 == 0) tmem_alloc<kCols>(&s_tbase);
      tmem_sync();
      const uint32_t tbase = s_tbase;
      for (int ch = blockIdx.x; ch < A.n_ch; ch += gridDim.x)
        march_channel(A, ch, smem, t, tmem_thread(tbase, t));
      tmem_sync();  // every thread's TMEM loads have completed (waited)
      if (t / 32 == 0) tmem_dealloc<kCols>(tbase);
    } else {
      for (int ch = blockIdx.x; ch < A.n_ch; ch += gridDim.x) march_channel(A, ch, smem, t);
    }
  }

  static BPM_DEV void run_item(const MarchArgs& A, int ch0, unsigned char* smem) {
    static_assert(!TMEM, "work-queue items read their tables from L2");
    if (ch0 < A.n_ch) march_channel(A, ch0, smem, threadIdx.x);
  }
};

}  // namespace bpm
