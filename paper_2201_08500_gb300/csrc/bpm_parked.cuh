// Resident march with one envelope parked in shared memory: the form of
// Nx = 8192, and the "parked" launch form of Nx = 1024..4096.
//
// One channel per block of T = N/16 threads (16 positions each).  At Nx = 8192
// both envelopes in registers need more than the 128 registers a 512-thread
// block allows, and the spills went to DRAM.  At Nx <= 4096 the parked form
// needs at most 128 registers and 3 (N + N/16) complex64 of shared memory
// (102.5 KB at 4096), so that two or more channel blocks share an SM and run
// their exchanges and butterflies at independent phases.  Here only one
// envelope lives in registers at a time: the other is parked in shared memory
// at the thread's own x positions (thread-private, so parking needs no
// barrier), and the two envelopes run the same single-envelope transform one
// after the other.  The arithmetic of every
// element is that of bpm_resident.cuh (same butterflies, twiddles, tables and
// coupling, in the same order), so the fields are bitwise the same.
//
// Shared memory: exchange buffer, E0 park and Eh park (N + N/16 complex64 each,
// the padded exchange size) and the reduction area: 209.4 KB at 8192.  Tables
// and stage twiddles are read from L2 (or TMEM).
//
// Barriers.  After the first radix-16 stage the transform splits into
// independent sub-transforms of L(1) = N/16 positions, each held by LN(1) =
// N/256 <= 32 threads of one warp in the layouts of stages 1 and 2, so the two
// middle exchanges (stage 1 -> 2 and back) are warp-local and synchronise with
// __syncwarp; only the first and the last exchange of a transform are
// block-wide.  The middle exchanges use the park area that is free while the
// envelope is in registers, the outer ones the exchange buffer: the first
// needs one block barrier (between its stores and its loads), the last two
// (its stores must wait for every warp's loads of the first).  A step adds one
// barrier at its start and one between the parking and the second transform:
// 8 block barriers a step.
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
// G channels per block (G x T threads; G > 1 at N = 1024, where a channel's 64
// threads would leave half of each block's tensor-memory lanes unused): each
// channel's T threads march their own channels with their own shared-memory
// region and synchronise through named barrier 1 + its index, so the G
// channels of a block run at independent phases like separate blocks.
template <int N, int SPLIT = 1, bool TMEM = false, bool WIDE = (N <= 4096), int G = 1>
struct Parked {
  static_assert(SPLIT == 1 || SPLIT == 2 || SPLIT == 4, "splitting order");
  static_assert(!TMEM || SPLIT != 4, "TMEM tables: one table set");
  using Gm = Geom<N>;
  static constexpr int T = Gm::T;
  static constexpr int S = Gm::S;
  static constexpr int kTabs = SPLIT == 4 ? 2 : 1;
  static_assert(G == 1 || (T % 32 == 0 && G * T <= 1024 && G <= 15), "channel groups of whole warps");
  // TMEM columns of the block: warps w and w + 4 share lanes, so each group of
  // four warps takes its own 128 columns
  static constexpr int kCols = 128 * (G * T >= 128 ? G * T / 128 : 1);
  // Wide layout (default at N <= 4096): stage twiddles loaded in 128-bit pairs
  // and the parked envelope in 128-bit slots.  At N = 8192 (128 registers for a
  // 512-thread block) and in the work-queue kernels the narrower per-element
  // layout spills less and measured faster.
  static constexpr bool kWide = WIDE;
  // Packed quarter-turn butterfly outputs (jout in bpm_fft.cuh): measured
  // faster at N <= 4096; at 8192, which spills at 128 registers, the scalar
  // outputs measured faster.
  static constexpr bool kPJ = (N <= 4096);

  __host__ __device__ static constexpr size_t xbuf_bytes() { return size_t(Pad<N>::kSlots) * sizeof(float2); }
  __host__ __device__ static constexpr size_t red_bytes() { return 64 * sizeof(double); }
  // The parks have the exchange buffer's padded size: each serves as the
  // second exchange buffer of the other envelope's transform.
  __host__ __device__ static constexpr size_t group_bytes() { return 3 * xbuf_bytes() + red_bytes(); }
  __host__ __device__ static constexpr size_t smem_bytes() { return size_t(G) * group_bytes(); }

  // Barrier of this channel's T threads: the block's when G = 1, otherwise
  // named barrier 1 + (channel group) over T threads.
  static BPM_DEV void gsync() {
    if constexpr (G == 1) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + int(threadIdx.x) / T), "r"(T) : "memory");
    }
  }

  // Per-element stage twiddles (twiddle_order on the host): stage s, output m
  // of thread t at tw_off(s) + (m - 1) LN(s) + t % LN(s).
  __host__ __device__ static constexpr int tw_off(int s) {
    return s == 0 ? 0 : tw_off(s - 1) + 15 * Gm::LN(s - 1);
  }
  template <int s>
  static BPM_DEV float2 twiddle(const float2* tw, int t, int m) {
    constexpr int ln = Gm::LN(s);
    return __ldg(tw + tw_off(s) + (m - 1) * ln + (t % ln));
  }

  // Stage twiddles in pairs (see twiddle_pairs on the host): stage s, outputs
  // m = 2i+1, 2i+2 (i = 0..7, the last pair padded) of thread t at float4
  // pair_off(s) + i LN(s) + t % LN(s), so one 128-bit load serves two outputs.
  __host__ __device__ static constexpr int pair_off(int s) {
    return s == 0 ? 0 : pair_off(s - 1) + 8 * Gm::LN(s - 1);
  }
  template <int s>
  static BPM_DEV float4 twiddle_pair(const float4* tw, int t, int i) {
    constexpr int ln = Gm::LN(s);
    return __ldg(tw + pair_off(s) + i * ln + (t % ln));
  }

  template <int s>
  static BPM_DEV void stage_fwd(float2 (&v)[16], const float4* tw, int t) {
    if constexpr (s < S - 1) {
      dft16_fwd<true, kPJ>(v);
      if constexpr (Gm::LN(s) == 2) {
        // W_32^(j m), j = t % 2: ones on even lanes, the fixed W_32^m on odd
        // ones, as immediates (no loads: the loaded twiddles made this
        // 512-thread kernel spill 300 B a thread).  Where the lane-pair swap
        // follows this stage they are applied after it (pair_twiddle: the
        // same constants on the same values, only the products by one left
        // out); otherwise selected per lane here (a branch on the lane
        // parity measured slower than the selection).
        if constexpr (!(kPairLast && s == S - 2)) {
          const bool odd = t & 1;
#pragma unroll
          for (int m = 1; m < 16; ++m)
            v[m] = c_mul(v[m], make_float2(odd ? w32_re(m) : 1.f, odd ? w32_im(m) : 0.f));
        }
      } else if constexpr (kWide) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 w = twiddle_pair<s>(tw, t, i);
          v[2 * i + 1] = c_mul(v[2 * i + 1], make_float2(w.x, w.y));
          if (i < 7) v[2 * i + 2] = c_mul(v[2 * i + 2], make_float2(w.z, w.w));
        }
      } else {
        const float2* t1 = reinterpret_cast<const float2*>(tw);
#pragma unroll
        for (int m = 1; m < 16; ++m) v[m] = c_mul(v[m], twiddle<s>(t1, t, m));
      }
    } else {
      last_stage<Gm::RLAST, false, true, kPJ>(v);
    }
  }

  template <int s>
  static BPM_DEV void stage_inv(float2 (&v)[16], const float4* tw, int t) {
    if constexpr (s < S - 1) {
      if constexpr (Gm::LN(s) == 2) {
        if constexpr (!(kPairLast && s == S - 2)) {  // see stage_fwd
          const bool odd = t & 1;
#pragma unroll
          for (int m = 1; m < 16; ++m)
            v[m] = c_mulc(v[m], make_float2(odd ? w32_re(m) : 1.f, odd ? w32_im(m) : 0.f));
        }
      } else if constexpr (kWide) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 w = twiddle_pair<s>(tw, t, i);
          v[2 * i + 1] = c_mulc(v[2 * i + 1], make_float2(w.x, w.y));
          if (i < 7) v[2 * i + 2] = c_mulc(v[2 * i + 2], make_float2(w.z, w.w));
        }
      } else {
        const float2* t1 = reinterpret_cast<const float2*>(tw);
#pragma unroll
        for (int m = 1; m < 16; ++m) v[m] = c_mulc(v[m], twiddle<s>(t1, t, m));
      }
      dft16_inv<true, kPJ>(v);
    } else {
      last_stage<Gm::RLAST, true, true, kPJ>(v);
    }
  }

  // Single-envelope exchange through the padded layout (Pad<N>, 64-bit slots).
  // WARP: the exchange moves data within each warp (the middle stages), so a
  // warp barrier orders it; LEAD: a leading barrier of that scope first (see
  // propagate for which exchange needs one).
  template <int SF, int ST, bool WARP, bool LEAD>
  static BPM_DEV void exchange(float2 (&v)[16], float2* x, int t) {
    using P = Pad<N>;
    float2* st = x + P::template base<SF>(t);
    const float2* ld = x + P::template base<ST>(t);
    if constexpr (LEAD) {
      if constexpr (WARP) __syncwarp(); else gsync();
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) st[P::template off<SF>(k)] = v[k];
    if constexpr (WARP) __syncwarp(); else gsync();
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = ld[P::template off<ST>(k)];
  }

  // One envelope: forward FFT, digit-reversed spectrum times the tilted
  // propagator (hi + lo table gt of this envelope), inverse FFT.
  // At N = 8192 (stages 16 x 16 x 16 x 2) the 32 positions of block b = t/2
  // of the last two stages belong to the lane pair (2b, 2b+1) in both layouts
  // (stage 2: 32 b + t%2 + 2k; stage 3: 16 t + k), so that exchange is done
  // with register shuffles between the pair: no shared memory, no barrier.
  static constexpr bool kPairLast = (S == 4 && Gm::RLAST == 2);

  static BPM_DEV float2 shfl_pair(float2 v) {
    return make_float2(__shfl_xor_sync(0xFFFFFFFFu, v.x, 1), __shfl_xor_sync(0xFFFFFFFFu, v.y, 1));
  }
  // In-place swap within the lane pair: the even lane sends v[8+i] and receives
  // the odd lane's v[i] into it, the odd lane the reverse.  Applied to stage-2
  // values it leaves the stage-3 positions 16 t + 2i in v[i] and 16 t + 2i + 1
  // in v[8+i] of every lane; applied to that arrangement it restores stage 2.
  static BPM_DEV void pair_swap(float2 (&v)[16], int t) {
    const bool odd = t & 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 r = shfl_pair(odd ? v[i] : v[8 + i]);
      if (odd) v[i] = r; else v[8 + i] = r;
    }
  }
  // The W_32 twiddles of stage S-2 on the swapped arrangement: before the
  // swap, odd lanes multiply their value m by W_32^m and even lanes by one;
  // after it, those products are exactly the values in v[8+i] (the even
  // lane's came from the odd lane's v[i], the odd lane's are its own v[8+i]),
  // so 8 products a thread replace 15.  INV: the conjugates, applied before
  // the swap that restores stage S-2.
  template <bool INV>
  static BPM_DEV void pair_twiddle(float2 (&v)[16], int t) {
    const bool odd = t & 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 w = make_float2(odd ? w32_re(8 + i) : (i == 0 ? 1.f : w32_re(i)),
                                   odd ? w32_im(8 + i) : (i == 0 ? 0.f : w32_im(i)));
      v[8 + i] = INV ? c_mulc(v[8 + i], w) : c_mul(v[8 + i], w);
    }
  }

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

  // Exchanges: block-wide through xa, warp-local through xb (twice), then
  // block-wide through xa after a leading barrier.  On entry no thread may
  // still be reading xa, and every read of xb must come before the first
  // exchange's barrier; on return xb is free and other threads may still load
  // from xa.
  static BPM_DEV void propagate(float2 (&v)[16], float2* xa, float2* xb, const float4* gt,
                                uint32_t tcol, const float4* tw, int t) {
    static_assert(S == 3 || (S == 4 && kPairLast), "parked form: 1024 <= N <= 8192, 4 exchanges");
    static_assert(Gm::LN(1) <= 32, "stage-1 sub-transforms within one warp");
    stage_fwd<0>(v, tw, t);
    exchange<0, 1, false, false>(v, xa, t);
    stage_fwd<1>(v, tw, t);
    exchange<1, 2, true, false>(v, xb, t);
    stage_fwd<2>(v, tw, t);
    if constexpr (kPairLast) {
      pair_swap(v, t);
      pair_twiddle<false>(v, t);
      float2 w[16];  // stage-3 register order (a renaming, no data movement)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        w[2 * i] = v[i];
        w[2 * i + 1] = v[8 + i];
      }
      stage_fwd<3>(w, tw, t);
      multiply(w, gt, tcol, t);
      stage_inv<3>(w, tw, t);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        v[i] = w[2 * i];
        v[8 + i] = w[2 * i + 1];
      }
      pair_twiddle<true>(v, t);
      pair_swap(v, t);
    } else {
      multiply(v, gt, tcol, t);
    }
    stage_inv<2>(v, tw, t);
    exchange<2, 1, true, true>(v, xb, t);
    stage_inv<1>(v, tw, t);
    exchange<1, 0, false, true>(v, xa, t);
    stage_inv<0>(v, tw, t);
  }

  // Parking, thread-private.  Wide: the 16 values as 8 float4 pairs
  // (v[2i], v[2i+1]) at slot 8 t + ((i + t) & 7), free of bank conflicts for
  // the 8 threads of a 128-bit phase.  Narrow: value k at k T + t (64-bit).
  static BPM_DEV int park_slot(int t, int i) { return 8 * t + ((i + t) & 7); }
  static BPM_DEV void park(const float2 (&v)[16], float2* p, int t) {
    if constexpr (kWide) {
      float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        q[park_slot(t, i)] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) p[k * T + t] = v[k];
    }
  }
  static BPM_DEV void unpark(float2 (&v)[16], const float2* p, int t) {
    if constexpr (kWide) {
      const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 w = q[park_slot(t, i)];
        v[2 * i] = make_float2(w.x, w.y);
        v[2 * i + 1] = make_float2(w.z, w.w);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = p[k * T + t];
    }
  }
  // Parked value k of this thread.
  static BPM_DEV float2 parked(const float2* p, int t, int k) {
    if constexpr (kWide) {
      const float4 w = reinterpret_cast<const float4*>(p)[park_slot(t, k / 2)];
      return (k % 2 == 0) ? make_float2(w.x, w.y) : make_float2(w.z, w.w);
    } else {
      return p[k * T + t];
    }
  }

  // [E0 in v, Eh parked] -> [Eh in v, E0 parked], both propagated (table set gt).
  // Before: each thread's last accesses of p0 and ph were to its own slots.
  // After: p0 and ph hold the parked E0 and (free) slots of Eh; other threads
  // may still load from x.
  static BPM_DEV void propagate_both(float2 (&v)[16], float2* x, float2* p0, float2* ph,
                                     const float4* gt, uint32_t tcol, const float4* tw, int t) {
    gsync();  // own-slot accesses of p0 / ph and loads of x are done
    propagate(v, x, p0, gt, tcol, tw, t);  // p0 is free while E0 is in registers
    park(v, p0, t);
    unpark(v, ph, t);
    gsync();  // x loads and the unparking of ph are done
    propagate(v, x, ph, gt + N, tcol + 64u, tw, t);
  }

  // [Eh in v, E0 parked] -> coupling at z_n -> [E0 in v, Eh parked].
  static BPM_DEV void couple_back(float2 (&v)[16], const float2* p0, float2* ph,
                                  const float2* crow, const ChannelCoef& cf, int t) {
    if constexpr (kWide) {
      const float4* q0 = reinterpret_cast<const float4*>(p0);
      float4* qh = reinterpret_cast<float4*>(ph);
#pragma unroll
      for (int i = 0; i < 8; ++i) {  // pair (2i, 2i+1)
        const float4 w = q0[park_slot(t, i)];
        float2 e0[2] = {make_float2(w.x, w.y), make_float2(w.z, w.w)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 c = __ldg(crow + t + T * (2 * i + h));
          if (c.x != 0.f || c.y != 0.f) couple_cell(e0[h], v[2 * i + h], c, cf);
        }
        qh[park_slot(t, i)] =
            make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
        v[2 * i] = e0[0];
        v[2 * i + 1] = e0[1];
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float2 c = __ldg(crow + t + T * k);
        float2 e0 = p0[k * T + t], eh = v[k];
        if (c.x != 0.f || c.y != 0.f) couple_cell(e0, eh, c, cf);
        ph[k * T + t] = eh;
        v[k] = e0;
      }
    }
  }

  // [E0 in v, Eh parked] -> coupling at z_n, same state.
  static BPM_DEV void couple_front(float2 (&v)[16], float2* ph, const float2* crow,
                                   const ChannelCoef& cf, int t) {
    if constexpr (kWide) {
      float4* qh = reinterpret_cast<float4*>(ph);
#pragma unroll
      for (int i = 0; i < 8; ++i) {  // pair (2i, 2i+1)
        const float4 w = qh[park_slot(t, i)];
        float2 eh[2] = {make_float2(w.x, w.y), make_float2(w.z, w.w)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 c = __ldg(crow + t + T * (2 * i + h));
          if (c.x != 0.f || c.y != 0.f) couple_cell(v[2 * i + h], eh[h], c, cf);
        }
        qh[park_slot(t, i)] = make_float4(eh[0].x, eh[0].y, eh[1].x, eh[1].y);
      }
    } else {
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
    float2* ph = p0 + Pad<N>::kSlots;
    double* red = reinterpret_cast<double*>(ph + Pad<N>::kSlots);
    const float4* gtab = A.tables + size_t(ch) * kTabs * 2 * N;
    // first order: the coupling coefficients are read from shared memory at
    // each coupling instead of held in eight registers across the transforms
    ChannelCoef* scf = reinterpret_cast<ChannelCoef*>(red + 32);
    if (SPLIT == 1 && t == 0) scf[0] = A.coef[ch];
    gsync();
    const ChannelCoef cfr = A.coef[size_t(ch) * kTabs];
    const ChannelCoef& cf = SPLIT == 1 ? scf[0] : cfr;
    const float4* tw = reinterpret_cast<const float4*>(kWide ? A.twiddle_p : A.twiddle_t);
    float2* e0 = A.e0 + size_t(ch) * N;
    float2* eh = A.eh + size_t(ch) * N;
    if constexpr (TMEM) tmem_fill(gtab, tcol, t);
    float2 v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = eh[t + T * k];
    park(v, ph, t);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = e0[t + T * k];
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
      const float2 m = parked(ph, t, k);
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
    gsync();
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
    gsync();  // smem reuse by the next channel
  }

  static BPM_DEV void run(const MarchArgs& A, unsigned char* smem) {
    const int tid = threadIdx.x;
    const int grp = G == 1 ? 0 : tid / T;  // channel group of this thread
    const int t = G == 1 ? tid : tid % T;
    unsigned char* gsmem = G == 1 ? smem : smem + size_t(grp) * group_bytes();
    if constexpr (TMEM) {
      __shared__ uint32_t s_tbase;
      if (tid / 32 == 0) tmem_alloc<kCols>(&s_tbase);
      tmem_sync();
      const uint32_t tbase = s_tbase;
      for (int ch = blockIdx.x * G + grp; ch < A.n_ch; ch += gridDim.x * G)
        march_channel(A, ch, gsmem, t, tmem_thread(tbase, tid));
      tmem_sync();  // every thread's TMEM loads have completed (waited)
      if (tid / 32 == 0) tmem_dealloc<kCols>(tbase);
    } else {
      for (int ch = blockIdx.x * G + grp; ch < A.n_ch; ch += gridDim.x * G)
        march_channel(A, ch, gsmem, t);
    }
  }

  static BPM_DEV void run_item(const MarchArgs& A, int ch0, unsigned char* smem) {
    static_assert(!TMEM && G == 1, "work-queue items: one channel a block, tables from L2");
    if (ch0 < A.n_ch) march_channel(A, ch0, smem, threadIdx.x);
  }
};

}  // namespace bpm
