// Register/shared-memory FFT building blocks of the resident BPM march kernel.
//
// An N-point transform (N = 2^p, 256 <= N <= 8192) is split into S = ceil(p/4)
// decimation-in-frequency stages: S-1 radix-16 stages and a last stage of radix
// R = N / 16^(S-1) in {2, 4, 8, 16}.  Every thread owns 16 elements of each
// envelope, T = N/16 threads per channel.  Elements live at "positions" of the
// in-place Cooley-Tukey array:
//   stage s < S-1: thread t = (b, j) with b = t / L(s+1), j = t % L(s+1) holds
//                  positions b L(s) + j + L(s+1) k, k = 0..15;
//   stage S-1:     thread t holds positions 16 t + k.
// Stage 0 is therefore the natural x layout x = t + T k, which is the layout of
// the pointwise coupling step, and the last stage holds the spectrum in
// mixed-radix digit-reversed order, which is the layout of the propagator
// multiply.  The forward transform runs stages 0..S-1 (butterfly, then the
// inter-stage twiddle W_L(s)^(j m)); the inverse is its exact adjoint (stages
// S-1..0, conjugate twiddle, then the conjugate butterfly), so the forward and
// inverse twiddle phase errors cancel on the diagonal of every round trip.
// Between stages the 16 values per thread are exchanged through shared memory
// (the resident march uses the padded layout of Pad<N>; the 3D passes the
// XOR swizzle p ^ ((p >> 4) & 15)); both keep every access phase of a warp on
// distinct banks for all stages and sizes.
#pragma once

#include <cuda_runtime.h>

namespace bpm {

#define BPM_DEV __device__ __forceinline__

// Complex sums in packed FP32: one Blackwell two-lane instruction (FADD2 /
// FFMA2, sm_100 and later) does both components, each rounded exactly like the
// scalar operation, so the butterflies' additions take half the issue slots.
// a - b is fma(b, -1, a): b * -1 is exact, so the one rounding is that of a - b.
#ifndef BPM_PACKED_F32
#define BPM_PACKED_F32 1
#endif
// PA selects the packed form; the 3D passes (FUSE = false below) keep the
// scalar form, which measured faster there (they hold two envelopes and more
// live values, and the packed pairs cost registers).
template <bool PA = true>
BPM_DEV float2 c_add(float2 a, float2 b) {
#if BPM_PACKED_F32
  if constexpr (PA) return __fadd2_rn(a, b);
#endif
  return make_float2(a.x + b.x, a.y + b.y);
}
template <bool PA = true>
BPM_DEV float2 c_sub(float2 a, float2 b) {
#if BPM_PACKED_F32
  if constexpr (PA) return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
#endif
  return make_float2(a.x - b.x, a.y - b.y);
}
// p * s + a per component (one rounding each)
template <bool PA = true>
BPM_DEV float2 c_fmas(float2 p, float s, float2 a) {
#if BPM_PACKED_F32
  if constexpr (PA) return __ffma2_rn(p, make_float2(s, s), a);
#endif
  return make_float2(fmaf(p.x, s, a.x), fmaf(p.y, s, a.y));
}
BPM_DEV float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
BPM_DEV float2 c_mulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a * (hi + lo) for a two-term FP32 constant (the lo products enter first).
BPM_DEV float2 c_mul2(float2 a, float4 hl) {
  const float re = fmaf(a.x, hl.x, fmaf(-a.y, hl.y, fmaf(a.x, hl.z, -a.y * hl.w)));
  const float im = fmaf(a.x, hl.y, fmaf(a.y, hl.x, fmaf(a.x, hl.w, a.y * hl.z)));
  return make_float2(re, im);
}

// Radix-16/8 butterfly constants (correctly rounded FP32).  The host-side gain
// model in bpm_api.cu uses the same literals.
#define BPM_C8 0.70710678118654752440f
#define BPM_C16 0.92387953251128675613f
#define BPM_S16 0.38268343236508977173f

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

template <int N>
struct Geom {
  static constexpr int LOGN = ilog2c(N);
  static constexpr int T = N / 16;
  static constexpr int S = (LOGN + 3) / 4;
  static constexpr int RLAST = N >> (4 * (S - 1));
  __host__ __device__ static constexpr int L(int s) { return N >> (4 * s); }
  __host__ __device__ static constexpr int LN(int s) { return s < S - 1 ? (N >> (4 * (s + 1))) : 1; }
  template <int s>
  static BPM_DEV int pos(int t, int k) {
    if constexpr (s == S - 1) {
      return 16 * t + k;
    } else {
      constexpr int ln = LN(s);
      return (t / ln) * L(s) + (t % ln) + ln * k;
    }
  }
};

BPM_DEV int swz(int p) { return p ^ ((p >> 4) & 15); }

// Padded exchange layout of the resident march: position p lives at slot
// p + p/16 (one spare slot per 16), N + N/16 slots in all.  For every stage s
// the slot of (t, k) is padbase<s>(t) + padoff<s>(k), a per-thread base plus a
// compile-time constant (the positions of one thread step by LN(s) in k, and
// the low four bits of its base are below LN(s) when LN(s) < 16), so an
// exchange needs one address register per pattern.  Consecutive threads land
// on distinct banks for 64-bit (16-thread phases) and 128-bit (8-thread
// phases) accesses at every size and stage.
template <int N>
struct Pad {
  using Gm = Geom<N>;
  static constexpr int kSlots = N + N / 16;
  template <int s>
  static BPM_DEV int base(int t) {
    const int p = Gm::template pos<s>(t, 0);
    return p + (p >> 4);
  }
  template <int s>
  __host__ __device__ static constexpr int off(int k) {
    return s == Gm::S - 1 ? k : Gm::LN(s) * k + ((Gm::LN(s) * k) >> 4);
  }
};

BPM_DEV float2 c_swap(float2 z) { return make_float2(z.y, z.x); }

// b = d0 -+ i s d1 and d = d0 +- i s d1 (forward: -i, INV: +i): the outputs of
// a 4-point butterfly that take d1 turned by a quarter turn (and scaled by s).
// PJ: as two packed FMAs of the swapped pair (d1.y, d1.x), which costs a
// register swap; otherwise four scalar FMAs.  The rounding is the same either
// way (one rounding per component), so PJ only trades issue slots against
// registers: it measured faster in the parked 2048- and 4096-point marches and
// slower at 8192 points and in the 3D passes, which hold more live values.
template <bool INV, bool PJ>
BPM_DEV void jout(float2 d0, float2 d1, float s, float2& b, float2& d) {
#if BPM_PACKED_F32
  if constexpr (PJ) {
    const float2 q = c_swap(d1);
    b = __ffma2_rn(q, INV ? make_float2(-s, s) : make_float2(s, -s), d0);
    d = __ffma2_rn(q, INV ? make_float2(s, -s) : make_float2(-s, s), d0);
    return;
  }
#endif
  if (!INV) {
    b = make_float2(fmaf(d1.y, s, d0.x), fmaf(-d1.x, s, d0.y));
    d = make_float2(fmaf(-d1.y, s, d0.x), fmaf(d1.x, s, d0.y));
  } else {
    b = make_float2(fmaf(-d1.y, s, d0.x), fmaf(d1.x, s, d0.y));
    d = make_float2(fmaf(d1.y, s, d0.x), fmaf(-d1.x, s, d0.y));
  }
}

// 4-point DFT in place: forward y_m = sum_k v_k exp(-2 pi i k m / 4); INV conjugates.
template <bool INV, bool PJ = false, bool PA = true>
BPM_DEV void dft4(float2& a, float2& b, float2& c, float2& d) {
  const float2 s0 = c_add<PA>(a, c), d0 = c_sub<PA>(a, c), s1 = c_add<PA>(b, d),
               d1 = c_sub<PA>(b, d);
  a = c_add<PA>(s0, s1);
  c = c_sub<PA>(s0, s1);
  jout<INV, PJ>(d0, d1, 1.f, b, d);
}

template <bool PA = true>
BPM_DEV void dft2(float2& a, float2& b) {
  const float2 s = c_add<PA>(a, b);
  b = c_sub<PA>(a, b);
  a = s;
}

// z * W16^E (forward) or z * conj(W16^E) (INV), W16 = exp(-2 pi i / 16).
template <int E, bool INV>
BPM_DEV float2 w16(float2 z) {
  const float x = z.x, y = z.y;
  if constexpr (E == 0) {
    return z;
  } else if constexpr (E == 4) {
    return INV ? make_float2(-y, x) : make_float2(y, -x);
  } else if constexpr (E == 2) {
    return INV ? make_float2((x - y) * BPM_C8, (x + y) * BPM_C8)
               : make_float2((x + y) * BPM_C8, (y - x) * BPM_C8);
  } else if constexpr (E == 6) {
    return INV ? make_float2((-x - y) * BPM_C8, (x - y) * BPM_C8)
               : make_float2((y - x) * BPM_C8, (-x - y) * BPM_C8);
  } else if constexpr (E == 1) {
    return INV ? make_float2(fmaf(x, BPM_C16, -y * BPM_S16), fmaf(y, BPM_C16, x * BPM_S16))
               : make_float2(fmaf(x, BPM_C16, y * BPM_S16), fmaf(y, BPM_C16, -x * BPM_S16));
  } else if constexpr (E == 3) {
    return INV ? make_float2(fmaf(x, BPM_S16, -y * BPM_C16), fmaf(y, BPM_S16, x * BPM_C16))
               : make_float2(fmaf(x, BPM_S16, y * BPM_C16), fmaf(y, BPM_S16, -x * BPM_C16));
  } else {
    static_assert(E == 9, "radix-16 internal twiddle exponent");
    return INV ? make_float2(fmaf(-x, BPM_C16, y * BPM_S16), fmaf(-y, BPM_C16, -x * BPM_S16))
               : make_float2(fmaf(-x, BPM_C16, -y * BPM_S16), fmaf(x, BPM_S16, -y * BPM_C16));
  }
}

// The W16^2 and W16^6 rotations are c8 (x +- y, y -+ x): the +-1 combination
// P_E(z) below, scaled by c8.  Where such a rotated value enters a 4-point
// butterfly, the c8 product goes into the butterfly's additions as an FMA
// (dft4_c, dft4_bd) instead of being rounded on its own: the same FP32
// constants, two to four fewer instructions per butterfly.
template <int E, bool INV>
BPM_DEV float2 pre8(float2 z) {
  static_assert(E == 2 || E == 6, "W8 rotations");
  const float x = z.x, y = z.y;
  if constexpr (!INV) {
    return E == 2 ? make_float2(x + y, y - x) : make_float2(y - x, -x - y);
  } else {
    return E == 2 ? make_float2(x - y, x + y) : make_float2(-x - y, x - y);
  }
}

// Outputs of a 4-point DFT from s0 = a + c, d0 = a - c, s1 = b + d, d1 = b - d.
template <bool INV, bool PJ>
BPM_DEV void dft4_out(float2 s0, float2 d0, float2 s1, float2 d1, float2& a, float2& b, float2& c,
                      float2& d) {
  a = c_add(s0, s1);
  c = c_sub(s0, s1);
  jout<INV, PJ>(d0, d1, 1.f, b, d);
}

// dft4 whose input c still owes the rotation W16^E (E = 2 or 6).
template <int E, bool INV, bool PJ>
BPM_DEV void dft4_c(float2& a, float2& b, float2& c, float2& d) {
  const float2 p = pre8<E, INV>(c);
  const float2 s0 = c_fmas(p, BPM_C8, a);
  const float2 d0 = c_fmas(p, -BPM_C8, a);
  dft4_out<INV, PJ>(s0, d0, c_add(b, d), c_sub(b, d), a, b, c, d);
}

// dft4 whose input b still owes W16^2 and d still owes W16^6.
template <bool INV, bool PJ>
BPM_DEV void dft4_bd(float2& a, float2& b, float2& c, float2& d) {
  const float2 pb = pre8<2, INV>(b), pd = pre8<6, INV>(d);
  const float2 P = c_add(pb, pd), Q = c_sub(pb, pd);  // s1 = c8 P, d1 = c8 Q
  const float2 s0 = c_add(a, c), d0 = c_sub(a, c);
  a = c_fmas(P, BPM_C8, s0);
  c = c_fmas(P, -BPM_C8, s0);
  jout<INV, PJ>(d0, Q, BPM_C8, b, d);
}

// 16-point DFT of v[0..15] as 4 x 4: k = 4 k1 + k2, m = m1 + 4 m2.
// Forward: DFT4 over k1 (fixed k2), twiddle W16^(k2 m1), DFT4 over k2 (fixed m1);
// the result y[m] is left in v[m] (natural order).  FUSE: the W16^2 / W16^6
// twiddles inside the second butterflies (fewer instructions; the march
// kernels); otherwise each twiddle is rounded on its own (the 3D passes, where
// the fused form cost registers and measured slower).
template <bool FUSE = true, bool PJ = FUSE, bool PA = FUSE>
BPM_DEV void dft16_fwd(float2 (&v)[16]) {
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) dft4<false, PJ, PA>(v[k2], v[k2 + 4], v[k2 + 8], v[k2 + 12]);
  v[5] = w16<1, false>(v[5]);
  v[7] = w16<3, false>(v[7]);
  v[10] = w16<4, false>(v[10]);
  v[13] = w16<3, false>(v[13]);
  v[15] = w16<9, false>(v[15]);
  // register 4 m1 + k2 holds u[k2][m1]
  if constexpr (FUSE) {
    // the twiddles of v6, v9 (W16^2) and v11, v14 (W16^6) inside the butterflies
    dft4<false, PJ>(v[0], v[1], v[2], v[3]);
    dft4_c<2, false, PJ>(v[4], v[5], v[6], v[7]);
    dft4_bd<false, PJ>(v[8], v[9], v[10], v[11]);
    dft4_c<6, false, PJ>(v[12], v[13], v[14], v[15]);
  } else {
    v[6] = w16<2, false>(v[6]);
    v[9] = w16<2, false>(v[9]);
    v[11] = w16<6, false>(v[11]);
    v[14] = w16<6, false>(v[14]);
#pragma unroll
    for (int m1 = 0; m1 < 4; ++m1)
      dft4<false, PJ, PA>(v[4 * m1], v[4 * m1 + 1], v[4 * m1 + 2], v[4 * m1 + 3]);
  }
  // register 4 m1 + m2 holds y[m1 + 4 m2]: transpose (register renaming only)
  float2 o[16];
#pragma unroll
  for (int m1 = 0; m1 < 4; ++m1)
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) o[m1 + 4 * m2] = v[4 * m1 + m2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// Exact adjoint of dft16_fwd (unnormalised inverse DFT): y[m] in v[m] -> x[k] in v[k].
template <bool FUSE = true, bool PJ = FUSE, bool PA = FUSE>
BPM_DEV void dft16_inv(float2 (&v)[16]) {
  float2 o[16];
#pragma unroll
  for (int m1 = 0; m1 < 4; ++m1)
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) o[4 * m1 + m2] = v[m1 + 4 * m2];
#pragma unroll
  for (int m1 = 0; m1 < 4; ++m1)
    dft4<true, PJ, PA>(o[4 * m1], o[4 * m1 + 1], o[4 * m1 + 2], o[4 * m1 + 3]);
  o[5] = w16<1, true>(o[5]);
  o[7] = w16<3, true>(o[7]);
  o[10] = w16<4, true>(o[10]);
  o[13] = w16<3, true>(o[13]);
  o[15] = w16<9, true>(o[15]);
  if constexpr (FUSE) {
    // o6, o9 (conj W16^2) and o11, o14 (conj W16^6) rotate inside the butterflies
    dft4<true, PJ>(o[0], o[4], o[8], o[12]);
    dft4_c<2, true, PJ>(o[1], o[5], o[9], o[13]);
    dft4_bd<true, PJ>(o[2], o[6], o[10], o[14]);
    dft4_c<6, true, PJ>(o[3], o[7], o[11], o[15]);
  } else {
    o[6] = w16<2, true>(o[6]);
    o[9] = w16<2, true>(o[9]);
    o[11] = w16<6, true>(o[11]);
    o[14] = w16<6, true>(o[14]);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) dft4<true, PJ, PA>(o[k2], o[k2 + 4], o[k2 + 8], o[k2 + 12]);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// 8-point DFT of v[OFF..OFF+7] as 4 x 2: k = 2 k1 + k2, m = m1 + 4 m2.
template <int OFF, bool PJ, bool PA>
BPM_DEV void dft8_fwd(float2 (&v)[16]) {
  float2* w = v + OFF;
  dft4<false, PJ, PA>(w[0], w[2], w[4], w[6]);
  dft4<false, PJ, PA>(w[1], w[3], w[5], w[7]);
  // register 2 m1 + k2 holds u[k2][m1]; twiddle W8^(k2 m1) = W16^(2 k2 m1)
  w[3] = w16<2, false>(w[3]);
  w[5] = w16<4, false>(w[5]);
  w[7] = w16<6, false>(w[7]);
#pragma unroll
  for (int m1 = 0; m1 < 4; ++m1) dft2<PA>(w[2 * m1], w[2 * m1 + 1]);
  float2 o[8];
#pragma unroll
  for (int m1 = 0; m1 < 4; ++m1)
#pragma unroll
    for (int m2 = 0; m2 < 2; ++m2) o[m1 + 4 * m2] = w[2 * m1 + m2];
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = o[i];
}

template <int OFF, bool PJ, bool PA>
BPM_DEV void dft8_inv(float2 (&v)[16]) {
  float2* w = v + OFF;
  float2 o[8];
#pragma unroll
  for (int m1 = 0; m1 < 4; ++m1)
#pragma unroll
    for (int m2 = 0; m2 < 2; ++m2) o[2 * m1 + m2] = w[m1 + 4 * m2];
#pragma unroll
  for (int m1 = 0; m1 < 4; ++m1) dft2<PA>(o[2 * m1], o[2 * m1 + 1]);
  o[3] = w16<2, true>(o[3]);
  o[5] = w16<4, true>(o[5]);
  o[7] = w16<6, true>(o[7]);
  dft4<true, PJ, PA>(o[0], o[2], o[4], o[6]);
  dft4<true, PJ, PA>(o[1], o[3], o[5], o[7]);
#pragma unroll
  for (int i = 0; i < 8; ++i) w[i] = o[i];
}

// Last-stage butterflies: 16/R independent R-point DFTs on consecutive registers.
template <int R, bool INV, bool FUSE = true, bool PJ = FUSE, bool PA = FUSE>
BPM_DEV void last_stage(float2 (&v)[16]) {
  if constexpr (R == 16) {
    if (INV) dft16_inv<FUSE, PJ, PA>(v); else dft16_fwd<FUSE, PJ, PA>(v);
  } else if constexpr (R == 8) {
    if (INV) {
      dft8_inv<0, PJ, PA>(v);
      dft8_inv<8, PJ, PA>(v);
    } else {
      dft8_fwd<0, PJ, PA>(v);
      dft8_fwd<8, PJ, PA>(v);
    }
  } else if constexpr (R == 4) {
#pragma unroll
    for (int g = 0; g < 4; ++g)
      dft4<INV, PJ, PA>(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
  } else {
    static_assert(R == 2, "last-stage radix");
#pragma unroll
    for (int g = 0; g < 8; ++g) dft2<PA>(v[2 * g], v[2 * g + 1]);
  }
}

}  // namespace bpm
