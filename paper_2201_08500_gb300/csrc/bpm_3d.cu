// 3D (x, y, z) form of the two-beam BPM: the transverse field of one channel
// (Nx x Ny complex64 per envelope) does not fit on chip, so every z step
// streams both envelopes through HBM in two passes (Eq. fov4 with the 2D
// transverse Laplacian, Eq. fov10 coupling):
//
//   column pass : per x-frequency column (contiguous in memory): forward
//                 y-FFT, multiply by the tilted propagator p+-(qx, qy), inverse
//                 y-FFT, write back;
//   row pass    : per row y: inverse x-FFT, pointwise coupling with
//                 c(x, y, z_n) = Pi(x) exp(+i h u(x, y, z_n)), then the next
//                 step's forward x-FFT, write back.
//
// Between passes the fields are stored transposed, [ch][c][y]: c = sigma(px) is
// the x-spectrum position px of the FFT's digit-reversed order permuted by
// sigma(px) = (px % 16) T + px / 16 (T = Nx / 16), which is the order of the row
// FFT's registers (thread t holds px = 16 t + k at c = k T + t).  Columns are
// then contiguous for the column pass, which loads them straight into
// registers; the row pass does the transposition: a block of R rows stages its
// [c][R] tile in shared memory (R x 8-byte segments per column in HBM), both
// envelopes of an element side by side in one 16-byte slot.  Between reading
// the tile and rewriting it, each row's transforms exchange through the row's
// own padded region of the same shared memory.  A run of n steps is
// one row pass (forward x of the natural-order fields), then n x (column pass,
// row pass); the last row pass writes natural [ch][y][x] order.  Traffic:
// 2 passes x 2 envelopes x (8 B read + 8 B write) = 64 B per cell-update.
//
// Propagator: p(qx, qy) = exp(i dz [sqrt(K^2 - qy^2) - k]), K^2 = k^2 - (qx +- h/2)^2,
// written as an FP64 anchor exp(i dz [K - k]) per column (FP32 hi + lo, with
// 1/(Nx Ny) and the x round-trip gain folded in) times
// 1 + i c - c^2/2 - delta_y, where c = -dz qy^2 / (2K) (|c| < 1e-4 here, so the
// dropped terms are below 1e-12) and delta_y removes the y round-trip gain.
#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is fetched at run time)
#include <cuda_runtime.h>

#include "bpm_fft.cuh"
#include "bpm_internal.h"
#include "bpm_tma.cuh"

namespace bpm {
namespace {

// Synchronisation of one transform group of T threads (g = group index in the block).
template <int T>
BPM_DEV void g3_sync(int g) {
  if constexpr (T == 16) {
    __syncwarp((threadIdx.x & 16u) ? 0xFFFF0000u : 0x0000FFFFu);
  } else if constexpr (T == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(T) : "memory");
  }
}

// Row-pass tile of R rows: element (c, r) (transposed-spectrum column c, tile
// row r) at 16-byte slot c R + (r ^ tile_swz<R>(c)), holding (E0, Eh).  Every
// access of the pass to the tile is 128-bit, so a warp splits into 8-thread
// phases; the XOR keeps each phase on distinct 16-byte bank groups for the
// column-segment staging and the row reads and writes (these place 8
// consecutive threads on consecutive columns, which the XOR maps to distinct
// slots mod 8).
template <int R>
__host__ __device__ constexpr int tile_swz(int c) {
  static_assert(R >= 4, "row tiles of at least 4 rows");
  return R >= 8 ? c % 8 : (c >> 1) % 4;
}
template <int R>
BPM_DEV int tile_at(int c, int r) {
  return c * R + (r ^ tile_swz<R>(c));
}

// Paired (E0, Eh) transform of size N held by a group of T = N/16 threads, 16
// values per thread and envelope.  `buf` is the group's exchange area: element p
// of envelope e lives at buf[(swz(p) * stride) + e * estride].  PA: butterfly
// additions in packed FP32 (the column passes; the row pass, with more live
// values, measured faster with scalar additions).  Both column-pass forms use
// the same PA, so they compute bitwise the same fields.
template <int N, bool PA = false>
struct Fft2Env {
  using Gm = Geom<N>;
  static constexpr int T = Gm::T;
  static constexpr int S = Gm::S;
  // N = 512 (16 x 16 x 2): the second stage's twiddles W_32^(j m), j = t % 2,
  // are applied on the other side of the exchange into the radix-2 last
  // stage (twid_last), where they fall on 8 values a thread instead of 15.
  static constexpr bool kTwAfter = (S == 3 && Gm::LN(1) == 2);

  // Offset of stage s in the thread-ordered twiddle table (see twiddle_order).
  __host__ __device__ static constexpr int tw_off(int s) {
    return s == 0 ? 0 : tw_off(s - 1) + 15 * Gm::LN(s - 1);
  }

  // W_L(s)^(j m) of stage s for this thread (j = t % LN(s)): from the table,
  // or, when LN(s) = 2 (the second stage of a 512-point transform), the
  // W_32 powers as immediates selected by the lane parity (the same values).
  template <int s>
  static BPM_DEV float2 stage_tw(const float2* tw, int t, int m) {
    constexpr int ln = Gm::LN(s);
    if constexpr (ln == 2) {
      const bool odd = t & 1;
      return make_float2(odd ? w32_re(m) : 1.f, odd ? w32_im(m) : 0.f);
    } else {
      return __ldg(tw + tw_off(s) + (t % ln) + (m - 1) * ln);  // consecutive threads adjacent
    }
  }

  template <int s>
  static BPM_DEV void twid(float2 (&a)[16], float2 (&b)[16], const float2* tw, int t, bool inv) {
    if constexpr (kTwAfter && s == 1) return;  // see twid_last
#pragma unroll
    for (int m = 1; m < 16; ++m) {
      const float2 w = stage_tw<s>(tw, t, m);
      a[m] = inv ? c_mulc(a[m], w) : c_mul(a[m], w);
      b[m] = inv ? c_mulc(b[m], w) : c_mul(b[m], w);
    }
  }

  // W_32 factor, in the last stage's layout, of value k = 2i + 1 of thread t:
  // position 16 t + k held, in stage 1, value m = 8 (t % 2) + i of a thread
  // with j = 1, so its factor is W_32^m (values of even k had j = 0: factor
  // one).  The same constants on the same values as stage_tw before the
  // exchange, without the products by one.
  static BPM_DEV float2 last_tw(int t, int i) {
    const bool odd = t & 1;
    return make_float2(odd ? w32_re(8 + i) : (i == 0 ? 1.f : w32_re(i)),
                       odd ? w32_im(8 + i) : (i == 0 ? 0.f : w32_im(i)));
  }
  template <bool INV>
  static BPM_DEV void twid_last(float2 (&a)[16], float2 (&b)[16], int t) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 w = last_tw(t, i);
      a[2 * i + 1] = INV ? c_mulc(a[2 * i + 1], w) : c_mul(a[2 * i + 1], w);
      b[2 * i + 1] = INV ? c_mulc(b[2 * i + 1], w) : c_mul(b[2 * i + 1], w);
    }
  }

  // TR = 0: element p of envelope e at buf[swz(p) * stride + e * estride]
  // (the column pass).  TR < 0: buf is this group's own region of
  // Pad<N>::kSlots 16-byte (E0, Eh) slots in the padded layout, one base
  // register per pattern and compile-time offsets (the row pass).
  template <int SF, int ST, int TR>
  static BPM_DEV void xchg(float2 (&a)[16], float2 (&b)[16], float2* buf, int stride, int estride,
                           int t, int g) {
    g3_sync<T>(g);
    if constexpr (TR < 0) {
      float4* q = reinterpret_cast<float4*>(buf);
      float4* st = q + Pad<N>::template base<SF>(t);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        st[Pad<N>::template off<SF>(k)] = make_float4(a[k].x, a[k].y, b[k].x, b[k].y);
      g3_sync<T>(g);
      const float4* ld = q + Pad<N>::template base<ST>(t);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 v = ld[Pad<N>::template off<ST>(k)];
        a[k] = make_float2(v.x, v.y);
        b[k] = make_float2(v.z, v.w);
      }
    } else {
      static_assert(TR == 0, "exchange layout");
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int p = swz(Gm::template pos<SF>(t, k)) * stride;
        buf[p] = a[k];
        buf[p + estride] = b[k];
      }
      g3_sync<T>(g);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int p = swz(Gm::template pos<ST>(t, k)) * stride;
        a[k] = buf[p];
        b[k] = buf[p + estride];
      }
    }
  }

  template <int s>
  static BPM_DEV void sfwd(float2 (&a)[16], float2 (&b)[16], const float2* tw, int t) {
    if constexpr (s < S - 1) {
      dft16_fwd<false, false, PA>(a);
      dft16_fwd<false, false, PA>(b);
      twid<s>(a, b, tw, t, false);
    } else {
      last_stage<Gm::RLAST, false, false, false, PA>(a);
      last_stage<Gm::RLAST, false, false, false, PA>(b);
    }
  }

  template <int s>
  static BPM_DEV void sinv(float2 (&a)[16], float2 (&b)[16], const float2* tw, int t) {
    if constexpr (s < S - 1) {
      twid<s>(a, b, tw, t, true);
      dft16_inv<false, false, PA>(a);
      dft16_inv<false, false, PA>(b);
    } else {
      last_stage<Gm::RLAST, true, false, false, PA>(a);
      last_stage<Gm::RLAST, true, false, false, PA>(b);
    }
  }

  // natural layout (pos<0>) -> digit-reversed spectrum (pos<S-1>); TR selects
  // the exchange layout (see xchg).
  template <int TR = 0>
  static BPM_DEV void fwd(float2 (&a)[16], float2 (&b)[16], float2* buf, int stride, int estride,
                          const float2* tw, int t, int g) {
    sfwd<0>(a, b, tw, t);
    if constexpr (S > 1) {
      xchg<0, 1, TR>(a, b, buf, stride, estride, t, g);
      sfwd<1>(a, b, tw, t);
    }
    if constexpr (S > 2) {
      xchg<1, 2, TR>(a, b, buf, stride, estride, t, g);
      if constexpr (kTwAfter) twid_last<false>(a, b, t);
      sfwd<2>(a, b, tw, t);
    }
    static_assert(S <= 3, "3D transforms up to 4096 points");
  }

  template <int TR = 0>
  static BPM_DEV void inv(float2 (&a)[16], float2 (&b)[16], float2* buf, int stride, int estride,
                          const float2* tw, int t, int g) {
    if constexpr (S > 2) {
      sinv<2>(a, b, tw, t);
      if constexpr (kTwAfter) twid_last<true>(a, b, t);
      xchg<2, 1, TR>(a, b, buf, stride, estride, t, g);
    }
    if constexpr (S > 1) {
      sinv<1>(a, b, tw, t);
      xchg<1, 0, TR>(a, b, buf, stride, estride, t, g);
    }
    sinv<0>(a, b, tw, t);
  }
};

// Eq. fov10 coupling of one cell (E0 = p, Eh = m) with c = Pi exp(i h u) != 0:
// E0 <- a p + b+ c m, Eh <- a m + b- conj(c) p, a = a_hi + a_lo (both row
// passes use this, so they compute bitwise the same fields).
BPM_DEV void couple3d(float2& pa, float2& mb, float2 c, const ChannelCoef& cf) {
  const float ahx = cf.a_hi.x, ahy = cf.a_hi.y, alx = cf.a_lo.x, aly = cf.a_lo.y;
  const float2 bpc = c_mul(cf.bp, c);
  const float2 bmc = c_mulc(cf.bm, c);
  const float2 p = pa, m = mb;
  pa = make_float2(
      fmaf(ahx, p.x, fmaf(-ahy, p.y, fmaf(bpc.x, m.x, fmaf(-bpc.y, m.y, fmaf(alx, p.x, -aly * p.y))))),
      fmaf(ahx, p.y, fmaf(ahy, p.x, fmaf(bpc.x, m.y, fmaf(bpc.y, m.x, fmaf(alx, p.y, aly * p.x))))));
  mb = make_float2(
      fmaf(ahx, m.x, fmaf(-ahy, m.y, fmaf(bmc.x, p.x, fmaf(-bmc.y, p.y, fmaf(alx, m.x, -aly * m.y))))),
      fmaf(ahx, m.y, fmaf(ahy, m.x, fmaf(bmc.x, p.y, fmaf(bmc.y, p.x, fmaf(alx, m.y, aly * m.x))))));
}

// Row pass over R = RT / T rows y0 .. y0 + R - 1 of one channel (T = NX/16,
// RT = 256 or 512 threads: the tile height, and with it the length R x 8 bytes
// of every column segment the transposed load / store moves, is a tuning
// choice of the plan).
// MODE 0: natural rows (e0, eh) in, forward x, transposed (s0, sh) out.
// MODE 1: transposed in, inverse x, coupling, forward x, transposed out (in
// place: every block reads and writes only its own rows of each column).
// MODE 2: transposed in, inverse x, coupling, natural rows out.
template <int NX, int MODE, int RT>
__global__ void __launch_bounds__(RT, 512 / RT) row_pass_kernel(Pass3DArgs A) {
  constexpr int kRowThreads = RT;
  constexpr int T = NX / 16;
  constexpr int R = kRowThreads / T;  // rows per block
  constexpr int HALF = R / 2;         // float4 (two y values) per column segment
  constexpr int VEC = NX * HALF / kRowThreads;  // segment pieces per thread and envelope
  static_assert(VEC * kRowThreads == NX * HALF, "tile split");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* tile = reinterpret_cast<float4*>(smem_raw);  // [NX][R] (E0, Eh) slots, swizzled (tile_at)
  const int g = threadIdx.x / T;
  // row g's exchange region (Pad<NX>::kSlots 16-byte slots), overlapping the
  // tile: the transforms run between the tile's read and its rewrite
  float2* xrow = reinterpret_cast<float2*>(tile + size_t(g) * Pad<NX>::kSlots);
  const int t = threadIdx.x % T;
  const int ch = blockIdx.y;
  const int y0 = blockIdx.x * R;
  const int y = y0 + g;
  const size_t chb = size_t(ch) * A.ny * NX;
  float2 a[16], b[16];
  if constexpr (MODE == 0) {
    const float2* e0 = A.e0 + chb + size_t(y) * NX;
    const float2* eh = A.eh + chb + size_t(y) * NX;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a[k] = e0[t + T * k];
      b[k] = eh[t + T * k];
    }
  } else {
    // transposed load: column c, rows y0 .. y0 + R - 1 (R x 8 bytes contiguous),
    // piece h = rows 2h, 2h + 1 of both envelopes
    float4 v0[VEC], v1[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int i = threadIdx.x + j * kRowThreads;
      const size_t off = chb + size_t(i / HALF) * A.ny + y0 + 2 * (i % HALF);
      v0[j] = __ldg(reinterpret_cast<const float4*>(A.s0 + off));
      v1[j] = __ldg(reinterpret_cast<const float4*>(A.sh + off));
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int i = threadIdx.x + j * kRowThreads;
      const int c = i / HALF;
      const int h = i % HALF;
      // pieces 4..7 of every 8 store their odd row first: that keeps both
      // stores of an 8-thread phase on distinct bank groups when R >= 16
      const int sw = (h >> 2) & 1;
      const float4 lo = make_float4(v0[j].x, v0[j].y, v1[j].x, v1[j].y);
      const float4 hi = make_float4(v0[j].z, v0[j].w, v1[j].z, v1[j].w);
      tile[tile_at<R>(c, 2 * h + sw)] = sw ? hi : lo;
      tile[tile_at<R>(c, 2 * h + 1 - sw)] = sw ? lo : hi;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float4 v = tile[tile_at<R>(k * T + t, g)];
      a[k] = make_float2(v.x, v.y);
      b[k] = make_float2(v.z, v.w);
    }
    __syncthreads();  // the rows' exchange regions overlap the tile
    Fft2Env<NX>::template inv<-1>(a, b, xrow, 0, 0, A.twx, t, g);
    const float2* crow = A.cfield + (size_t(A.z) * A.ny + y) * NX;
    const int2 sp = __ldg(A.cspan + size_t(A.z) * A.ny + y);  // crystal extent of the row
    const ChannelCoef cf = A.coef[ch];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      // c = 0 marks vacuum, where the coupling is the identity (warp-uniform
      // except at the crystal's surfaces: a warp holds consecutive x); the row
      // is loaded only inside its crystal extent
      const int xk = t + T * k;
      const float2 c = (xk >= sp.x && xk < sp.y) ? __ldg(crow + xk) : make_float2(0.f, 0.f);
      if (c.x == 0.f && c.y == 0.f) continue;
      couple3d(a[k], b[k], c, cf);
    }
  }
  if constexpr (MODE == 2) {
    float2* e0 = A.e0 + chb + size_t(y) * NX;
    float2* eh = A.eh + chb + size_t(y) * NX;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      e0[t + T * k] = a[k];
      eh[t + T * k] = b[k];
    }
  } else {
    Fft2Env<NX>::template fwd<-1>(a, b, xrow, 0, 0, A.twx, t, g);
    __syncthreads();  // every row is done with its exchange region
#pragma unroll
    for (int k = 0; k < 16; ++k)
      tile[tile_at<R>(k * T + t, g)] = make_float4(a[k].x, a[k].y, b[k].x, b[k].y);
    __syncthreads();
    float4 v0[VEC], v1[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int i = threadIdx.x + j * kRowThreads;
      const int c = i / HALF;
      const int h = i % HALF;
      const int sw = (h >> 2) & 1;
      const float4 p = tile[tile_at<R>(c, 2 * h + sw)];
      const float4 q = tile[tile_at<R>(c, 2 * h + 1 - sw)];
      const float4 lo = sw ? q : p, hi = sw ? p : q;
      v0[j] = make_float4(lo.x, lo.y, hi.x, hi.y);
      v1[j] = make_float4(lo.z, lo.w, hi.z, hi.w);
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      const int i = threadIdx.x + j * kRowThreads;
      const size_t off = chb + size_t(i / HALF) * A.ny + y0 + 2 * (i % HALF);
      *reinterpret_cast<float4*>(A.s0 + off) = v0[j];
      *reinterpret_cast<float4*>(A.sh + off) = v1[j];
    }
  }
}

constexpr int kColThreads = 256;

// Column pass: each group of T = NY/16 threads transforms both envelopes of one
// stored column c, contiguous in the transposed layout.
template <int NY>
__global__ void __launch_bounds__(kColThreads, 2) col_pass_kernel(Pass3DArgs A) {
  constexpr int T = NY / 16;
  constexpr int W = kColThreads / T;  // columns per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x % T;
  const int ch = blockIdx.y;
  const int cs = blockIdx.x * W + g;
  float2* buf = reinterpret_cast<float2*>(smem_raw) + size_t(g) * 2 * NY;
  const size_t colb = (size_t(ch) * A.nx + cs) * NY;
  float2* e0 = A.s0 + colb;
  float2* eh = A.sh + colb;
  float2 a[16], b[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    a[k] = e0[t + T * k];
    b[k] = eh[t + T * k];
  }
  Fft2Env<NY, true>::fwd(a, b, buf, 1, NY, A.twy, t, g);
  const float4 an0 = __ldg(A.anchor + (size_t(ch) * 2 + 0) * A.nx + cs);
  const float4 an1 = __ldg(A.anchor + (size_t(ch) * 2 + 1) * A.nx + cs);
  const float g0 = __ldg(A.gcorr + (size_t(ch) * 2 + 0) * A.nx + cs);
  const float g1 = __ldg(A.gcorr + (size_t(ch) * 2 + 1) * A.nx + cs);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float2 qd = __ldg(A.qy + k * T + t);  // {qy^2, 1/g_y - 1} at position 16 t + k
    const float c0r = qd.x * g0, c1r = qd.x * g1;
    float2 v = c_mul2(a[k], an0);
    const float2 f0 = make_float2(fmaf(-0.5f * c0r, c0r, qd.y), c0r);
    a[k] = make_float2(fmaf(v.x, f0.x, fmaf(-v.y, f0.y, v.x)), fmaf(v.x, f0.y, fmaf(v.y, f0.x, v.y)));
    v = c_mul2(b[k], an1);
    const float2 f1 = make_float2(fmaf(-0.5f * c1r, c1r, qd.y), c1r);
    b[k] = make_float2(fmaf(v.x, f1.x, fmaf(-v.y, f1.y, v.x)), fmaf(v.x, f1.y, fmaf(v.y, f1.x, v.y)));
  }
  Fft2Env<NY, true>::inv(a, b, buf, 1, NY, A.twy, t, g);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    e0[t + T * k] = a[k];
    eh[t + T * k] = b[k];
  }
}

// Single-envelope transform of N points held by a group of T = N/16 threads,
// exchanging through the group's own region of Pad<N>::kSlots 64-bit slots
// (the padded layout of the 1D march: conflict-free, one base register per
// pattern).  Butterflies (with packed additions), twiddles and their order
// are those of the column pass's Fft2Env<N, true>, so every element is
// computed bitwise as there.
template <int N>
struct Fft1Env {
  using Gm = Geom<N>;
  static constexpr int T = Gm::T;
  static constexpr int S = Gm::S;
  static constexpr bool kTwAfter = Fft2Env<N>::kTwAfter;  // as there

  template <int s>
  static BPM_DEV void twid(float2 (&a)[16], const float2* tw, int t, bool inv) {
    if constexpr (kTwAfter && s == 1) return;  // see twid_last
#pragma unroll
    for (int m = 1; m < 16; ++m) {
      const float2 w = Fft2Env<N>::template stage_tw<s>(tw, t, m);
      a[m] = inv ? c_mulc(a[m], w) : c_mul(a[m], w);
    }
  }
  template <bool INV>
  static BPM_DEV void twid_last(float2 (&a)[16], int t) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 w = Fft2Env<N>::last_tw(t, i);
      a[2 * i + 1] = INV ? c_mulc(a[2 * i + 1], w) : c_mul(a[2 * i + 1], w);
    }
  }

  template <int SF, int ST>
  static BPM_DEV void xchg(float2 (&a)[16], float2* buf, int t, int g) {
    g3_sync<T>(g);  // the group's loads of the previous exchange are done
    float2* st = buf + Pad<N>::template base<SF>(t);
#pragma unroll
    for (int k = 0; k < 16; ++k) st[Pad<N>::template off<SF>(k)] = a[k];
    g3_sync<T>(g);
    const float2* ld = buf + Pad<N>::template base<ST>(t);
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = ld[Pad<N>::template off<ST>(k)];
  }

  template <int s>
  static BPM_DEV void sfwd(float2 (&a)[16], const float2* tw, int t) {
    if constexpr (s < S - 1) {
      dft16_fwd<false, false, true>(a);
      twid<s>(a, tw, t, false);
    } else {
      last_stage<Gm::RLAST, false, false, false, true>(a);
    }
  }

  template <int s>
  static BPM_DEV void sinv(float2 (&a)[16], const float2* tw, int t) {
    if constexpr (s < S - 1) {
      twid<s>(a, tw, t, true);
      dft16_inv<false, false, true>(a);
    } else {
      last_stage<Gm::RLAST, true, false, false, true>(a);
    }
  }

  static BPM_DEV void fwd(float2 (&a)[16], float2* buf, const float2* tw, int t, int g) {
    static_assert(S == 2 || S == 3, "3D transforms of 256..1024 points");
    sfwd<0>(a, tw, t);
    xchg<0, 1>(a, buf, t, g);
    sfwd<1>(a, tw, t);
    if constexpr (S == 3) {
      xchg<1, 2>(a, buf, t, g);
      if constexpr (kTwAfter) twid_last<false>(a, t);
      sfwd<2>(a, tw, t);
    }
  }

  static BPM_DEV void inv(float2 (&a)[16], float2* buf, const float2* tw, int t, int g) {
    if constexpr (S == 3) {
      sinv<2>(a, tw, t);
      if constexpr (kTwAfter) twid_last<true>(a, t);
      xchg<2, 1>(a, buf, t, g);
    }
    sinv<1>(a, tw, t);
    xchg<1, 0>(a, buf, t, g);
    sinv<0>(a, tw, t);
  }
};

// True in every thread of transform group g (T threads) iff `ok` is true in all
// of them (flags: one int per warp of the block, for T > 32).
template <int T>
BPM_DEV bool group_all(bool ok, int g, int* flags) {
  if constexpr (T == 16) {
    return __all_sync((threadIdx.x & 16u) ? 0xFFFF0000u : 0x0000FFFFu, ok);
  } else if constexpr (T == 32) {
    return __all_sync(0xFFFFFFFFu, ok);
  } else {
    const bool w = __all_sync(0xFFFFFFFFu, ok);
    if ((threadIdx.x & 31) == 0) flags[threadIdx.x / 32] = w ? 1 : 0;
    g3_sync<T>(g);
    bool all = true;
#pragma unroll
    for (int i = 0; i < T / 32; ++i) all = all && flags[g * (T / 32) + i] != 0;
    g3_sync<T>(g);
    return all;
  }
}

// Column pass streamed by the copy engine (launch form 1 of 3D plans).
// Persistent: every group of T = NY/16 threads walks its share of the
// 2 n_ch nx single-envelope columns (E0 columns first, then Eh; each NY
// contiguous complex64 in the transposed layout).  While it transforms one
// column, a bulk copy (cp.async.bulk, completing on the group's mbarrier)
// brings its next column into the group's stage buffer, so every SM keeps
// kColTmaBlocksPerSm x 256 / T columns of loads in flight under the
// arithmetic.  Results are stored straight from registers (coalesced).  The
// arithmetic of every element is that of col_pass_kernel.
// A wait that gives up writes kStatusTmaTimeout to *status, waits once more
// (bounded) for the group's copy in flight and ends the group's work.
constexpr int kColTmaThreads = 256;
#ifndef BPM_COL_TMA_BPS
#define BPM_COL_TMA_BPS 2
#endif
constexpr int kColTmaBlocksPerSm = BPM_COL_TMA_BPS;

template <int NY>
__global__ void __launch_bounds__(kColTmaThreads, kColTmaBlocksPerSm)
    col_pass_tma_kernel(Pass3DArgs A, int n_ch, int* status) {
  constexpr int T = NY / 16;
  constexpr int G = kColTmaThreads / T;  // groups (columns in flight) per block
  constexpr uint32_t kBytes = NY * sizeof(float2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x % T;
  float2* stage = reinterpret_cast<float2*>(smem_raw) + size_t(g) * NY;
  float2* xbuf = reinterpret_cast<float2*>(smem_raw) + size_t(G) * NY + size_t(g) * Pad<NY>::kSlots;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + size_t(G) * (NY + Pad<NY>::kSlots) *
                                                             sizeof(float2)) + g;
  int* flags = reinterpret_cast<int*>(bar - g + G);
  const long long n_cols = (long long)n_ch * A.nx;
  const long long n_items = 2 * n_cols;
  const long long stride = (long long)gridDim.x * G;
  long long item = (long long)blockIdx.x * G + g;
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  g3_sync<T>(g);
  if (t == 0 && item < n_items) {
    mbar_arrive_expect_tx(bar, kBytes);
    bulk_load(stage, (item < n_cols ? A.s0 : A.sh) + (item % n_cols) * NY, kBytes, bar);
  }
  uint32_t phase = 0;
  for (; item < n_items; item += stride) {
    if (!group_all<T>(mbar_wait(bar, phase), g, flags)) {
      if (t == 0) atomicExch(status, kStatusTmaTimeout);
      mbar_wait(bar, phase);  // the copy still in flight, bounded
      return;
    }
    phase ^= 1u;
    float2 a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = stage[t + T * k];
    g3_sync<T>(g);  // every read of the stage is done before it is refilled
    const long long next = item + stride;
    if (t == 0 && next < n_items) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, kBytes);
      bulk_load(stage, (next < n_cols ? A.s0 : A.sh) + (next % n_cols) * NY, kBytes, bar);
    }
    const int env = item < n_cols ? 0 : 1;
    const long long cidx = item % n_cols;
    const int ch = int(cidx / A.nx);
    const int cs = int(cidx % A.nx);
    Fft1Env<NY>::fwd(a, xbuf, A.twy, t, g);
    const float4 an = __ldg(A.anchor + (size_t(ch) * 2 + env) * A.nx + cs);
    const float gc = __ldg(A.gcorr + (size_t(ch) * 2 + env) * A.nx + cs);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 qd = __ldg(A.qy + k * T + t);  // {qy^2, 1/g_y - 1} at position 16 t + k
      const float cr = qd.x * gc;
      const float2 v = c_mul2(a[k], an);
      const float2 f = make_float2(fmaf(-0.5f * cr, cr, qd.y), cr);
      a[k] = make_float2(fmaf(v.x, f.x, fmaf(-v.y, f.y, v.x)), fmaf(v.x, f.y, fmaf(v.y, f.x, v.y)));
    }
    Fft1Env<NY>::inv(a, xbuf, A.twy, t, g);
    float2* col = (env == 0 ? A.s0 : A.sh) + cidx * NY;
#pragma unroll
    for (int k = 0; k < 16; ++k) col[t + T * k] = a[k];
  }
}

// Row pass streamed by the copy engine (MODE 1 of launch form 2 of 3D plans):
// inverse x, coupling, forward x of every row, tiles of R = RT / T rows in and
// out through tensor copies.  Persistent: each block walks the tiles
// (channel, y0) of the pass.  A tile of one envelope is the box {2R floats
// (R rows of y), NX columns c} of the transposed spectrum [ch][c][y]; the copy
// engine lays it in shared memory as NX segments of R x 8 bytes, 16-byte
// chunks swizzled within each 32/64/128-byte span (the span is the segment).
// A warp's row read (8 bytes from each of 32 consecutive c of one row) and
// output write then reach 8 of the 16 eight-byte bank pairs: four wavefronts
// an access (8 or 16 without the swizzle, at 32- or 64-byte segments), so a
// cell's two 64-bit reads cost what the 128-bit store and load of
// row_pass_kernel's staging cost.  While a block transforms one tile the
// next one arrives in the stage buffer (one mbarrier phase a tile).  The output
// tile goes into the rows' exchange regions once the forward transforms are
// done and leaves by tensor stores; the next tile's first exchange waits
// until those stores have read it.  Stage (2 x NX x R x 8 B) + exchange
// regions (R x Pad<NX>::kSlots x 16 B): 67 KB for three blocks a SM at R x 8
// = 32 or 64 bytes of 128-thread tiles, 134 KB for one block of 256 threads.
// The arithmetic of every element is that of row_pass_kernel MODE 1.
template <int NX, int RT>
struct RowTma {
  static constexpr int T = NX / 16;
  static constexpr int R = RT / T;                           // rows a tile
  static constexpr int kSeg = R * int(sizeof(float2));      // bytes of a column segment
  static constexpr int kBoxC = NX < 256 ? NX : 256;          // columns a tensor copy
  static constexpr int kBoxes = NX / kBoxC;
  static constexpr uint32_t kPlane = uint32_t(NX) * kSeg;   // one envelope's tile
  static constexpr uint32_t kStage = 2 * kPlane;
  static constexpr uint32_t kXchg =
      (uint32_t(R) * Pad<NX>::kSlots * uint32_t(sizeof(float4)) + 1023u) / 1024u * 1024u;
  // 1 KB of slack aligns the stage to the swizzle pattern's 1024-byte period
  static constexpr size_t kSmem = 1024 + size_t(kStage) + kXchg + 16;
  static constexpr int kBlocksPerSm = kSmem <= 70 * 1024 ? 3 : 1;
  static_assert(kSeg == 32 || kSeg == 64 || kSeg == 128, "segment = swizzle span");
  static_assert(kXchg >= kStage, "the output tile fits in the exchange regions");
  static_assert(kSmem <= 227 * 1024, "shared memory of a block");

  // Byte offset of element (c, r) in an envelope's tile: the copy engine's
  // swizzle (16-byte chunk index XOR bits 7.. of the offset, as many bits as
  // the span has chunks minus one).
  static BPM_DEV uint32_t at(int c, int r) {
    const uint32_t lin = uint32_t(c) * uint32_t(kSeg) + uint32_t(r) * 8u;
    return lin ^ (((lin >> 7) & uint32_t(kSeg / 16 - 1)) << 4);
  }
};

template <int NX, int RT>
__global__ void __launch_bounds__(RT, RowTma<NX, RT>::kBlocksPerSm)
    row_pass_tma_kernel(const __grid_constant__ CUtensorMap map0,
                        const __grid_constant__ CUtensorMap maph, Pass3DArgs A, int n_ch,
                        int* status) {
  using L = RowTma<NX, RT>;
  constexpr int T = L::T;
  constexpr int R = L::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* stage = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  unsigned char* xreg = stage + L::kStage;  // exchange regions, then the output tile
  uint64_t* bar = reinterpret_cast<uint64_t*>(xreg + L::kXchg);
  const int g = threadIdx.x / T;  // row of the tile
  const int t = threadIdx.x % T;
  float2* xrow = reinterpret_cast<float2*>(reinterpret_cast<float4*>(xreg) + size_t(g) * Pad<NX>::kSlots);
  const int tiles_per_ch = A.ny / R;
  const int n_tiles = n_ch * tiles_per_ch;
  // one thread: announce and issue the tensor copies of tile `tile`
  auto issue = [&](int tile) {
    const int cy = (tile / tiles_per_ch) * NX;
    const int x = 2 * (tile % tiles_per_ch) * R;
    mbar_arrive_expect_tx(bar, L::kStage);
#pragma unroll
    for (int bx = 0; bx < L::kBoxes; ++bx) {
      tma_load_2d(stage + bx * L::kBoxC * L::kSeg, &map0, x, cy + bx * L::kBoxC, bar);
      tma_load_2d(stage + L::kPlane + bx * L::kBoxC * L::kSeg, &maph, x, cy + bx * L::kBoxC, bar);
    }
  };
  int tile = blockIdx.x;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
    if (tile < n_tiles) issue(tile);
  }
  __syncthreads();
  uint32_t phase = 0;
  for (; tile < n_tiles; tile += gridDim.x) {
    if (!__syncthreads_and(mbar_wait(bar, phase))) {
      if (threadIdx.x == 0) {
        atomicExch(status, kStatusTmaTimeout);
        mbar_wait(bar, phase);  // the tile still in flight, bounded
        bulk_wait_all();
      }
      return;
    }
    phase ^= 1u;
    float2 a[16], b[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t o = L::at(k * T + t, g);
      a[k] = *reinterpret_cast<const float2*>(stage + o);
      b[k] = *reinterpret_cast<const float2*>(stage + L::kPlane + o);
    }
    const int ch = tile / tiles_per_ch;
    const int y0 = (tile % tiles_per_ch) * R;
    const int y = y0 + g;
    // the row's deformation factor, loaded under the inverse transform (zero
    // outside the row's crystal extent, where the coupling is the identity)
    const float2* crow = A.cfield + (size_t(A.z) * A.ny + y) * NX;
    const int2 sp = __ldg(A.cspan + size_t(A.z) * A.ny + y);
    float2 cv[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int xk = t + T * k;
      cv[k] = (xk >= sp.x && xk < sp.y) ? __ldg(crow + xk) : make_float2(0.f, 0.f);
    }
    if (threadIdx.x == 0) bulk_wait_read_all();  // the last tile's stores have read xreg
    __syncthreads();  // every read of the stage is done; xreg is free
    if (threadIdx.x == 0 && tile + int(gridDim.x) < n_tiles) {
      fence_proxy_async_smem();
      issue(tile + gridDim.x);
    }
    Fft2Env<NX>::template inv<-1>(a, b, xrow, 0, 0, A.twx, t, g);
    const ChannelCoef cf = A.coef[ch];
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (cv[k].x != 0.f || cv[k].y != 0.f) couple3d(a[k], b[k], cv[k], cf);
    Fft2Env<NX>::template fwd<-1>(a, b, xrow, 0, 0, A.twx, t, g);
    __syncthreads();  // every row is done with its exchange region
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t o = L::at(k * T + t, g);
      *reinterpret_cast<float2*>(xreg + o) = a[k];
      *reinterpret_cast<float2*>(xreg + L::kPlane + o) = b[k];
    }
    fence_proxy_async_smem();  // this thread's writes, before the copy engine reads them
    __syncthreads();
    if (threadIdx.x == 0) {
      const int cy = ch * NX;
#pragma unroll
      for (int bx = 0; bx < L::kBoxes; ++bx) {
        tma_store_2d(&map0, 2 * y0, cy + bx * L::kBoxC, xreg + bx * L::kBoxC * L::kSeg);
        tma_store_2d(&maph, 2 * y0, cy + bx * L::kBoxC, xreg + L::kPlane + bx * L::kBoxC * L::kSeg);
      }
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

// Per-channel sums of |E0|^2 and |Eh|^2 over the plane (FP64), divided by the
// incident norm.
__global__ void reduce3d_kernel(const float2* e0, const float2* eh, long long plane,
                                const double* inc, double* refl, double* trans) {
  const int ch = blockIdx.x;
  double sa = 0.0, sb = 0.0;
  for (long long i = threadIdx.x; i < plane; i += blockDim.x) {
    const float2 a = e0[ch * plane + i], b = eh[ch * plane + i];
    sa += double(a.x) * a.x + double(a.y) * a.y;
    sb += double(b.x) * b.x + double(b.y) * b.y;
  }
  __shared__ double ra[32], rb[32];
  for (int off = 16; off > 0; off >>= 1) {
    sa += __shfl_xor_sync(0xFFFFFFFFu, sa, off);
    sb += __shfl_xor_sync(0xFFFFFFFFu, sb, off);
  }
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x / 32] = sa;
    rb[threadIdx.x / 32] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sa = 0.0;
    sb = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) {
      sa += ra[w];
      sb += rb[w];
    }
    refl[ch] = sb / inc[ch];
    trans[ch] = sa / inc[ch];
  }
}

// The larger of the tile (NX x R slots) and the rows' exchange regions
// (R x Pad<NX>::kSlots slots), 16 bytes a slot.
template <int NX, int RT>
size_t row_smem() {
  return size_t(RT / (NX / 16)) * Pad<NX>::kSlots * sizeof(float4);
}

template <int NY>
size_t col_smem() {
  return size_t(kColThreads / (NY / 16)) * 2 * NY * sizeof(float2);
}

// Stage buffers, exchange regions, mbarriers and vote flags of col_pass_tma_kernel.
template <int NY>
size_t col_tma_smem() {
  constexpr int G = kColTmaThreads / (NY / 16);
  return size_t(G) * (NY + Pad<NY>::kSlots) * sizeof(float2) + G * sizeof(uint64_t) +
         (kColTmaThreads / 32) * sizeof(int);
}

template <int NX, int MODE, int RT>
cudaError_t row_launch(const Pass3DArgs& a, int n_ch, cudaStream_t s) {
  constexpr int R = RT / (NX / 16);
  dim3 grid(unsigned((a.ny + R - 1) / R), unsigned(n_ch));
  row_pass_kernel<NX, MODE, RT><<<grid, RT, row_smem<NX, RT>(), s>>>(a);
  return cudaGetLastError();
}

template <int NY>
cudaError_t col_launch(const Pass3DArgs& a, int n_ch, cudaStream_t s) {
  constexpr int W = kColThreads / (NY / 16);
  dim3 grid(unsigned(a.nx / W), unsigned(n_ch));
  col_pass_kernel<NY><<<grid, kColThreads, col_smem<NY>(), s>>>(a);
  return cudaGetLastError();
}

template <int NY>
cudaError_t col_tma_launch(const Pass3DArgs& a, int n_ch, int sms, int* status, cudaStream_t s) {
  constexpr int G = kColTmaThreads / (NY / 16);
  const long long items = 2LL * n_ch * a.nx;
  const long long need = (items + G - 1) / G;
  const int blocks = int(need < (long long)sms * kColTmaBlocksPerSm ? need
                                                                    : (long long)sms * kColTmaBlocksPerSm);
  col_pass_tma_kernel<NY><<<blocks, kColTmaThreads, col_tma_smem<NY>(), s>>>(a, n_ch, status);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled, fetched from the driver through the runtime (no
// link-time dependency on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return EncodeTiledFn(nullptr);
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Tensor map of one envelope's transposed spectrum [n_ch * NX][ny] complex64
// as FP32 pairs, boxes of the streamed row pass's tile.
template <int NX, int RT>
bool encode_row_map(CUtensorMap* m, float2* base, int ny, int n_ch) {
  using L = RowTma<NX, RT>;
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cuuint64_t(2) * ny, cuuint64_t(NX) * n_ch};
  const cuuint64_t strides[1] = {cuuint64_t(ny) * sizeof(float2)};
  const cuuint32_t box[2] = {cuuint32_t(2 * L::R), cuuint32_t(L::kBoxC)};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = L::kSeg == 32   ? CU_TENSOR_MAP_SWIZZLE_32B
                                : L::kSeg == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                : CU_TENSOR_MAP_SWIZZLE_128B;
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NX, int RT>
cudaError_t row_tma_launch(const Pass3DArgs& a, int n_ch, int sms, int* status, cudaStream_t s) {
  using L = RowTma<NX, RT>;
  if (a.ny % L::R != 0) return cudaErrorInvalidValue;
  CUtensorMap m0, mh;
  if (!encode_row_map<NX, RT>(&m0, a.s0, a.ny, n_ch) ||
      !encode_row_map<NX, RT>(&mh, a.sh, a.ny, n_ch))
    return cudaErrorInvalidValue;
  const long long tiles = (long long)n_ch * (a.ny / L::R);
  const long long cap = (long long)sms * L::kBlocksPerSm;
  const int blocks = int(tiles < cap ? tiles : cap);
  if (blocks == 0) return cudaSuccess;
  row_pass_tma_kernel<NX, RT><<<blocks, RT, L::kSmem, s>>>(m0, mh, a, n_ch, status);
  return cudaGetLastError();
}

template <int NX, int RT>
cudaError_t row_tma_attrs() {
  return cudaFuncSetAttribute(row_pass_tma_kernel<NX, RT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(RowTma<NX, RT>::kSmem));
}

template <int NX, int RT>
cudaError_t row_attrs() {
  cudaError_t e = cudaSuccess, r;
  const int smem = int(row_smem<NX, RT>());
  if ((r = cudaFuncSetAttribute(row_pass_kernel<NX, 0, RT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    e = r;
  if ((r = cudaFuncSetAttribute(row_pass_kernel<NX, 1, RT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    e = r;
  if ((r = cudaFuncSetAttribute(row_pass_kernel<NX, 2, RT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    e = r;
  return e;
}

template <int NY>
cudaError_t col_attrs() {
  cudaError_t e = cudaFuncSetAttribute(col_pass_kernel<NY>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(col_smem<NY>()));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(col_pass_tma_kernel<NY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(col_tma_smem<NY>()));
}

}  // namespace

bool pass3d_supported(int nx, int ny) {
  auto ok = [](int n) { return n == 256 || n == 512 || n == 1024; };
  return ok(nx) && ok(ny);
}

cudaError_t pass3d_set_attributes() {
  cudaError_t e = cudaSuccess, r;
  if ((r = row_attrs<256, 256>()) != cudaSuccess) e = r;
  if ((r = row_attrs<512, 256>()) != cudaSuccess) e = r;
  if ((r = row_attrs<1024, 256>()) != cudaSuccess) e = r;
  if ((r = row_attrs<256, 512>()) != cudaSuccess) e = r;
  if ((r = row_attrs<512, 512>()) != cudaSuccess) e = r;
  if ((r = row_attrs<1024, 512>()) != cudaSuccess) e = r;
  if ((r = col_attrs<256>()) != cudaSuccess) e = r;
  if ((r = col_attrs<512>()) != cudaSuccess) e = r;
  if ((r = col_attrs<1024>()) != cudaSuccess) e = r;
  if ((r = row_tma_attrs<256, 128>()) != cudaSuccess) e = r;
  if ((r = row_tma_attrs<512, 128>()) != cudaSuccess) e = r;
  if ((r = row_tma_attrs<512, 256>()) != cudaSuccess) e = r;
  if ((r = row_tma_attrs<1024, 256>()) != cudaSuccess) e = r;
  return e;
}

bool row_tma_supported(int nx, int row_threads) {
  return (nx == 256 && row_threads == 128) || (nx == 512 && (row_threads == 128 || row_threads == 256)) ||
         (nx == 1024 && row_threads == 256);
}

cudaError_t launch_row_pass_tma(int row_threads, const Pass3DArgs& a, int n_ch, int sms,
                                int* status, cudaStream_t s) {
  if (a.nx == 256 && row_threads == 128) return row_tma_launch<256, 128>(a, n_ch, sms, status, s);
  if (a.nx == 512 && row_threads == 128) return row_tma_launch<512, 128>(a, n_ch, sms, status, s);
  if (a.nx == 512 && row_threads == 256) return row_tma_launch<512, 256>(a, n_ch, sms, status, s);
  if (a.nx == 1024 && row_threads == 256) return row_tma_launch<1024, 256>(a, n_ch, sms, status, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_row_pass(int mode, int row_threads, const Pass3DArgs& a, int n_ch,
                            cudaStream_t s) {
#define BPM_ROW(NXV, RTV)                                                 \
  if (a.nx == NXV && row_threads == RTV) {                                \
    if (mode == 0) return row_launch<NXV, 0, RTV>(a, n_ch, s);            \
    if (mode == 1) return row_launch<NXV, 1, RTV>(a, n_ch, s);            \
    return row_launch<NXV, 2, RTV>(a, n_ch, s);                           \
  }
  BPM_ROW(256, 256) BPM_ROW(512, 256) BPM_ROW(1024, 256)
  BPM_ROW(256, 512) BPM_ROW(512, 512) BPM_ROW(1024, 512)
#undef BPM_ROW
  return cudaErrorInvalidValue;
}

cudaError_t launch_col_pass(int form, const Pass3DArgs& a, int n_ch, int sms, int* status,
                            cudaStream_t s) {
  if (form >= 1) {
    if (a.ny == 256) return col_tma_launch<256>(a, n_ch, sms, status, s);
    if (a.ny == 512) return col_tma_launch<512>(a, n_ch, sms, status, s);
    if (a.ny == 1024) return col_tma_launch<1024>(a, n_ch, sms, status, s);
    return cudaErrorInvalidValue;
  }
  if (a.ny == 256) return col_launch<256>(a, n_ch, s);
  if (a.ny == 512) return col_launch<512>(a, n_ch, s);
  if (a.ny == 1024) return col_launch<1024>(a, n_ch, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_reduce3d(const float2* e0, const float2* eh, long long plane, int n_ch,
                            const double* inc, double* refl, double* trans, cudaStream_t s) {
  reduce3d_kernel<<<n_ch, 256, 0, s>>>(e0, eh, plane, inc, refl, trans);
  return cudaGetLastError();
}

}  // namespace bpm
