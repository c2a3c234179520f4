// Register FFT of two float sequences at once with packed two-wide FP32 arithmetic.
//
// GB300 (sm_100 family) executes add/sub/mul/fma on a pair of floats held in one
// 64-bit register pair as a single instruction (.f32x2).  The column pass transforms
// two frequency columns A and B with identical operations, so every complex value of
// the transform is kept as a pair of pairs
//     CP = { re = (re_A, re_B), im = (im_A, im_B) }
// and every butterfly, rotation and twiddle product advances both columns with one
// instruction per real operation: half the arithmetic instructions of two separate
// float transforms, and one 16-byte shared-memory access per element and exchange.
//
// The algorithm is that of fft_reg.cuh (self-sorting Stockham stages of radix R with
// a small last stage, one shared-memory exchange between stages); only the element
// type and the twiddle form differ.  Twiddles are shared by A and B (same index):
// they are kept "broadcast", w -> (wr, wr), (wi, wi), (-wi, -wi), so that a product
// with a CP takes four packed instructions and no register shuffling.  A packed
// instruction still occupies the FMA pipe for two cycles, so the arithmetic that is
// the same for both columns (products of twiddles, sign flips) stays scalar or moves
// to the integer pipe.  The stage tables store, per k, the broadcast
// (wr, wr, wi, wi) of the exponents
// Q = 16: 1, 2, 3, 4, 8, 12;  Q = 8: 1, 2, 3, 4;  Q = 4: 1, 2, 3;  Q = 2: 1
// in planes [plane][k] (one 16-byte load each, consecutive k in consecutive threads);
// the other exponents are products of two stored ones, formed in scalar arithmetic.
#pragma once

#include "fft_reg.cuh"

namespace bem {
namespace pr {   // the pair forms; kept apart from the scalar templates of fft_reg.cuh

typedef unsigned long long f2x;   // two floats (lo, hi) in one 64-bit register pair

__device__ __forceinline__ f2x pk2(float lo, float hi) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void up2(f2x v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// a * b + c
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

struct __align__(16) CP {
  f2x re, im;
};

__device__ __forceinline__ CP cp_zero() { return CP{0ull, 0ull}; }
// (A, B) complex values -> CP and back
__device__ __forceinline__ CP cp_make(float2 a, float2 b) { return CP{pk2(a.x, b.x), pk2(a.y, b.y)}; }
__device__ __forceinline__ CP cp_load(const float4* p) {
  const float4 v = *p;
  return CP{pk2(v.x, v.y), pk2(v.z, v.w)};
}
__device__ __forceinline__ void cp_store(float4* p, CP c) {
  float4 v;
  up2(c.re, v.x, v.y);
  up2(c.im, v.z, v.w);
  *p = v;
}

__device__ __forceinline__ CP cadd(CP a, CP b) { return CP{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ CP csub(CP a, CP b) { return CP{sub2(a.re, b.re), sub2(a.im, b.im)}; }
// multiply both columns by a real pair (s_A, s_B)
__device__ __forceinline__ CP cscale2(CP a, f2x s) { return CP{mul2(a.re, s), mul2(a.im, s)}; }

// sign flip of both halves on the integer pipe (the FMA pipe is the busy one)
__device__ __forceinline__ f2x neg2(f2x a) {
  f2x d;
  asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(d) : "l"(a));
  return d;
}
__device__ __forceinline__ float negf(float a) { return __int_as_float(__float_as_int(a) ^ 0x80000000); }

// broadcast twiddle (wr, wr), (wi, wi), (-wi, -wi), and its scalar value w
struct TW {
  f2x r, i, ni;
  float2 w;
};
__device__ __forceinline__ TW tw_load(const float4* p) {
  const float4 v = *p;   // (wr, wr, wi, wi)
  const f2x i = pk2(v.z, v.w);
  return TW{pk2(v.x, v.y), i, neg2(i), make_float2(v.x, v.z)};
}
// product of two twiddles: one scalar complex product (the value is the same for
// both columns) broadcast by register moves
__device__ __forceinline__ TW tw_prod(const TW& a, const TW& b) {
  const float2 c = make_float2(a.w.x * b.w.x - a.w.y * b.w.y, a.w.x * b.w.y + a.w.y * b.w.x);
  return TW{pk2(c.x, c.x), pk2(c.y, c.y), pk2(negf(c.y), negf(c.y)), c};
}
// x * w (forward) or x * conj(w) (inverse)
template <bool INV>
__device__ __forceinline__ CP twmul(CP x, const TW& w) {
  if (INV) return CP{fma2(x.im, w.i, mul2(x.re, w.r)), fma2(x.re, w.ni, mul2(x.im, w.r))};
  return CP{fma2(x.im, w.ni, mul2(x.re, w.r)), fma2(x.im, w.r, mul2(x.re, w.i))};
}

// constant pairs
__device__ __forceinline__ f2x cpair(float c) { return pk2(c, c); }

// multiply by -+i (INV: +i); the negation is a sign flip on the integer pipe
template <bool INV>
__device__ __forceinline__ CP rot4(CP a) {
  return INV ? CP{neg2(a.im), a.re} : CP{a.im, neg2(a.re)};
}
// multiply by e^{-+ i pi/4}
template <bool INV>
__device__ __forceinline__ CP rot8(CP a) {
  const f2x r = cpair(0.70710678118654752440f);
  return INV ? CP{mul2(sub2(a.re, a.im), r), mul2(add2(a.re, a.im), r)}
             : CP{mul2(add2(a.re, a.im), r), mul2(sub2(a.im, a.re), r)};
}
// multiply by e^{-+ 3 i pi/4}
template <bool INV>
__device__ __forceinline__ CP rot8_3(CP a) {
  const f2x r = cpair(0.70710678118654752440f), nr = cpair(-0.70710678118654752440f);
  return INV ? CP{mul2(add2(a.re, a.im), nr), mul2(sub2(a.re, a.im), r)}
             : CP{mul2(sub2(a.im, a.re), r), mul2(add2(a.re, a.im), nr)};
}
// multiply by the constant e^{-+ i theta}, (c, s) = (cos, sin) theta
template <bool INV>
__device__ __forceinline__ CP rotc(CP a, float c, float s) {
  const f2x C = cpair(c), S = cpair(s), NS = cpair(-s);
  return INV ? CP{fma2(a.im, NS, mul2(a.re, C)), fma2(a.re, S, mul2(a.im, C))}
             : CP{fma2(a.im, S, mul2(a.re, C)), fma2(a.re, NS, mul2(a.im, C))};
}

template <bool INV>
__device__ __forceinline__ void dft2(CP& a, CP& b) {
  const CP t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// b + (-+i) d and b - (-+i) d without a negation
template <bool INV>
__device__ __forceinline__ void pm_rot4(CP b, CP d, CP& plus, CP& minus) {
  if (INV) {
    plus = CP{sub2(b.re, d.im), add2(b.im, d.re)};
    minus = CP{add2(b.re, d.im), sub2(b.im, d.re)};
  } else {
    plus = CP{add2(b.re, d.im), sub2(b.im, d.re)};
    minus = CP{sub2(b.re, d.im), add2(b.im, d.re)};
  }
}

// 4-point DFT of (v0, v1, v2, v3); Z2: v2 = v3 = 0
template <bool INV, bool Z2>
__device__ __forceinline__ void dft4z(CP& v0, CP& v1, CP& v2, CP& v3) {
  if (Z2) {
    const CP a = v0, c = v1;
    v0 = cadd(a, c);
    v2 = csub(a, c);
    pm_rot4<INV>(a, c, v1, v3);
  } else {
    const CP a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = csub(v1, v3);
    v0 = cadd(a, c);
    v2 = csub(a, c);
    pm_rot4<INV>(b, d, v1, v3);
  }
}

// 8-point DFT as in fft_reg.cuh; HALF: inputs 4..7 are zero
template <bool INV, bool HALF>
__device__ __forceinline__ void dft8(CP* v) {
  dft4z<INV, HALF>(v[0], v[2], v[4], v[6]);
  dft4z<INV, HALF>(v[1], v[3], v[5], v[7]);
  v[3] = rot8<INV>(v[3]);
  v[5] = rot4<INV>(v[5]);
  v[7] = rot8_3<INV>(v[7]);
  CP o[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[q] = cadd(v[2 * q], v[2 * q + 1]);
    o[q + 4] = csub(v[2 * q], v[2 * q + 1]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = o[q];
}

// 16-point DFT as in fft_reg.cuh; HALF: inputs 8..15 are zero
template <bool INV, bool HALF>
__device__ __forceinline__ void dft16(CP* v) {
#pragma unroll
  for (int k = 0; k < 4; ++k) dft4z<INV, HALF>(v[k], v[k + 4], v[k + 8], v[k + 12]);
  const float c = 0.92387953251128675613f, s = 0.38268343236508977173f;
  v[1 + 4] = rotc<INV>(v[1 + 4], c, s);      // w16^1
  v[2 + 4] = rot8<INV>(v[2 + 4]);            // w16^2
  v[3 + 4] = rotc<INV>(v[3 + 4], s, c);      // w16^3
  v[1 + 8] = rot8<INV>(v[1 + 8]);            // w16^2
  v[2 + 8] = rot4<INV>(v[2 + 8]);            // w16^4
  v[3 + 8] = rot8_3<INV>(v[3 + 8]);          // w16^6
  v[1 + 12] = rotc<INV>(v[1 + 12], s, c);    // w16^3
  v[2 + 12] = rot8_3<INV>(v[2 + 12]);        // w16^6
  v[3 + 12] = rotc<INV>(v[3 + 12], -c, -s);  // w16^9 = -w16^1
#pragma unroll
  for (int q = 0; q < 4; ++q) dft4z<INV, false>(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  CP o[16];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) o[q + 4 * p] = v[p + 4 * q];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

template <int Q, bool INV, bool HALF>
__device__ __forceinline__ void dftq(CP* v) {
  if constexpr (Q == 2) dft2<INV>(v[0], v[1]);
  if constexpr (Q == 4) dft4z<INV, HALF>(v[0], v[1], v[2], v[3]);
  if constexpr (Q == 8) dft8<INV, HALF>(v);
  if constexpr (Q == 16) dft16<INV, HALF>(v);
}

// stored broadcast twiddle planes of a stage of radix q (see the header comment)
__host__ __device__ constexpr int twp_planes(int q) { return q == 16 ? 6 : (q == 8 ? 4 : (q == 4 ? 3 : 1)); }
// exponent held by plane p of a stage of radix q
__host__ __device__ constexpr int twp_exponent(int q, int p) {
  return (q == 16 && p >= 4) ? 8 + 4 * (p - 4) : p + 1;
}
// offset (in float4 records) of the planes of stage s of a length-2^LOGL plan
template <int LOGL, int LOGR>
__host__ __device__ constexpr int twp_offset(int s) {
  using P = Plan<LOGL, LOGR>;
  int off = 0, ns = 1;
  for (int i = 0; i < s; ++i) {
    if (i > 0) off += twp_planes(P::radix(i)) * ns;
    ns *= P::radix(i);
  }
  return off;
}

// x(r) *= w_r (conjugated for INV), r = 1..Q-1, for one k of a stage whose planes
// start at tws (ns records per plane)
template <int Q, bool INV, typename X>
__device__ __forceinline__ void apply_twiddles_pair(const float4* tws, int ns, int k, X&& x) {
  const TW w1 = tw_load(tws + k);
  x(1) = twmul<INV>(x(1), w1);
  if constexpr (Q >= 4) {
    const TW w2 = tw_load(tws + ns + k), w3 = tw_load(tws + 2 * ns + k);
    x(2) = twmul<INV>(x(2), w2);
    x(3) = twmul<INV>(x(3), w3);
    if constexpr (Q >= 8) {
      const TW w4 = tw_load(tws + 3 * ns + k);
      x(4) = twmul<INV>(x(4), w4);
      x(5) = twmul<INV>(x(5), tw_prod(w1, w4));
      x(6) = twmul<INV>(x(6), tw_prod(w2, w4));
      x(7) = twmul<INV>(x(7), tw_prod(w3, w4));
      if constexpr (Q == 16) {
        const TW w8 = tw_load(tws + 4 * ns + k), w12 = tw_load(tws + 5 * ns + k);
        x(8) = twmul<INV>(x(8), w8);
        x(9) = twmul<INV>(x(9), tw_prod(w1, w8));
        x(10) = twmul<INV>(x(10), tw_prod(w2, w8));
        x(11) = twmul<INV>(x(11), tw_prod(w3, w8));
        x(12) = twmul<INV>(x(12), w12);
        x(13) = twmul<INV>(x(13), tw_prod(w1, w12));
        x(14) = twmul<INV>(x(14), tw_prod(w2, w12));
        x(15) = twmul<INV>(x(15), tw_prod(w3, w12));
      }
    }
  }
}

// Full transform of the pair on the thread's registers v[q] = x[t + T q] ->
// X[t + T q] (see reg_fft in fft_reg.cuh; same stages, exchanges and groups).
template <int LOGL, int LOGR, bool INV, bool HALF, int PER_BLOCK = 1>
__device__ __forceinline__ void pair_fft(CP* v, CP* sh, const float4* __restrict__ twp, int t, int group = 0) {
  using P = Plan<LOGL, LOGR>;
  constexpr int R = P::R, TT = P::T, RL = P::RL;
  int ns = 1;
#pragma unroll
  for (int s = 0; s < P::NSTAGES; ++s) {
    const bool small = (s == P::SR);
    if (s > 0) {
      const float4* tws = opaque(twp + twp_offset<LOGL, LOGR>(s));
      if (!small) {
        apply_twiddles_pair<R, INV>(tws, ns, t & (ns - 1), [&](int r) -> CP& { return v[r]; });
      } else {
#pragma unroll
        for (int b = 0; b < R / RL; ++b) {
          const int k = (t + TT * b) & (ns - 1);
          apply_twiddles_pair<RL, INV>(tws, ns, k, [&](int r) -> CP& { return v[b + r * (R / RL)]; });
        }
      }
    }
    if (!small) {
      if (s == 0 && HALF) dftq<R, INV, true>(v);
      else dftq<R, INV, false>(v);
    } else {
#pragma unroll
      for (int b = 0; b < R / RL; ++b) {
        CP w[RL > 1 ? RL : 2];
#pragma unroll
        for (int r = 0; r < RL; ++r) w[r] = v[b + r * (R / RL)];
        dftq<RL, INV, false>(w);
#pragma unroll
        for (int r = 0; r < RL; ++r) v[b + r * (R / RL)] = w[r];
      }
    }
    if (s + 1 < P::NSTAGES) {
      const int base = (t / ns) * ns * R + (t & (ns - 1));
#pragma unroll
      for (int r = 0; r < R; ++r) sh[padi<LOGR>(base + r * ns)] = v[r];
      GroupSync<TT, PER_BLOCK>::sync(group);
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = sh[padi<LOGR>(t + TT * q)];
      GroupSync<TT, PER_BLOCK>::sync(group);
    }
    ns *= small ? RL : R;
  }
}

}  // namespace pr
}  // namespace bem
