// Register-resident Stockham FFT: each thread holds R complex values (R = 8 or 16);
// the threads of one transform exchange through a padded shared-memory buffer
// between stages.
//
// A length-L transform (L = 2^LOGL >= R) uses T = L/R threads and the stage
// radices R, ..., R, RL with RL = 2^(LOGL mod LOGR) (no small stage when that is 0).
// Stage s (span Ns, radix Q) takes x[j + r L/Q], multiplies by e^{-+2 pi i (j mod Ns) r / (Ns Q)},
// applies the Q-point DFT and writes y[(j/Ns) Ns Q + (j mod Ns) + r Ns] (the
// self-sorting form).  With j = t for radix-R stages and j = t + T b (b < R/RL)
// for the small last stage, thread t holds x[t + T q], q < R, before the first
// stage and X[t + T q] after the last one (natural order in both).
//
// Twiddles w_r = e^{-2 pi i k r/(Ns Q)} (k = j mod Ns) come from per-stage tables in
// global memory, built once per operator, laid out in planes [plane][k][2] (one
// 16-byte load per plane in float; consecutive threads read consecutive k).  Float
// stores a few per k: Q = 16: (w1, w2), (w3, w4), (w8, w12); Q = 8: (w1, w2), (w3, w4);
// Q = 4: (w1, w2), (w3, -); Q = 2: (w1, -); the others are products of two stored ones
// (w5 = w1 w4, w9 = w1 w8, w13 = w1 w12, ...), one rounding above a stored value, so
// that a stage costs 3 loads instead of 8.  Double (where the FP64 pipe, not the loads,
// bounds the pass) stores all of them: plane p holds (w_{2p+1}, w_{2p+2}).
#pragma once

#include "bem_internal.cuh"

namespace bem {

// --- small DFTs in registers (natural order in and out) -----------------------
template <typename T> struct Consts;
template <> struct Consts<float> {
  static constexpr float r2 = 0.70710678118654752440f;   // cos(pi/4)
  static constexpr float c8 = 0.92387953251128675613f;   // cos(pi/8)
  static constexpr float s8 = 0.38268343236508977173f;   // sin(pi/8)
};
template <> struct Consts<double> {
  static constexpr double r2 = 0.70710678118654752440;
  static constexpr double c8 = 0.92387953251128675613;
  static constexpr double s8 = 0.38268343236508977173;
};

// multiply by e^{-+ i pi/4} (INV: +)
template <bool INV, typename C, typename T>
__device__ __forceinline__ C rot8(C a) {
  const T r = Consts<T>::r2;
  return INV ? mk((a.x - a.y) * r, (a.x + a.y) * r) : mk((a.x + a.y) * r, (a.y - a.x) * r);
}
// multiply by e^{-+ 3 i pi/4}
template <bool INV, typename C, typename T>
__device__ __forceinline__ C rot8_3(C a) {
  const T r = Consts<T>::r2;
  return INV ? mk(-(a.x + a.y) * r, (a.x - a.y) * r) : mk((a.y - a.x) * r, -(a.x + a.y) * r);
}
// multiply by -+i
template <bool INV, typename C>
__device__ __forceinline__ C rot4(C a) {
  return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
}
// multiply by a constant e^{-+ i theta} given (cos, sin)
template <bool INV, typename C, typename T>
__device__ __forceinline__ C rotc(C a, T c, T s) {
  return INV ? mk(a.x * c - a.y * s, a.y * c + a.x * s) : mk(a.x * c + a.y * s, a.y * c - a.x * s);
}

template <bool INV, typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// 4-point DFT of (v0, v1, v2, v3); Z2: v2 = v3 = 0 (inputs known to be zero)
template <bool INV, bool Z2, typename C>
__device__ __forceinline__ void dft4z(C& v0, C& v1, C& v2, C& v3) {
  if (Z2) {
    const C a = v0, c = v1;
    const C dm = rot4<INV>(c);
    v0 = cadd(a, c);
    v2 = csub(a, c);
    v1 = cadd(a, dm);
    v3 = csub(a, dm);
  } else {
    const C a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = csub(v1, v3);
    const C dm = rot4<INV>(d);
    v0 = cadd(a, c);
    v2 = csub(a, c);
    v1 = cadd(b, dm);
    v3 = csub(b, dm);
  }
}

// 8-point DFT, n = k + 2m: DFT4 over m for k = 0, 1; twiddle w8^{kq}; DFT2 over k.
// HALF: inputs 4..7 are zero.
template <bool INV, bool HALF, typename C, typename T>
__device__ __forceinline__ void dft8(C* v) {
  dft4z<INV, HALF>(v[0], v[2], v[4], v[6]);
  dft4z<INV, HALF>(v[1], v[3], v[5], v[7]);
  v[3] = rot8<INV, C, T>(v[3]);
  v[5] = rot4<INV>(v[5]);
  v[7] = rot8_3<INV, C, T>(v[7]);
  C o[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[q] = cadd(v[2 * q], v[2 * q + 1]);
    o[q + 4] = csub(v[2 * q], v[2 * q + 1]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = o[q];
}

// 16-point DFT, n = k + 4m, K = q + 4p: DFT4 over m, twiddle w16^{kq}, DFT4 over k.
// HALF: inputs 8..15 are zero.
template <bool INV, bool HALF, typename C, typename T>
__device__ __forceinline__ void dft16(C* v) {
#pragma unroll
  for (int k = 0; k < 4; ++k) dft4z<INV, HALF>(v[k], v[k + 4], v[k + 8], v[k + 12]);
  // v[k + 4q] = Y[k][q];  twiddle by w16^{kq}
  const T c = Consts<T>::c8, s = Consts<T>::s8;
  v[1 + 4] = rotc<INV, C, T>(v[1 + 4], c, s);          // kq = 1
  v[2 + 4] = rot8<INV, C, T>(v[2 + 4]);                // 2
  v[3 + 4] = rotc<INV, C, T>(v[3 + 4], s, c);          // 3
  v[1 + 8] = rot8<INV, C, T>(v[1 + 8]);                // 2
  v[2 + 8] = rot4<INV>(v[2 + 8]);                      // 4
  v[3 + 8] = rot8_3<INV, C, T>(v[3 + 8]);              // 6
  v[1 + 12] = rotc<INV, C, T>(v[1 + 12], s, c);        // 3
  v[2 + 12] = rot8_3<INV, C, T>(v[2 + 12]);            // 6
  v[3 + 12] = rotc<INV, C, T>(v[3 + 12], -c, -s);      // 9: w16^9 = -w16^1
#pragma unroll
  for (int q = 0; q < 4; ++q) dft4z<INV, false>(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  // v[p + 4q] = X[q + 4p]: transpose the 4x4 index grid
  C o[16];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) o[q + 4 * p] = v[p + 4 * q];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

template <int Q, bool INV, bool HALF, typename C, typename T>
__device__ __forceinline__ void dftq(C* v) {
  if constexpr (Q == 2) dft2<INV>(v[0], v[1]);
  if constexpr (Q == 4) dft4z<INV, HALF>(v[0], v[1], v[2], v[3]);
  if constexpr (Q == 8) dft8<INV, HALF, C, T>(v);
  if constexpr (Q == 16) dft16<INV, HALF, C, T>(v);
}

// --- stage plan ----------------------------------------------------------------
// float stages store a few twiddles and form the rest as products
template <typename T>
__host__ __device__ constexpr bool tw_products() { return sizeof(T) == 4; }
// planes of stored twiddles per k for a stage of radix q (see the header comment)
template <typename T>
__host__ __device__ constexpr int tw_planes(int q) {
  return tw_products<T>() ? (q == 16 ? 3 : (q >= 4 ? 2 : 1)) : q / 2;
}
// exponent r of the twiddle held at (plane, e) of a stage of radix q
template <typename T>
__host__ __device__ constexpr int tw_exponent(int plane, int e) {
  return tw_products<T>() ? (plane == 0 ? 1 + e : (plane == 1 ? 3 + e : 8 + 4 * e)) : 2 * plane + 1 + e;
}

template <int LOGL, int LOGR>
struct Plan {
  static constexpr int L = 1 << LOGL;
  static constexpr int R = 1 << LOGR;
  static constexpr int T = L / R;                     // threads per transform
  static constexpr int SR = LOGL / LOGR;              // radix-R stages
  static constexpr int LOGRL = LOGL % LOGR;           // small last stage (0: none)
  static constexpr int RL = 1 << LOGRL;
  static constexpr int NSTAGES = SR + (LOGRL ? 1 : 0);
  static constexpr int PADL = L + (L >> LOGR);        // padded shared-memory length
  __host__ __device__ static constexpr int radix(int s) { return s < SR ? R : RL; }
  // twiddle-table offset of stage s (stage 0 has none): stage i >= 1 stores
  // tw_planes(radix(i)) planes of Ns pairs
  template <typename T>
  __host__ __device__ static constexpr int tw_offset(int s) {
    int off = 0, ns = 1;
    for (int i = 0; i < s; ++i) {
      if (i > 0) off += 2 * tw_planes<T>(radix(i)) * ns;
      ns *= radix(i);
    }
    return off;
  }
};

template <int LOGR>
__device__ __forceinline__ int padi(int i) { return i + (i >> LOGR); }

// two consecutive complex values with one load where the type allows it
__device__ __forceinline__ void load_pair(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const double2* p, double2& a, double2& b) {
  a = p[0];
  b = p[1];
}

// Hides a pointer's value from the optimiser so that loads through it are not merged
// with earlier loads of the same addresses (which would keep the first transform's
// twiddles alive in registers until the second one).
template <typename P>
__device__ __forceinline__ const P* opaque(const P* p) {
  const P* q;
  asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p));
  return q;
}

template <bool INV, typename C>
__device__ __forceinline__ C twmul(C a, C w) { return INV ? cmulc(a, w) : cmul(a, w); }

// (cos, sin)(pi q / 16), q < 16: the constant factors e^{-+ i pi q / R} (R = 16 or 8,
// index q 16 / R) that relate the twiddles of the points t + (N/R) q to that of t.
static __constant__ double c_pi16d[16][2] = {
    {1.0, 0.0},
    {0.98078528040323044912618223613424, 0.19509032201612826784828486847702},
    {0.92387953251128675612818318939679, 0.38268343236508977172845998403040},
    {0.83146961230254523707878837761791, 0.55557023301960222474283081394853},
    {0.70710678118654752440084436210485, 0.70710678118654752440084436210485},
    {0.55557023301960222474283081394853, 0.83146961230254523707878837761791},
    {0.38268343236508977172845998403040, 0.92387953251128675612818318939679},
    {0.19509032201612826784828486847702, 0.98078528040323044912618223613424},
    {0.0, 1.0},
    {-0.19509032201612826784828486847702, 0.98078528040323044912618223613424},
    {-0.38268343236508977172845998403040, 0.92387953251128675612818318939679},
    {-0.55557023301960222474283081394853, 0.83146961230254523707878837761791},
    {-0.70710678118654752440084436210485, 0.70710678118654752440084436210485},
    {-0.83146961230254523707878837761791, 0.55557023301960222474283081394853},
    {-0.92387953251128675612818318939679, 0.38268343236508977172845998403040},
    {-0.98078528040323044912618223613424, 0.19509032201612826784828486847702}};
static __constant__ float c_pi16f[16][2] = {
    {1.0f, 0.0f},
    {0.98078528040323044912618223613424f, 0.19509032201612826784828486847702f},
    {0.92387953251128675612818318939679f, 0.38268343236508977172845998403040f},
    {0.83146961230254523707878837761791f, 0.55557023301960222474283081394853f},
    {0.70710678118654752440084436210485f, 0.70710678118654752440084436210485f},
    {0.55557023301960222474283081394853f, 0.83146961230254523707878837761791f},
    {0.38268343236508977172845998403040f, 0.92387953251128675612818318939679f},
    {0.19509032201612826784828486847702f, 0.98078528040323044912618223613424f},
    {0.0f, 1.0f},
    {-0.19509032201612826784828486847702f, 0.98078528040323044912618223613424f},
    {-0.38268343236508977172845998403040f, 0.92387953251128675612818318939679f},
    {-0.55557023301960222474283081394853f, 0.83146961230254523707878837761791f},
    {-0.70710678118654752440084436210485f, 0.70710678118654752440084436210485f},
    {-0.83146961230254523707878837761791f, 0.55557023301960222474283081394853f},
    {-0.92387953251128675612818318939679f, 0.38268343236508977172845998403040f},
    {-0.98078528040323044912618223613424f, 0.19509032201612826784828486847702f}};
template <typename T> __device__ __forceinline__ cplx<T> pi16(int q);
template <> __device__ __forceinline__ float2 pi16<float>(int q) { return make_float2(c_pi16f[q][0], c_pi16f[q][1]); }
template <> __device__ __forceinline__ double2 pi16<double>(int q) { return make_double2(c_pi16d[q][0], c_pi16d[q][1]); }

// Multiplies x(r), r = 1..Q-1, by w_r (conjugated for INV) for one k of a stage whose
// table planes start at tws (Ns pairs per plane).
template <int Q, bool INV, typename C, typename X>
__device__ __forceinline__ void apply_twiddles(const C* tws, int ns, int k, X&& x) {
  if constexpr (!tw_products<decltype(C::x)>()) {   // every twiddle stored
#pragma unroll
    for (int pl = 0; pl < Q / 2; ++pl) {
      C w1, w2;
      load_pair(tws + 2 * (pl * ns + k), w1, w2);
      x(2 * pl + 1) = twmul<INV>(x(2 * pl + 1), w1);
      if (2 * pl + 2 < Q) x(2 * pl + 2) = twmul<INV>(x(2 * pl + 2), w2);
    }
    return;
  }
  C w1, w2;
  load_pair(tws + 2 * k, w1, w2);
  x(1) = twmul<INV>(x(1), w1);
  if constexpr (Q >= 4) {
    C w3, w4;
    load_pair(tws + 2 * (ns + k), w3, w4);
    x(2) = twmul<INV>(x(2), w2);
    x(3) = twmul<INV>(x(3), w3);
    if constexpr (Q >= 8) {
      x(4) = twmul<INV>(x(4), w4);
      x(5) = twmul<INV>(x(5), cmul(w1, w4));
      x(6) = twmul<INV>(x(6), cmul(w2, w4));
      x(7) = twmul<INV>(x(7), cmul(w3, w4));
    }
    if constexpr (Q == 16) {
      C w8, w12;
      load_pair(tws + 2 * (2 * ns + k), w8, w12);
      x(8) = twmul<INV>(x(8), w8);
      x(9) = twmul<INV>(x(9), cmul(w1, w8));
      x(10) = twmul<INV>(x(10), cmul(w2, w8));
      x(11) = twmul<INV>(x(11), cmul(w3, w8));
      x(12) = twmul<INV>(x(12), w12);
      x(13) = twmul<INV>(x(13), cmul(w1, w12));
      x(14) = twmul<INV>(x(14), cmul(w2, w12));
      x(15) = twmul<INV>(x(15), cmul(w3, w12));
    }
  }
}

// Synchronisation of the threads of one transform around its exchanges.  When a
// block holds several transforms, each exchanges through its own buffer, so it
// waits only for its own threads: one warp (__syncwarp), or a named barrier per
// transform (ids 1..15, id 0 being __syncthreads); otherwise the whole block.
template <int TT, int PER_BLOCK>
struct GroupSync {
  static constexpr int kind = (PER_BLOCK == 1) ? 0 : (TT == 32 ? 1 : ((TT > 32 && PER_BLOCK <= 15) ? 2 : 0));
  __device__ __forceinline__ static void sync(int group) {
    if constexpr (kind == 1) {
      __syncwarp();
    } else if constexpr (kind == 2) {
      asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(TT) : "memory");
    } else {
      __syncthreads();
    }
  }
};

// Full transform on the thread's registers v[q] = x[t + T q] -> X[t + T q].
// sh: this transform's padded shared buffer (PADL complex).  HALF: x = 0 for
// index >= L/2 (v[R/2..R-1] zero on entry).  PER_BLOCK transforms share the block;
// group is this one's index (see GroupSync).  All threads of the group (of the block
// when the block-wide barrier is used) must call it.
template <int LOGL, int LOGR, bool INV, bool HALF, typename T, int PER_BLOCK = 1>
__device__ __forceinline__ void reg_fft(cplx<T>* v, cplx<T>* sh, const cplx<T>* __restrict__ tw, int t,
                                        int group = 0) {
  using C = cplx<T>;
  using P = Plan<LOGL, LOGR>;
  constexpr int R = P::R, TT = P::T, RL = P::RL;
  int ns = 1;
#pragma unroll
  for (int s = 0; s < P::NSTAGES; ++s) {
    const bool small = (s == P::SR);   // the radix-RL stage
    if (s > 0) {
      const C* tws = opaque(tw + P::template tw_offset<T>(s));
      if (!small) {
        apply_twiddles<R, INV>(tws, ns, t & (ns - 1), [&](int r) -> C& { return v[r]; });
      } else {
#pragma unroll
        for (int b = 0; b < R / RL; ++b) {
          const int k = (t + TT * b) & (ns - 1);
          apply_twiddles<RL, INV>(tws, ns, k, [&](int r) -> C& { return v[b + r * (R / RL)]; });
        }
      }
    }
    if (!small) {
      if (s == 0 && HALF) dftq<R, INV, true, C, T>(v);
      else dftq<R, INV, false, C, T>(v);
    } else {
      // R/RL butterflies of radix RL: butterfly b holds v[b + r (R/RL)], r < RL
#pragma unroll
      for (int b = 0; b < R / RL; ++b) {
        C w[RL > 1 ? RL : 2];
#pragma unroll
        for (int r = 0; r < RL; ++r) w[r] = v[b + r * (R / RL)];
        dftq<RL, INV, false, C, T>(w);
#pragma unroll
        for (int r = 0; r < RL; ++r) v[b + r * (R / RL)] = w[r];
      }
    }
    if (s + 1 < P::NSTAGES) {
      // exchange: write at the self-sorting output positions, read x[t + T q]
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

}  // namespace bem
