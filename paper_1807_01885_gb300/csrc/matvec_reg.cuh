// Register-FFT implementation of the three passes of u = K p (Eq. 11), N >= 16.
// Included by matvec_f32.cu and matvec_f64.cu (one precision per translation unit).
//
// Pass 1 (rows): row r packs its N reals as z[m] = p[2m] + i p[2m+1] (m < N/2),
//   takes the length-N complex FFT of z padded with N/2 zeros (first stage pruned),
//   and recombines X[j] = (Z[j] + Z*[N-j])/2 - (i/2) e^{-2 pi i j/2N} (Z[j] - Z*[N-j]),
//   j in [0, N], the half spectrum of the zero-padded length-2N real row, stored
//   column-major (spec[j N + r]) through shared memory so that each warp store
//   writes whole 32-byte sectors of neighbouring rows.
// Pass 2 (columns): per frequency column, the length-2N FFT of the N nonzero rows
//   (first stage pruned), times K^ (table folded on |k|, scaled by 1/(2N)^2), the
//   inverse length-2N FFT, of which only the first N rows are kept.
// Pass 3 (rows): Zi[j] = (Y[j] + Y*[N-j]) + i e^{+2 pi i j/2N} (Y[j] - Y*[N-j]),
//   the inverse length-N FFT (only the first N/2 outputs), u[2m] + i u[2m+1] = z[m].
#pragma once

#include "bem_internal.cuh"
#include "fft_pair.cuh"
#include "fft_reg.cuh"

namespace bem {

// Launch bounds per (precision, radix, pass): KIND 0 = rows, 1 = columns.
template <typename T, int LOGR, int KIND> struct RegCfg { static constexpr int MAXT = 512, MINB = 2; };
template <> struct RegCfg<float, 4, 1> { static constexpr int MAXT = 256, MINB = 3; };
template <> struct RegCfg<float, 3, 0> { static constexpr int MAXT = 512, MINB = 3; };
template <int KIND> struct RegCfg<double, 3, KIND> { static constexpr int MAXT = 512, MINB = 1; };
template <int KIND> struct RegCfg<double, 4, KIND> { static constexpr int MAXT = 256, MINB = 1; };


// e^{-i pi j / N} for j = t + (N/R) q: in float tw[t] times the constant e^{-i pi q / R}
// (one load per thread instead of R); in double (FP64-pipe bound) the table entry.
template <typename T, int R>
__device__ __forceinline__ cplx<T> recomb_tw(const cplx<T>* __restrict__ tw, cplx<T> wt, int j, int q) {
  if constexpr (sizeof(T) == 4) return cmulc(wt, pi16<T>(q * 16 / R));
  else return tw[j];
}

// asynchronous global -> shared copy of one complex value (8 or 16 bytes, L1-cached)
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* smem, const C* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(a), "l"(gmem), "n"(sizeof(C)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// complex slots of one row's shared buffer in the row passes: the padded exchange
// buffer plus 8, rounded up to an even count so that every row's buffer starts on a
// 16-byte boundary (the float inverse pass copies 16-byte records into it)
template <int LOGN, int LOGR>
__host__ __device__ constexpr int row_sh() {
  return Plan<LOGN, LOGR>::PADL + 8 + (Plan<LOGN, LOGR>::PADL & 1);
}

// rows per block of the row passes and columns per block of the column pass
template <typename T, int LOGN, int LOGR>
__host__ __device__ constexpr int rows_per_block() {
  constexpr int r = RegCfg<T, LOGR, 0>::MAXT / Plan<LOGN, LOGR>::T;
  return r < 1 ? 1 : (r > (1 << LOGN) ? (1 << LOGN) : r);
}
template <typename T, int LOGM, int LOGR>
__host__ __device__ constexpr int cols_per_block() {
  constexpr int c = RegCfg<T, LOGR, 1>::MAXT / Plan<LOGM, LOGR>::T;
  return c < 1 ? 1 : c;
}

template <typename T, int LOGN, int LOGR>
__global__ void __launch_bounds__(RegCfg<T, LOGR, 0>::MAXT, RegCfg<T, LOGR, 0>::MINB)
k_row_fwd_r(const T* __restrict__ p, cplx<T>* __restrict__ spec, const cplx<T>* __restrict__ twr,
            const cplx<T>* __restrict__ tw, const int* __restrict__ skip) {
  using C = cplx<T>;
  using P = Plan<LOGN, LOGR>;
  constexpr int N = 1 << LOGN, TT = P::T, SH = row_sh<LOGN, LOGR>(), R = P::R;
  constexpr int RPB = rows_per_block<T, LOGN, LOGR>();
  pdl_enter();
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* const sh0 = reinterpret_cast<C*>(smem_raw);
  const int rl = threadIdx.x / TT, t = threadIdx.x - rl * TT;
  const int r0 = blockIdx.x * RPB;
  C* sh = sh0 + rl * SH;
  C v[R];
  const C* prow = reinterpret_cast<const C*>(p + (size_t)(r0 + rl) * N);
#pragma unroll
  for (int q = 0; q < R / 2; ++q) v[q] = prow[t + TT * q];
#pragma unroll
  for (int q = R / 2; q < R; ++q) v[q] = mk((T)0, (T)0);
  reg_fft<LOGN, LOGR, false, true, T, RPB>(v, sh, twr, t, rl);
#pragma unroll
  for (int q = 0; q < R; ++q) sh[padi<LOGR>(t + TT * q)] = v[q];
  __syncthreads();
  const int j0 = threadIdx.x / RPB, rr = threadIdx.x - j0 * RPB;
  const C* shr = sh0 + rr * SH;
  if constexpr (sizeof(T) == 4) {
    // Float: the spectrum is stored in column pairs (spec4[jp N + r] holds the re and
    // im of frequencies 2jp and 2jp + 1 of row r as (re_2jp, re_2jp+1, im_2jp,
    // im_2jp+1)), the layout the paired column pass reads.  Thread (j0, rr) forms X[j]
    // and X[j + 1] of row r0 + rr for j = 2 (j0 + TT k / 2), k = 0, 2, .., R - 2, so
    // that the RPB rows of one frequency pair go out as one 16-byte store each.
    float4* out4 = reinterpret_cast<float4*>(spec) + r0 + rr;
    const C wa = tw[2 * j0], wb = tw[2 * j0 + 1];
#pragma unroll
    for (int k = 0; k < R; k += 2) {
      const int j = 2 * j0 + TT * k;   // TT k = N k / R: the frequencies 2 j0 + (N/R) k and + 1
      C X2[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int jj = j + e;
        const C za = shr[padi<LOGR>(jj)];
        const C zb = cconj(shr[padi<LOGR>((N - jj) & (N - 1))]);
        const C E = cscale(cadd(za, zb), (T)0.5);
        const C O = cscale(cmul_mi(csub(za, zb)), (T)0.5);
        X2[e] = cadd(E, cmul(O, recomb_tw<T, R>(tw, e ? wb : wa, jj, k)));
      }
      out4[(size_t)(j / 2) * N] = make_float4(X2[0].x, X2[1].x, X2[0].y, X2[1].y);
    }
    if (j0 == 0) {
      // pair N/2: j = N (Nyquist, X[N] = Re Z[0] - Im Z[0]) and an empty column N + 1
      const C z0 = shr[0];
      out4[(size_t)(N / 2) * N] = make_float4(z0.x - z0.y, 0.f, 0.f, 0.f);
    }
  } else {
    // Recombination and column-major store: thread (j0, rr) = (tid / RPB, tid mod RPB)
    // forms X[j] of row r0 + rr for j = j0 + TT k, k = 0..R (k = R: only j = N), so
    // that the RPB rows of one frequency, contiguous in spec, go out in one sector.
    C* out = spec + r0 + rr;
    const C wt = mk((T)0, (T)0);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int j = j0 + TT * k;
      const C za = shr[padi<LOGR>(j)];
      const C zb = cconj(shr[padi<LOGR>((N - j) & (N - 1))]);
      const C E = cscale(cadd(za, zb), (T)0.5);
      const C O = cscale(cmul_mi(csub(za, zb)), (T)0.5);
      out[(size_t)j * N] = cadd(E, cmul(O, recomb_tw<T, R>(tw, wt, j, k)));
    }
    if (j0 == 0) {
      // j = N (Nyquist): X[N] = Re Z[0] - Im Z[0]
      const C z0 = shr[0];
      out[(size_t)N * N] = mk(z0.x - z0.y, (T)0);
    }
  }
}

template <typename T, int LOGN, int LOGR>
__global__ void __launch_bounds__(RegCfg<T, LOGR, 0>::MAXT, RegCfg<T, LOGR, 0>::MINB)
k_row_inv_r(const cplx<T>* __restrict__ spec, T* __restrict__ u, const cplx<T>* __restrict__ twr,
            const cplx<T>* __restrict__ tw, const int* __restrict__ skip) {
  using C = cplx<T>;
  using P = Plan<LOGN, LOGR>;
  constexpr int N = 1 << LOGN, TT = P::T, SH = row_sh<LOGN, LOGR>(), R = P::R;
  constexpr int RPB = rows_per_block<T, LOGN, LOGR>(), NT = RPB * TT;
  pdl_enter();
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* const sh0 = reinterpret_cast<C*>(smem_raw);
  const int rl = threadIdx.x / TT, t = threadIdx.x - rl * TT;
  const int r0 = blockIdx.x * RPB;
  C* sh = sh0 + rl * SH;
  C v[R];
  if constexpr (sizeof(T) == 4) {
    // float: the RPB rows' frequency pairs (spec4[jp N + r], jp in [0, N/2], the
    // layout of the paired column pass) copied asynchronously as 16-byte records into
    // each row's buffer, record jp at float offset 4 jp: Y[j] = (buf[4 (j/2) + j%2],
    // buf[4 (j/2) + 2 + j%2])
    const float4* in4 = reinterpret_cast<const float4*>(spec) + r0;
    constexpr int NP = N / 2 + 1;
#pragma unroll
    for (int k = 0; k < (RPB * NP + NT - 1) / NT; ++k) {
      const int e = threadIdx.x + NT * k;
      if (e < RPB * NP) {
        const int jp = e / RPB, rr = e - jp * RPB;
        cp_async_elem(reinterpret_cast<float4*>(sh0 + rr * SH) + jp, in4 + (size_t)jp * N + rr);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    const float* buf = reinterpret_cast<const float*>(sh);
    const C wt = tw[t];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int j = t + TT * q, jr = N - j;
      const C y1 = mk(buf[4 * (j >> 1) + (j & 1)], buf[4 * (j >> 1) + 2 + (j & 1)]);
      const C y2 = mk(buf[4 * (jr >> 1) + (jr & 1)], -buf[4 * (jr >> 1) + 2 + (jr & 1)]);
      const C e = cadd(y1, y2);
      const C o = cmul_pi(cmulc(csub(y1, y2), recomb_tw<T, R>(tw, wt, j, q)));
      v[q] = cadd(e, o);
    }
  } else {
    // column-major load of the RPB rows' half spectra Y[j], j in [0, N], copied
    // asynchronously from global to shared memory (no register staging)
    const C* in = spec + r0;
#pragma unroll
    for (int k = 0; k < (RPB * (N + 1) + NT - 1) / NT; ++k) {
      const int e = threadIdx.x + NT * k;
      if (e < RPB * (N + 1)) {
        const int j = e / RPB, rr = e - j * RPB;
        cp_async_elem(sh0 + rr * SH + j, in + (size_t)j * N + rr);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    const C wt = mk((T)0, (T)0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int j = t + TT * q;
      const C y1 = sh[j];
      const C y2 = cconj(sh[N - j]);
      const C e = cadd(y1, y2);
      const C o = cmul_pi(cmulc(csub(y1, y2), recomb_tw<T, R>(tw, wt, j, q)));
      v[q] = cadd(e, o);
    }
  }
  __syncthreads();
  reg_fft<LOGN, LOGR, true, false, T, RPB>(v, sh, twr, t, rl);
  C* urow = reinterpret_cast<C*>(u + (size_t)(r0 + rl) * N);
#pragma unroll
  for (int q = 0; q < R / 2; ++q) urow[t + TT * q] = v[q];
}

template <typename T, int LOGM, int LOGR>
__global__ void __launch_bounds__(RegCfg<T, LOGR, 1>::MAXT, RegCfg<T, LOGR, 1>::MINB)
k_col_r(cplx<T>* __restrict__ spec, const T* __restrict__ table, const cplx<T>* __restrict__ twc, int nslots,
        const int* __restrict__ skip) {
  using C = cplx<T>;
  using P = Plan<LOGM, LOGR>;
  constexpr int M = 1 << LOGM, N = M / 2, TT = P::T, SH = P::PADL + 8, R = P::R;
  constexpr int CPB = cols_per_block<T, LOGM, LOGR>();
  pdl_enter();
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x / TT, t = threadIdx.x - c * TT;
  const int slot = blockIdx.x * CPB + c;   // frequency column j
  const bool active = slot < nslots;
  C* sh = reinterpret_cast<C*>(smem_raw) + c * SH;
  C* col = spec + (size_t)slot * N;
  C v[R];
#pragma unroll
  for (int q = 0; q < R / 2; ++q) v[q] = active ? col[t + TT * q] : mk((T)0, (T)0);
#pragma unroll
  for (int q = R / 2; q < R; ++q) v[q] = mk((T)0, (T)0);
  reg_fft<LOGM, LOGR, false, true, T, CPB>(v, sh, twc, t, c);
  const T* kt = table + (size_t)slot * (N + 4);   // column j = slot of the square table (row stride N + 4)
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = t + TT * q;
    const int f = (q < R / 2) ? i : M - i;
    const T kv = active ? kt[f] : (T)0;
    v[q] = cscale(v[q], kv);
  }
  reg_fft<LOGM, LOGR, true, false, T, CPB>(v, sh, twc, t, c);
  if (active) {
#pragma unroll
    for (int q = 0; q < R / 2; ++q) col[t + TT * q] = v[q];
  }
}

// Float column pass on column pairs: block c-slot handles the frequency columns 2 pr
// and 2 pr + 1 (pr < npairs = N/2 + 1; the second column of the last pair is the
// empty column N + 1, whose compliance is 0) as one packed transform (fft_pair.cuh):
// the length-2N FFT of the N nonzero rows (first stage pruned), times the pair of
// compliances (tab2[pr (N + 1) + f] = (K(f, 2 pr), K(f, 2 pr + 1)) / M^2, f the folded
// row wave number), the inverse FFT, the first N rows kept.
template <int LOGR> struct ColPairCfg { static constexpr int MAXT = 256, MINB = 2; };
template <> struct ColPairCfg<3> { static constexpr int MAXT = 512, MINB = 1; };

template <int LOGM, int LOGR>
__host__ __device__ constexpr int pairs_per_block() {
  constexpr int c = ColPairCfg<LOGR>::MAXT / Plan<LOGM, LOGR>::T;
  return c < 1 ? 1 : c;
}

template <int LOGM, int LOGR>
__global__ void __launch_bounds__(ColPairCfg<LOGR>::MAXT, ColPairCfg<LOGR>::MINB)
k_col_p(float4* __restrict__ spec4, const float2* __restrict__ tab2, const float4* __restrict__ twp, int npairs,
        const int* __restrict__ skip) {
  using P = Plan<LOGM, LOGR>;
  using pr::CP;
  constexpr int M = 1 << LOGM, N = M / 2, TT = P::T, SH = P::PADL + 8, R = P::R;
  constexpr int CPB = pairs_per_block<LOGM, LOGR>();
  pdl_enter();
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = threadIdx.x / TT, t = threadIdx.x - c * TT;
  const int pair = blockIdx.x * CPB + c;
  const bool active = pair < npairs;
  CP* sh = reinterpret_cast<CP*>(smem_raw) + c * SH;
  // the block's compliance rows, copied to shared memory while the forward FFT runs
  float2* ksh = reinterpret_cast<float2*>(reinterpret_cast<CP*>(smem_raw) + CPB * SH);
  {
    const int pair0 = blockIdx.x * CPB;
    const int nact = min(CPB, npairs - pair0);
    const float2* src = tab2 + (size_t)pair0 * (N + 1);
    for (int e = threadIdx.x; e < nact * (N + 1); e += CPB * TT) cp_async_elem(ksh + e, src + e);
  }
  float4* col = spec4 + (size_t)pair * N;
  CP v[R];
#pragma unroll
  for (int q = 0; q < R / 2; ++q) v[q] = active ? pr::cp_load(col + t + TT * q) : pr::cp_zero();
#pragma unroll
  for (int q = R / 2; q < R; ++q) v[q] = pr::cp_zero();
  pr::pair_fft<LOGM, LOGR, false, true, CPB>(v, sh, twp, t, c);
  cp_async_wait_all();
  __syncthreads();
  const float2* kt = ksh + c * (N + 1);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = t + TT * q;
    const int f = (q < R / 2) ? i : M - i;
    const float2 kv = active ? kt[f] : make_float2(0.f, 0.f);
    v[q] = pr::cscale2(v[q], pr::pk2(kv.x, kv.y));
  }
  pr::pair_fft<LOGM, LOGR, true, false, CPB>(v, sh, twp, t, c);
  if (active) {
#pragma unroll
    for (int q = 0; q < R / 2; ++q) pr::cp_store(col + t + TT * q, v[q]);
  }
}

// stage twiddles of the paired FFT (fft_pair.cuh) of length 2^logl, radix 2^logr:
// stage s >= 1 (radix Q, span Ns) holds, in plane p and record k, the broadcast
// (wr, wr, wi, wi) of w = e^{-2 pi i k e / (Ns Q)}, e = twp_exponent(Q, p)
static __global__ void k_stage_twiddles_pair(float4* __restrict__ out, int logl, int logr) {
  const int sr = logl / logr, logrl = logl % logr;
  const int nst = sr + (logrl ? 1 : 0);
  int off = 0, ns = 1;
  for (int s = 0; s < nst; ++s) {
    const int Q = (s < sr) ? (1 << logr) : (1 << logrl);
    if (s > 0) {
      const int cnt = pr::twp_planes(Q) * ns;
      for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < cnt; idx += gridDim.x * blockDim.x) {
        const int k = idx % ns, plane = idx / ns;
        const int e = pr::twp_exponent(Q, plane);
        double sn = 0.0, cs = 1.0;
        sincospi(2.0 * (double)k * (double)e / (double)(ns * Q), &sn, &cs);
        out[off + idx] = make_float4((float)cs, (float)cs, (float)(-sn), (float)(-sn));
      }
      off += cnt;
    }
    ns *= Q;
  }
}

// stage twiddle tables of the register FFT of length 2^logl with radix 2^logr:
// stage s >= 1 (radix Q, span Ns) holds w(r, k) = e^{-2 pi i k r / (Ns Q)} in
// tw_planes<T>(Q) planes [plane][k][2], r = tw_exponent<T>(plane, e)
template <typename T>
__global__ void k_stage_twiddles(cplx<T>* __restrict__ out, int logl, int logr) {
  const int sr = logl / logr, logrl = logl % logr;
  const int nst = sr + (logrl ? 1 : 0);
  int off = 0, ns = 1;
  for (int s = 0; s < nst; ++s) {
    const int R = (s < sr) ? (1 << logr) : (1 << logrl);
    if (s > 0) {
      const int cnt = 2 * tw_planes<T>(R) * ns;
      for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < cnt; idx += gridDim.x * blockDim.x) {
        const int e = idx & 1, k = (idx >> 1) % ns, plane = (idx >> 1) / ns;
        const int r = tw_exponent<T>(plane, e);
        double sn = 0.0, cs = 1.0;
        sincospi(2.0 * (double)k * (double)r / (double)(ns * R), &sn, &cs);
        out[off + idx] = mk((T)cs, (T)(-sn));
      }
      off += cnt;
    }
    ns *= R;
  }
}

// ---------------------------------------------------------------------------
template <typename T, int LOGN, int LOGR>
struct RowLaunch {
  using C = cplx<T>;
  // one-time per-device kernel attributes (also called before a graph capture)
  static void prepare() {
    static std::atomic<unsigned long long> attr{0};
    if (first_on_device(attr)) {
      cudaFuncSetAttribute(k_row_fwd_r<T, LOGN, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(k_row_inv_r<T, LOGN, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
  }
  static void pass(const bem_kernel_s* k, int which, const T* p, T* u, cudaStream_t s, const int* skip) {
    prepare();
    constexpr int N = 1 << LOGN;
    using PR = Plan<LOGN, LOGR>;

    constexpr int rpb = rows_per_block<T, LOGN, LOGR>();
    const size_t smem = (size_t)rpb * row_sh<LOGN, LOGR>() * sizeof(C);
    C* spec = (C*)k->ws.spec;
    if (which == 0)
      launch_pdl(k_row_fwd_r<T, LOGN, LOGR>, N / rpb, rpb * PR::T, smem, s, p, spec, (const C*)k->ws.twr,
                 (const C*)k->ws.tw, skip);
    else
      launch_pdl(k_row_inv_r<T, LOGN, LOGR>, N / rpb, rpb * PR::T, smem, s, (const C*)spec, u,
                 (const C*)k->ws.twr, (const C*)k->ws.tw, skip);
  }
};

template <typename T, int LOGN, int LOGR>
struct ColLaunch {
  using C = cplx<T>;
  static void prepare() {
    static std::atomic<unsigned long long> attr{0};
    if (first_on_device(attr)) {
      if constexpr (sizeof(T) == 4)
        cudaFuncSetAttribute(k_col_p<LOGN + 1, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      else
        cudaFuncSetAttribute(k_col_r<T, LOGN + 1, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
  }
  static void pass(const bem_kernel_s* k, const int* skip, cudaStream_t s) {
    prepare();
    constexpr int N = 1 << LOGN;
    using PC = Plan<LOGN + 1, LOGR>;
    if constexpr (sizeof(T) == 4) {
      constexpr int ppb = pairs_per_block<LOGN + 1, LOGR>();
      const int npairs = N / 2 + 1;
      const int grid = (npairs + ppb - 1) / ppb;
      const size_t smem = (size_t)ppb * ((PC::PADL + 8) * sizeof(pr::CP) + (N + 1) * sizeof(float2));
      launch_pdl(k_col_p<LOGN + 1, LOGR>, grid, ppb * PC::T, smem, s, (float4*)k->ws.spec,
                 (const float2*)k->ws.table, (const float4*)k->ws.twpc, npairs, skip);
    } else {
      constexpr int cpb = cols_per_block<T, LOGN + 1, LOGR>();
      const int nslots = N + 1;
      const int grid = (nslots + cpb - 1) / cpb;
      const size_t smem = (size_t)cpb * (PC::PADL + 8) * sizeof(C);
      launch_pdl(k_col_r<T, LOGN + 1, LOGR>, grid, cpb * PC::T, smem, s, (C*)k->ws.spec, (const T*)k->ws.table,
                 (const C*)k->ws.twc, nslots, skip);
    }
  }
};

template <typename T> struct Radix;
template <> struct Radix<float> { static constexpr int ROW = 4, ROW_ALT = 3, COL = 4, COL_ALT = 3; };
template <> struct Radix<double> { static constexpr int ROW = 3, ROW_ALT = 3, COL = 3, COL_ALT = 3; };

template <typename T, template <typename, int, int> class L, int LOGR, typename... A>
void by_logn(int logn, A... a) {
  switch (logn) {
    case 4: L<T, 4, LOGR>::pass(a...); break;
    case 5: L<T, 5, LOGR>::pass(a...); break;
    case 6: L<T, 6, LOGR>::pass(a...); break;
    case 7: L<T, 7, LOGR>::pass(a...); break;
    case 8: L<T, 8, LOGR>::pass(a...); break;
    case 9: L<T, 9, LOGR>::pass(a...); break;
    case 10: L<T, 10, LOGR>::pass(a...); break;
    case 11: L<T, 11, LOGR>::pass(a...); break;
    default: break;
  }
}

template <typename T, template <typename, int, int> class L, int LOGR>
void by_logn_prepare(int logn) {
  switch (logn) {
    case 4: L<T, 4, LOGR>::prepare(); break;
    case 5: L<T, 5, LOGR>::prepare(); break;
    case 6: L<T, 6, LOGR>::prepare(); break;
    case 7: L<T, 7, LOGR>::prepare(); break;
    case 8: L<T, 8, LOGR>::prepare(); break;
    case 9: L<T, 9, LOGR>::prepare(); break;
    case 10: L<T, 10, LOGR>::prepare(); break;
    case 11: L<T, 11, LOGR>::prepare(); break;
    default: break;
  }
}

template <typename T>
int row_logr(const bem_kernel_s* k) { return k->row_radix_alt ? Radix<T>::ROW_ALT : Radix<T>::ROW; }
template <typename T>
int col_logr(const bem_kernel_s* k) { return k->col_radix_alt ? Radix<T>::COL_ALT : Radix<T>::COL; }

template <typename T>
void reg_pass(const bem_kernel_s* k, int which, const T* p, T* u, cudaStream_t s, const int* skip) {
  if (which == 1) {
    if (col_logr<T>(k) == 4) by_logn<T, ColLaunch, 4>(k->logN, k, skip, s);
    else by_logn<T, ColLaunch, 3>(k->logN, k, skip, s);
  } else {
    if (row_logr<T>(k) == 4) by_logn<T, RowLaunch, 4>(k->logN, k, which, p, u, s, skip);
    else by_logn<T, RowLaunch, 3>(k->logN, k, which, p, u, s, skip);
  }
}

// kernel attributes of the passes a handle launches, set before a graph capture
template <typename T>
void reg_prepare(const bem_kernel_s* k) {
  if (col_logr<T>(k) == 4) by_logn_prepare<T, ColLaunch, 4>(k->logN);
  else by_logn_prepare<T, ColLaunch, 3>(k->logN);
  if (row_logr<T>(k) == 4) by_logn_prepare<T, RowLaunch, 4>(k->logN);
  else by_logn_prepare<T, RowLaunch, 3>(k->logN);
}

template <typename T>
void reg_twiddles(const bem_kernel_s* k, cudaStream_t s) {
  k_stage_twiddles<T><<<64, 256, 0, s>>>((cplx<T>*)k->ws.twr, k->logN, row_logr<T>(k));
  if constexpr (sizeof(T) == 4)
    k_stage_twiddles_pair<<<64, 256, 0, s>>>((float4*)k->ws.twpc, k->logN + 1, col_logr<T>(k));
  else
    k_stage_twiddles<T><<<64, 256, 0, s>>>((cplx<T>*)k->ws.twc, k->logN + 1, col_logr<T>(k));
}

}  // namespace bem
