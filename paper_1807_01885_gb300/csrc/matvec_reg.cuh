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
  constexpr int N = 1 << LOGN, TT = P::T, SH = P::PADL + 8, R = P::R;
  constexpr int RPB = rows_per_block<T, LOGN, LOGR>();
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
  // Recombination and column-major store: thread (j0, rr) = (tid / RPB, tid mod RPB)
  // forms X[j] of row r0 + rr for j = j0 + TT k, k = 0..R (k = R: only j = N), so
  // that the RPB rows of one frequency, contiguous in spec, go out in one sector.
  const int j0 = threadIdx.x / RPB, rr = threadIdx.x - j0 * RPB;
  const C* shr = sh0 + rr * SH;
  C* out = spec + r0 + rr;
  const C wt = sizeof(T) == 4 ? tw[j0] : mk((T)0, (T)0);
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

template <typename T, int LOGN, int LOGR>
__global__ void __launch_bounds__(RegCfg<T, LOGR, 0>::MAXT, RegCfg<T, LOGR, 0>::MINB)
k_row_inv_r(const cplx<T>* __restrict__ spec, T* __restrict__ u, const cplx<T>* __restrict__ twr,
            const cplx<T>* __restrict__ tw, const int* __restrict__ skip) {
  using C = cplx<T>;
  using P = Plan<LOGN, LOGR>;
  constexpr int N = 1 << LOGN, TT = P::T, SH = P::PADL + 8, R = P::R;
  constexpr int RPB = rows_per_block<T, LOGN, LOGR>(), NT = RPB * TT;
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* const sh0 = reinterpret_cast<C*>(smem_raw);
  const int rl = threadIdx.x / TT, t = threadIdx.x - rl * TT;
  const int r0 = blockIdx.x * RPB;
  C* sh = sh0 + rl * SH;
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
  C v[R];
  const C wt = sizeof(T) == 4 ? tw[t] : mk((T)0, (T)0);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = t + TT * q;
    const C y1 = sh[j];
    const C y2 = cconj(sh[N - j]);
    const C e = cadd(y1, y2);
    const C o = cmul_pi(cmulc(csub(y1, y2), recomb_tw<T, R>(tw, wt, j, q)));
    v[q] = cadd(e, o);
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
    const size_t smem = (size_t)rpb * (PR::PADL + 8) * sizeof(C);
    C* spec = (C*)k->ws.spec;
    if (which == 0)
      k_row_fwd_r<T, LOGN, LOGR><<<N / rpb, rpb * PR::T, smem, s>>>(p, spec, (const C*)k->ws.twr,
                                                                    (const C*)k->ws.tw, skip);
    else
      k_row_inv_r<T, LOGN, LOGR><<<N / rpb, rpb * PR::T, smem, s>>>(spec, u, (const C*)k->ws.twr,
                                                                    (const C*)k->ws.tw, skip);
  }
};

template <typename T, int LOGN, int LOGR>
struct ColLaunch {
  using C = cplx<T>;
  static void prepare() {
    static std::atomic<unsigned long long> attr{0};
    if (first_on_device(attr))
      cudaFuncSetAttribute(k_col_r<T, LOGN + 1, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  static void pass(const bem_kernel_s* k, const int* skip, cudaStream_t s) {
    prepare();
    constexpr int N = 1 << LOGN;
    using PC = Plan<LOGN + 1, LOGR>;
    constexpr int cpb = cols_per_block<T, LOGN + 1, LOGR>();
    const int nslots = N + 1;
    const int grid = (nslots + cpb - 1) / cpb;
    const size_t smem = (size_t)cpb * (PC::PADL + 8) * sizeof(C);
    k_col_r<T, LOGN + 1, LOGR><<<grid, cpb * PC::T, smem, s>>>((C*)k->ws.spec, (const T*)k->ws.table,
                                                             (const C*)k->ws.twc, nslots, skip);
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
  k_stage_twiddles<T><<<64, 256, 0, s>>>((cplx<T>*)k->ws.twc, k->logN + 1, col_logr<T>(k));
}

}  // namespace bem
