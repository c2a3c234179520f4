// Register-FFT implementation of the three passes of u = K p (Eq. 11), N >= 16.
// Included by matvec_f32.cu and matvec_f64.cu (one precision per translation unit).
//
// Pass 1 (rows): row r packs its N reals as z[m] = p[2m] + i p[2m+1] (m < N/2),
//   takes the length-N complex FFT of z padded with N/2 zeros (first stage pruned),
//   and recombines X[j] = (Z[j] + Z*[N-j])/2 - (i/2) e^{-2 pi i j/2N} (Z[j] - Z*[N-j]),
//   j in [0, N], the half spectrum of the zero-padded length-2N real row.
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
template <> struct RegCfg<float, 4, 1> { static constexpr int MAXT = 256, MINB = 2; };
template <> struct RegCfg<float, 3, 0> { static constexpr int MAXT = 512, MINB = 3; };
template <int KIND> struct RegCfg<double, 3, KIND> { static constexpr int MAXT = 512, MINB = 1; };
template <int KIND> struct RegCfg<double, 4, KIND> { static constexpr int MAXT = 256, MINB = 1; };

__host__ __device__ constexpr int spec_index_base(int j, int N, int r) { return ((j >> 2) * N + r) * 4 + (j & 3); }

template <typename T, int LOGN, int LOGR>
__global__ void __launch_bounds__(RegCfg<T, LOGR, 0>::MAXT, RegCfg<T, LOGR, 0>::MINB)
k_row_fwd_r(const T* __restrict__ p, cplx<T>* __restrict__ spec, const cplx<T>* __restrict__ twr,
            const cplx<T>* __restrict__ tw, const int* __restrict__ skip) {
  using C = cplx<T>;
  using P = Plan<LOGN, LOGR>;
  constexpr int N = 1 << LOGN, TT = P::T, SH = P::PADL + 8, R = P::R;
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rpb = blockDim.x / TT;
  const int rl = threadIdx.x / TT, t = threadIdx.x - rl * TT;
  const int r = blockIdx.x * rpb + rl;
  C* sh = reinterpret_cast<C*>(smem_raw) + rl * SH;
  C v[R];
  const C* prow = reinterpret_cast<const C*>(p + (size_t)r * N);
#pragma unroll
  for (int q = 0; q < R / 2; ++q) v[q] = prow[t + TT * q];
#pragma unroll
  for (int q = R / 2; q < R; ++q) v[q] = mk((T)0, (T)0);
  reg_fft<LOGN, LOGR, false, true, T>(v, sh, twr, t);
#pragma unroll
  for (int q = 0; q < R; ++q) sh[padi<LOGR>(t + TT * q)] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = t + TT * q;
    const C za = v[q];
    const C zb = cconj(sh[padi<LOGR>((N - j) & (N - 1))]);
    const C E = cscale(cadd(za, zb), (T)0.5);
    const C O = cscale(cmul_mi(csub(za, zb)), (T)0.5);
    spec[spec_index_base(j, N, r)] = cadd(E, cmul(O, tw[j]));
  }
  if (t < 4) {
    // j = N (Nyquist): X[N] = Re Z[0] - Im Z[0]; the other three slots of that block are zero
    const C z0 = sh[0];
    spec[spec_index_base(N + t, N, r)] = (t == 0) ? mk(z0.x - z0.y, (T)0) : mk((T)0, (T)0);
  }
}

template <typename T, int LOGN, int LOGR>
__global__ void __launch_bounds__(RegCfg<T, LOGR, 0>::MAXT, RegCfg<T, LOGR, 0>::MINB)
k_row_inv_r(const cplx<T>* __restrict__ spec, T* __restrict__ u, const cplx<T>* __restrict__ twr,
            const cplx<T>* __restrict__ tw, const int* __restrict__ skip) {
  using C = cplx<T>;
  using P = Plan<LOGN, LOGR>;
  constexpr int N = 1 << LOGN, TT = P::T, SH = P::PADL + 8, R = P::R;
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rpb = blockDim.x / TT;
  const int rl = threadIdx.x / TT, t = threadIdx.x - rl * TT;
  const int r = blockIdx.x * rpb + rl;
  C* sh = reinterpret_cast<C*>(smem_raw) + rl * SH;
  C v[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = t + TT * q;
    const C y1 = spec[spec_index_base(j, N, r)];
    const C y2 = cconj(spec[spec_index_base(N - j, N, r)]);
    const C e = cadd(y1, y2);
    const C o = cmul_pi(cmulc(csub(y1, y2), tw[j]));
    v[q] = cadd(e, o);
  }
  reg_fft<LOGN, LOGR, true, false, T>(v, sh, twr, t);
  C* urow = reinterpret_cast<C*>(u + (size_t)r * N);
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
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cpb = blockDim.x / TT;
  const int cl = cpb < 4 ? cpb : 4;
  const int c_lo = threadIdx.x % cl, rest = threadIdx.x / cl;
  const int t = rest % TT, c_hi = rest / TT;
  const int c = c_hi * cl + c_lo;
  const int slot = blockIdx.x * cpb + c;
  const bool active = slot < nslots;
  const int cb = slot >> 2, tc = slot & 3;
  C* sh = reinterpret_cast<C*>(smem_raw) + c * SH;
  C* col = spec + (size_t)cb * N * 4 + tc;
  C v[R];
#pragma unroll
  for (int q = 0; q < R / 2; ++q) v[q] = active ? col[(size_t)(t + TT * q) * 4] : mk((T)0, (T)0);
#pragma unroll
  for (int q = R / 2; q < R; ++q) v[q] = mk((T)0, (T)0);
  reg_fft<LOGM, LOGR, false, true, T>(v, sh, twc, t);
  const T* kt = table + (size_t)slot * (N + 4);   // column j = slot of the square table (row stride N + 4)
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int i = t + TT * q;
    const int f = (q < R / 2) ? i : M - i;
    const T kv = active ? kt[f] : (T)0;
    v[q] = cscale(v[q], kv);
  }
  reg_fft<LOGM, LOGR, true, false, T>(v, sh, twc, t);
  if (active) {
#pragma unroll
    for (int q = 0; q < R / 2; ++q) col[(size_t)(t + TT * q) * 4] = v[q];
  }
}

// cp.async helpers (asynchronous global -> shared copies, completion by group)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Persistent column pass: each block walks the columns slot = blockIdx.x + k gridDim.x
// and, while transforming one column, copies the next column's N input values and
// its table row into the other half of a double-buffered shared stage.
template <typename T, int LOGM, int LOGR>
__global__ void __launch_bounds__(RegCfg<T, LOGR, 1>::MAXT, RegCfg<T, LOGR, 1>::MINB)
k_col_p(cplx<T>* __restrict__ spec, const T* __restrict__ table, const cplx<T>* __restrict__ twc, int nslots,
        const int* __restrict__ skip) {
  using C = cplx<T>;
  using P = Plan<LOGM, LOGR>;
  constexpr int M = 1 << LOGM, N = M / 2, TT = P::T, R = P::R, NS = N + 4;
  static_assert(sizeof(T) == 4, "persistent column pass is float only");
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sh = reinterpret_cast<C*>(smem_raw);                       // exchange, PADL + 8
  C* instage = sh + (P::PADL + 8);                               // [2][N]
  T* tabstage = reinterpret_cast<T*>(instage + 2 * N);           // [2][NS]
  const int t = threadIdx.x;
  auto issue = [&](int slot, int b) {
    const int cb = slot >> 2, tc = slot & 3;
    const C* col = spec + (size_t)cb * N * 4 + tc;
    C* dst = instage + b * N;
#pragma unroll
    for (int q = 0; q < R / 2; ++q) cp_async8(dst + t + TT * q, col + (size_t)(t + TT * q) * 4);
    const T* kt = table + (size_t)slot * NS;
    T* tdst = tabstage + b * NS;
    for (int c4 = t; c4 < NS / 4; c4 += TT) cp_async16(tdst + 4 * c4, kt + 4 * c4);
  };
  int slot = blockIdx.x;
  if (slot < nslots) issue(slot, 0);
  cp_async_commit();
  for (int it = 0; slot < nslots; ++it, slot += gridDim.x) {
    const int b = it & 1;
    const int nslot = slot + gridDim.x;
    if (nslot < nslots) issue(nslot, b ^ 1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    C v[R];
    const C* src = instage + b * N;
#pragma unroll
    for (int q = 0; q < R / 2; ++q) v[q] = src[t + TT * q];
#pragma unroll
    for (int q = R / 2; q < R; ++q) v[q] = mk((T)0, (T)0);
    reg_fft<LOGM, LOGR, false, true, T>(v, sh, twc, t);
    const T* kt = tabstage + b * NS;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = t + TT * q;
      v[q] = cscale(v[q], kt[(q < R / 2) ? i : M - i]);
    }
    reg_fft<LOGM, LOGR, true, false, T>(v, sh, twc, t);
    const int cb = slot >> 2, tc = slot & 3;
    C* col = spec + (size_t)cb * N * 4 + tc;
#pragma unroll
    for (int q = 0; q < R / 2; ++q) col[(size_t)(t + TT * q) * 4] = v[q];
    __syncthreads();   // every read of stage b is done before it is refilled
  }
}

// stage twiddle tables of the register FFT of length 2^logl with radix 2^logr:
// stage s >= 1 holds w(r, k) = e^{-2 pi i k r / (Ns R)} at [(r-1)/2][k][(r-1)%2]
template <typename T>
__global__ void k_stage_twiddles(cplx<T>* __restrict__ out, int logl, int logr) {
  const int sr = logl / logr, logrl = logl % logr;
  const int nst = sr + (logrl ? 1 : 0);
  int off = 0, ns = 1;
  for (int s = 0; s < nst; ++s) {
    const int R = (s < sr) ? (1 << logr) : (1 << logrl);
    if (s > 0) {
      const int cnt = R * ns;
      for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < cnt; idx += gridDim.x * blockDim.x) {
        const int e = idx & 1, k = (idx >> 1) % ns, pr = (idx >> 1) / ns;
        const int r = 2 * pr + 1 + e;
        double sn = 0.0, cs = 1.0;
        if (r < R) sincospi(2.0 * (double)k * (double)r / (double)(ns * R), &sn, &cs);
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
  static void pass(const bem_kernel_s* k, int which, const T* p, T* u, cudaStream_t s, const int* skip) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_row_fwd_r<T, LOGN, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(k_row_inv_r<T, LOGN, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr = true;
    }
    constexpr int N = 1 << LOGN;
    using PR = Plan<LOGN, LOGR>;
    int rpb = RegCfg<T, LOGR, 0>::MAXT / PR::T;
    if (rpb < 1) rpb = 1;
    if (rpb > N) rpb = N;
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
  static void pass(const bem_kernel_s* k, const int* skip, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_col_r<T, LOGN + 1, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr = true;
    }
    constexpr int N = 1 << LOGN;
    using PC = Plan<LOGN + 1, LOGR>;
    if constexpr (sizeof(T) == 4 && LOGN >= 6) {
      if (k->col_persist) {
        static int grid = 0;
        const size_t smem = (size_t)(PC::PADL + 8 + 2 * N) * sizeof(C) + 2 * (N + 4) * sizeof(T);
        if (grid == 0) {
          cudaFuncSetAttribute(k_col_p<T, LOGN + 1, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
          int per_sm = 0, sms = 0, dev = 0;
          cudaGetDevice(&dev);
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_col_p<T, LOGN + 1, LOGR>, PC::T, smem);
          grid = (per_sm > 0 ? per_sm : 1) * sms;
        }
        const int nslots = N + 4;
        k_col_p<T, LOGN + 1, LOGR><<<grid < nslots ? grid : nslots, PC::T, smem, s>>>(
            (C*)k->ws.spec, (const T*)k->ws.table, (const C*)k->ws.twc, nslots, skip);
        return;
      }
    }
    int cpb = RegCfg<T, LOGR, 1>::MAXT / PC::T;
    if (cpb < 1) cpb = 1;
    const int nslots = N + 4;
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

template <typename T>
void reg_twiddles(const bem_kernel_s* k, cudaStream_t s) {
  k_stage_twiddles<T><<<64, 256, 0, s>>>((cplx<T>*)k->ws.twr, k->logN, row_logr<T>(k));
  k_stage_twiddles<T><<<64, 256, 0, s>>>((cplx<T>*)k->ws.twc, k->logN + 1, col_logr<T>(k));
}

}  // namespace bem
