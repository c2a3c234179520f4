// Block-cooperative Stockham FFT in shared memory (radix 4, one radix-2 stage when
// log2 L is odd).  Unnormalised in both directions: forward uses e^{-2 pi i kn/L},
// inverse e^{+2 pi i kn/L}.
#pragma once

#include "bem_internal.cuh"

namespace bem {

// tw[m] = e^{-2 pi i m / M} for m in [0, M); the inverse direction conjugates it.
template <bool INV, typename C>
__device__ __forceinline__ C twid(const C* __restrict__ tw, int idx) {
  C w = tw[idx];
  return INV ? cconj(w) : w;
}

template <bool INV, typename C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  const C a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = csub(v1, v3);
  const C dm = INV ? cmul_pi(d) : cmul_mi(d);
  v0 = cadd(a, c);
  v2 = csub(a, c);
  v1 = cadd(b, dm);
  v3 = csub(b, dm);
}

// nb sequences of length L = 2^logL (L >= 2) stored back to back in `a`; `b` is
// scratch of the same size.  Every thread of the block must call this after a
// __syncthreads() that publishes `a`; it ends with one.  Returns the buffer that
// holds the result.  Stage s of the self-sorting (Stockham) form with radix R and
// span Ns reads x[j + r L/R], twiddles by e^{-+2 pi i (j mod Ns) r/(Ns R)}, applies
// the R-point DFT and writes y[(j/Ns) Ns R + (j mod Ns) + r Ns].
template <bool INV, typename C>
__device__ C* block_fft(C* a, C* b, int logL, int nb, const C* __restrict__ tw, int logM) {
  int logNs = 0;
  while (logNs < logL) {
    const bool r4 = (logL - logNs) >= 2;
    const int logR = r4 ? 2 : 1;
    const int Ns = 1 << logNs;
    const int nbf_log = logL - logR;
    const int nbf = 1 << nbf_log;
    const int total = nb << nbf_log;
    const int twshift = logM - logNs - logR;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int s = idx >> nbf_log;
      const int j = idx & (nbf - 1);
      const C* src = a + (s << logL);
      C* dst = b + (s << logL);
      const int k = j & (Ns - 1);
      const int ob = ((j >> logNs) << (logNs + logR)) + k;
      if (r4) {
        C v0 = src[j], v1 = src[j + nbf], v2 = src[j + 2 * nbf], v3 = src[j + 3 * nbf];
        if (logNs > 0) {
          v1 = cmul(v1, twid<INV>(tw, k << twshift));
          v2 = cmul(v2, twid<INV>(tw, (2 * k) << twshift));
          v3 = cmul(v3, twid<INV>(tw, (3 * k) << twshift));
        }
        dft4<INV>(v0, v1, v2, v3);
        dst[ob] = v0;
        dst[ob + Ns] = v1;
        dst[ob + 2 * Ns] = v2;
        dst[ob + 3 * Ns] = v3;
      } else {
        C v0 = src[j], v1 = src[j + nbf];
        if (logNs > 0) v1 = cmul(v1, twid<INV>(tw, k << twshift));
        dst[ob] = cadd(v0, v1);
        dst[ob + Ns] = csub(v0, v1);
      }
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
    logNs += logR;
  }
  return a;
}

}  // namespace bem
