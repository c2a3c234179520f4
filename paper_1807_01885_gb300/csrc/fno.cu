// Fourier-neural-operator warm start: forward, backward and Adam on the GPU.
//
// The network (layers defined in include/bem.h, bem_fno_*): a pointwise lift from 7
// input features to W channels, L layers z = S(v) + W_l v + b_l with v' = gelu(z)
// (no gelu after the last), and a projection h = gelu(Q1 v + q1), out = Q2 h + q2.
// S is the spectral convolution on the retained modes kx in {0..m-1, N-m..N-1},
// ky in {0..m-1}: a truncated DFT of each channel, a complex W x W mixing per mode
// and the truncated inverse with half-spectrum weights c_0 = 1, c_ky = 2.
//
// Precision: parameters are kept in float (master copy, Adam state) and used by every
// kernel from a bfloat16 copy refreshed after each update; activations, gradients and
// all accumulations are float (bf16 in, fp32 accumulate).  The truncated transforms
// are direct sums against a float twiddle table (the retained modes are few, so the
// O(N m) sums are cheaper than full FFTs).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "bem_internal.cuh"

namespace bem {
namespace {

constexpr int FT = 256;   // threads per block
using bf16 = __nv_bfloat16;

__device__ __forceinline__ float b2f(bf16 x) { return __bfloat162float(x); }

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
// gelu of two values at once on packed .f32x2 arithmetic (the fused layer and
// projection epilogues), with erf by Abramowitz & Stegun 7.1.26 (|error| <= 1.5e-7):
// 1 + erf(u) = 2 - y for u >= 0 and y for u < 0, y = t P(t) e^{-u^2} = erfc(|u|),
// t = 1 / (1 + p |u|).  The polynomial and the products run two lanes per
// instruction; the reciprocal and the exponential stay per value (MUFU).
typedef unsigned long long g2x;
__device__ __forceinline__ g2x gpk(float a, float b) {
  g2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void gup(g2x v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ g2x gfma(g2x a, g2x b, g2x c) {
  g2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ g2x gmul(g2x a, g2x b) {
  g2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ g2x gsplat(float a) { return gpk(a, a); }
__device__ __forceinline__ void gelu2(float& z0, float& z1) {
  const g2x z = gpk(z0, z1);
  const g2x u = gmul(z, gsplat(0.70710678118654752f));
  const g2x a = u & 0x7fffffff7fffffffull;   // |u| in both lanes
  float d0, d1;
  gup(gfma(a, gsplat(0.3275911f), gsplat(1.f)), d0, d1);
  const g2x t = gpk(__fdividef(1.f, d0), __fdividef(1.f, d1));
  g2x y = gfma(t, gsplat(1.061405429f), gsplat(-1.453152027f));
  y = gfma(t, y, gsplat(1.421413741f));
  y = gfma(t, y, gsplat(-0.284496736f));
  y = gfma(t, y, gsplat(0.254829592f));
  float q0, q1;
  gup(gmul(a, a), q0, q1);
  y = gmul(gmul(t, y), gpk(__expf(-q0), __expf(-q1)));
  float y0, y1, u0, u1;
  gup(y, y0, y1);
  gup(u, u0, u1);
  gup(gmul(gmul(z, gsplat(0.5f)), gpk(u0 >= 0.f ? 2.f - y0 : y0, u1 >= 0.f ? 2.f - y1 : y1)), z0, z1);
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + FT - 1) / FT, 65535u * 16u); }

#define FOR_N(i, n) for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// inputs

// per-sample mean and standard deviation of the height map: kMomChunks blocks per
// sample add the values and squares of their chunk in double (a few per thread,
// spread over the whole GPU: double arithmetic runs at a fraction of the float
// rate), then one block per sample adds its chunk sums in chunk order
constexpr int kMomChunks = 64;

__global__ void k_fno_moments_part(const float* __restrict__ f, double* __restrict__ part, size_t P) {
  const int b = blockIdx.y, ch = blockIdx.x;
  const size_t lo = P * ch / kMomChunks, hi = P * (ch + 1) / kMomChunks;
  const float* fb = f + (size_t)b * P;
  double s = 0.0, s2 = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double v = fb[i];
    s += v;
    s2 += v * v;
  }
  __shared__ double sh[2][FT];
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = s2;
  __syncthreads();
  for (int o = FT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((size_t)b * kMomChunks + ch) * 2] = sh[0][0];
    part[((size_t)b * kMomChunks + ch) * 2 + 1] = sh[1][0];
  }
}

// mom[4b .. 4b+3] = mean, 1/std, log(h/delta)/log 200, log(E1/E2)/log 20 of sample b
__global__ void k_fno_moments(const double* __restrict__ part, const double* __restrict__ sp,
                              float* __restrict__ mom, size_t P) {
  if (threadIdx.x != 0) return;
  const double* pb = part + (size_t)blockIdx.x * kMomChunks * 2;
  double s = 0.0, s2 = 0.0;
  for (int ch = 0; ch < kMomChunks; ++ch) {
    s += pb[2 * ch];
    s2 += pb[2 * ch + 1];
  }
  const double mean = s / (double)P;
  const double var = fmax(s2 / (double)P - mean * mean, 1e-30);
  float* mb = mom + 4 * (size_t)blockIdx.x;
  mb[0] = (float)mean;
  mb[1] = (float)(1.0 / sqrt(var));
  mb[2] = (float)(log(sp[4 * blockIdx.x]) / log(200.0));
  mb[3] = (float)(log(sp[4 * blockIdx.x + 1]) / log(20.0));
}

// x[b][0] = normalised height, [1] = log(h/delta)/log 200, [2] = log(E1/E2)/log 20,
// [3] = nu1, [4] = nu2, [5] = (c + 1/2)/N, [6] = (r + 1/2)/N
__global__ void k_fno_features(const float* __restrict__ f, const float* __restrict__ mom,
                               const double* __restrict__ sp, float* __restrict__ x, int N, int B) {
  const size_t P = (size_t)N * N;
  FOR_N(i, (size_t)B * P) {
    const int b = (int)(i / P);
    const size_t pix = i % P;
    const int r = (int)(pix / N), c = (int)(pix % N);
    float* xb = x + (size_t)b * 7 * P;
    const float* mb = mom + 4 * (size_t)b;
    xb[pix] = (f[i] - mb[0]) * mb[1];
    xb[P + pix] = mb[2];
    xb[2 * P + pix] = mb[3];
    xb[3 * P + pix] = (float)sp[4 * b + 2];
    xb[4 * P + pix] = (float)sp[4 * b + 3];
    xb[5 * P + pix] = ((float)c + 0.5f) / (float)N;
    xb[6 * P + pix] = ((float)r + 0.5f) / (float)N;
  }
}

// ---------------------------------------------------------------------------
// pointwise (1x1) layers: Y[b][o][p] = bias[o] + sum_c W[o][c] X[b][c][p]
// TRANS: use W^T (backward data pass: W stored [Cout_fwd][Cin_fwd], here o = c_fwd).
template <int CIN, bool TRANS, bool ACCUM, bool GELU>
__global__ void k_pw(const float* __restrict__ X, const bf16* __restrict__ Wt, const bf16* __restrict__ bias,
                     float* __restrict__ Y, float* __restrict__ Yact, int cout, size_t P) {
  extern __shared__ float wsh[];
  for (int i = threadIdx.x; i < cout * CIN; i += blockDim.x) {
    const int o = i / CIN, c = i % CIN;
    wsh[i] = TRANS ? b2f(Wt[(size_t)c * cout + o]) : b2f(Wt[i]);
  }
  __syncthreads();
  const int b = blockIdx.y;
  const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= P) return;
  float xr[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) xr[c] = X[((size_t)b * CIN + c) * P + p];
  for (int o = 0; o < cout; ++o) {
    float acc = bias != nullptr ? b2f(bias[o]) : 0.f;
    const float* w = wsh + o * CIN;
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc = fmaf(w[c], xr[c], acc);
    float* y = Y + ((size_t)b * cout + o) * P + p;
    if (ACCUM) acc += *y;
    *y = acc;
    if (GELU) Yact[((size_t)b * cout + o) * P + p] = gelu_f(acc);
  }
}

// weight gradient partials: per block of FT pixels (of one sample) the Cout x Cin
// products and the Cout bias sums; summed over blocks by k_pw_wgrad_sum
__global__ void k_pw_wgrad(const float* __restrict__ dY, const float* __restrict__ X, float* __restrict__ part,
                           int cout, int cin, size_t P) {
  extern __shared__ float sh[];
  float* dys = sh;                 // [cout][FT]
  float* xs = sh + cout * FT;      // [cin][FT]
  const int b = blockIdx.y;
  const size_t p0 = blockIdx.x * (size_t)FT;
  const int np = (int)std::min<size_t>(FT, P - p0);
  for (int o = 0; o < cout; ++o)
    dys[o * FT + threadIdx.x] = (int)threadIdx.x < np ? dY[((size_t)b * cout + o) * P + p0 + threadIdx.x] : 0.f;
  for (int c = 0; c < cin; ++c)
    xs[c * FT + threadIdx.x] = (int)threadIdx.x < np ? X[((size_t)b * cin + c) * P + p0 + threadIdx.x] : 0.f;
  __syncthreads();
  const size_t blk = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  const int nout = cout * cin + cout;
  for (int e = threadIdx.x; e < nout; e += blockDim.x) {
    float acc = 0.f;
    if (e < cout * cin) {
      const int o = e / cin, c = e % cin;
      for (int k = 0; k < FT; ++k) acc = fmaf(dys[o * FT + k], xs[c * FT + k], acc);
    } else {
      const int o = e - cout * cin;
      for (int k = 0; k < FT; ++k) acc += dys[o * FT + k];
    }
    part[blk * nout + e] = acc;
  }
}

__global__ void k_pw_wgrad_sum(const float* __restrict__ part, int nblk, int cout, int cin, float* __restrict__ gw,
                               float* __restrict__ gb) {
  const int nout = cout * cin + cout;
  FOR_N(e, (size_t)nout) {
    float acc = 0.f;
    for (int k = 0; k < nblk; ++k) acc += part[(size_t)k * nout + e];
    if (e < (size_t)cout * cin) gw[e] = acc;
    else gb[e - (size_t)cout * cin] = acc;
  }
}

__global__ void k_gelu_bwd(const float* __restrict__ dv, const float* __restrict__ z, float* __restrict__ dz, size_t n) {
  FOR_N(i, n) dz[i] = dv[i] * gelu_grad_f(z[i]);
}

// ---------------------------------------------------------------------------
// truncated transforms; tw[k] = e^{-2 pi i k / N}

__device__ __forceinline__ int kx_of(int kxi, int m, int N) { return kxi < m ? kxi : N - 2 * m + kxi; }



// A[bc][x][ky] = sum_kxi Y[bc][kxi][ky] e^{+2 pi i kx x/N}: one thread per (bc, x) and
// four consecutive ky (one twiddle load serves four outputs)
__global__ void k_idft_x(const float2* __restrict__ Y, float2* __restrict__ A, const float2* __restrict__ tw, int N,
                         int m, size_t bc) {
  const int mq = (m + 3) / 4;
  FOR_N(i, bc * (size_t)N * mq) {
    const size_t q = i / ((size_t)N * mq);
    const int rem = (int)(i - q * ((size_t)N * mq));
    const int x = rem / mq, ky0 = 4 * (rem - (rem / mq) * mq);
    const int nk = min(4, m - ky0);
    const float2* y = Y + q * 2 * m * m + ky0;
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    // twiddle index kx x mod N, stepped by x: kx = kxi for kxi < m, kx = kxi - 2m (mod N) after
    int idx = 0;
    for (int kxi = 0; kxi < 2 * m; ++kxi) {
      if (kxi == m) idx = (int)((N - (int)(((long long)m * x) % N)) % N);
      const float2 w = tw[idx];   // e^{-i theta}; conjugate below
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (e < nk) {
          const float2 v = y[(size_t)kxi * m + e];
          re[e] += v.x * w.x + v.y * w.y;
          im[e] += v.y * w.x - v.x * w.y;
        }
      }
      idx += x;
      if (idx >= N) idx -= N;
    }
    float2* a = A + (q * N + x) * m + ky0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < nk) a[e] = make_float2(re[e], im[e]);
  }
}


// Truncated transforms along y as matrix products (FP32, register-blocked tiles in
// shared memory).  Tf[y][2k] + i Tf[y][2k+1] = e^{-2 pi i k y / N} (k < m) and
// Ti[2k + e][y] = Tf[y][2k + e]: the forward transform of every row is A = V Tf,
// the inverse out[y] = sum_k c_k Re(A_k conj(w_k(y))) is (A diag(c)) Ti.
__global__ void k_twiddle_mats(const float2* __restrict__ tw, float* __restrict__ Tf, float* __restrict__ Ti, int N,
                               int m) {
  FOR_N(i, (size_t)N * m) {
    const int y = (int)(i / m), k = (int)(i % m);
    const float2 w = tw[((size_t)k * y) % N];
    Tf[(size_t)y * 2 * m + 2 * k] = w.x;
    Tf[(size_t)y * 2 * m + 2 * k + 1] = w.y;
    Ti[(size_t)(2 * k) * N + y] = w.x;
    Ti[(size_t)(2 * k + 1) * N + y] = w.y;
  }
}

// ---- truncated transforms along y on the tensor cores ----------------------------
// Both y-transforms are matrix products with a dimension of 2m (= n2m) on one side:
// forward C (rows x n2m) = V (rows x N) Tf (N x n2m), inverse out (rows x N) =
// (A diag(cs)) (rows x n2m) Ti (n2m x N).  They run as mma.sync m16n8k16 with bf16
// operands and float accumulation.  A bf16 value keeps 8 significant bits, so every
// float operand x is split into hi = bf16(x) and lo = bf16(x - hi) (together 16 bits,
// |x - hi - lo| <= 2^-18 |x|), and a product takes the three terms hi.hi, hi.lo, lo.hi
// (the dropped lo.lo is below 2^-18 of it): float-level products from bf16 inputs.
// The constant operand (Tf or Ti) is stored split and in fragment order: for k-block
// kb (16 k) and n-tile nt (8 columns), lane l holds uint4 (hi b0, hi b1, lo b0, lo b1)
// with b0 = (B[16 kb + 2t][8 nt + g], B[16 kb + 2t + 1][.]), b1 = the same 8 k further,
// g = l / 4, t = l % 4 (the m16n8k16 B layout); entries outside the matrix are 0.
__device__ __forceinline__ unsigned pack_bf16x2(float lo_elem, float hi_elem) {
  unsigned d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_elem), "f"(lo_elem));
  return d;
}
__device__ __forceinline__ float bf16_lo_f(unsigned v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi_f(unsigned v) { return __uint_as_float(v & 0xffff0000u); }
// (x0, x1) -> hi and lo bf16 pairs, x0 in the lower half
__device__ __forceinline__ void split2(float x0, float x1, unsigned& hi, unsigned& lo) {
  hi = pack_bf16x2(x0, x1);
  lo = pack_bf16x2(x0 - bf16_lo_f(hi), x1 - bf16_hi_f(hi));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// hi.hi + hi.lo + lo.hi
__device__ __forceinline__ void mma3(float (&d)[4], const unsigned (&ah)[4], const unsigned (&al)[4], uint4 b) {
  mma_bf16(d, ah, b.x, b.y);
  mma_bf16(d, ah, b.z, b.w);
  mma_bf16(d, al, b.x, b.y);
}

// fragment-ordered split copy of B (K x Ncols, element (k, n) at Bm[k ldk + n ldn])
__global__ void k_frag_b(const float* __restrict__ Bm, int K, int Nc, size_t ldk, size_t ldn, uint4* __restrict__ out) {
  const int KT = (K + 15) / 16, NT = (Nc + 7) / 8;
  FOR_N(i, (size_t)KT * NT * 32) {
    const int lane = (int)(i % 32), nt = (int)((i / 32) % NT), kb = (int)(i / (32 * (size_t)NT));
    const int g = lane / 4, t = lane % 4, n = 8 * nt + g;
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 16 * kb + 2 * t + (e & 1) + 8 * (e >> 1);
      v[e] = (k < K && n < Nc) ? Bm[(size_t)k * ldk + (size_t)n * ldn] : 0.f;
    }
    unsigned h0, l0, h1, l1;
    split2(v[0], v[1], h0, l0);
    split2(v[2], v[3], h1, l1);
    out[i] = make_uint4(h0, h1, l0, l1);
  }
}

constexpr int TC_NT_MAX = 8;   // n2m <= 64 (modes <= 32) on the tensor-core path

// C[r][j] = sum_y V[r][y] Tf[y][j]: one warp per 32 rows (two m-tiles sharing every
// B fragment), every n-tile of n2m (NT = ceil(n2m / 8))
template <int NT>
__global__ void __launch_bounds__(128) k_dft_y_tc(const float* __restrict__ V, const uint4* __restrict__ TfB,
                                                  float* __restrict__ C, size_t rows, int N, int n2m) {
  const int lane = threadIdx.x % 32, g = lane / 4, t = lane % 4;
  const size_t R0 = ((size_t)blockIdx.x * 4 + threadIdx.x / 32) * 32;
  if (R0 >= rows) return;
  const int KT = (N + 15) / 16;
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
  size_t r[2][2];
  bool ok[2][2];
  const float* vr[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      r[mt][h] = R0 + 16 * mt + g + 8 * h;
      ok[mt][h] = r[mt][h] < rows;
      vr[mt][h] = V + (ok[mt][h] ? r[mt][h] : 0) * N;
    }
  const bool full = (N % 16) == 0;
#pragma unroll 2
  for (int kb = 0; kb < KT; ++kb) {
    const int k0 = 16 * kb + 2 * t, k1 = k0 + 8;
    unsigned ah[2][4], al[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      float2 x[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int h = e & 1, k = (e < 2) ? k0 : k1;
        x[e] = (ok[mt][h] && (full || k < N)) ? *reinterpret_cast<const float2*>(vr[mt][h] + k)
                                               : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) split2(x[e].x, x[e].y, ah[mt][e], al[mt][e]);
    }
    const uint4* bk = TfB + (size_t)kb * NT * 32 + lane;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const uint4 b = bk[nt * 32];
      mma3(acc[0][nt], ah[0], al[0], b);
      mma3(acc[1][nt], ah[1], al[1], b);
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int col = 8 * nt + 2 * t;
      if (col < n2m) {
        if (ok[mt][0]) *reinterpret_cast<float2*>(C + r[mt][0] * n2m + col) = make_float2(acc[mt][nt][0], acc[mt][nt][1]);
        if (ok[mt][1]) *reinterpret_cast<float2*>(C + r[mt][1] * n2m + col) = make_float2(acc[mt][nt][2], acc[mt][nt][3]);
      }
    }
}

// out[r][y] (+)= sum_k A[r][k] cs(k) Ti[k][y], cs(k) = scale (c ? c[k/2] : 1): one
// warp per 16 rows and 64 columns (8 n-tiles), the scaled A split once per warp
constexpr int TC_IY = 64;
template <bool ACCUM>
__global__ void __launch_bounds__(128) k_idft_y_tc(const float* __restrict__ A, const uint4* __restrict__ TiB,
                                                   const float* __restrict__ c, float scale, float* __restrict__ out,
                                                   size_t rows, int N, int n2m) {
  const int lane = threadIdx.x % 32, g = lane / 4, t = lane % 4;
  const size_t R0 = ((size_t)blockIdx.x * 4 + threadIdx.x / 32) * 16;
  if (R0 >= rows) return;
  const int y0 = blockIdx.y * TC_IY;
  const int KT = (n2m + 15) / 16, NT = (N + 7) / 8;
  const size_t ra = R0 + g, rb = R0 + g + 8;
  const bool oka = ra < rows, okb = rb < rows;
  unsigned ah[4][4], al[4][4];   // k-blocks (n2m <= 64)
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    const int k0 = 16 * kb + 2 * t, k1 = k0 + 8;
    auto ld = [&](bool ok, size_t r, int k) -> float2 {
      if (!ok || k >= n2m) return make_float2(0.f, 0.f);
      const float2 v = *reinterpret_cast<const float2*>(A + r * n2m + k);
      const float s0 = scale * (c != nullptr ? c[k / 2] : 1.f), s1 = scale * (c != nullptr ? c[(k + 1) / 2] : 1.f);
      return make_float2(v.x * s0, v.y * s1);
    };
    float2 x0 = make_float2(0.f, 0.f), x1 = x0, x2 = x0, x3 = x0;
    if (kb < KT) {
      x0 = ld(oka, ra, k0);
      x1 = ld(okb, rb, k0);
      x2 = ld(oka, ra, k1);
      x3 = ld(okb, rb, k1);
    }
    split2(x0.x, x0.y, ah[kb][0], al[kb][0]);
    split2(x1.x, x1.y, ah[kb][1], al[kb][1]);
    split2(x2.x, x2.y, ah[kb][2], al[kb][2]);
    split2(x3.x, x3.y, ah[kb][3], al[kb][3]);
  }
#pragma unroll
  for (int j = 0; j < TC_IY / 8; ++j) {
    const int nt = y0 / 8 + j;
    if (nt >= NT) break;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kb = 0; kb < 4; ++kb)
      if (kb < KT) mma3(acc, ah[kb], al[kb], TiB[((size_t)kb * NT + nt) * 32 + lane]);
    const int y = 8 * nt + 2 * t;
    if (y < N) {
      if (oka) {
        float2* o = reinterpret_cast<float2*>(out + ra * N + y);
        float2 v = make_float2(acc[0], acc[1]);
        if (ACCUM) { const float2 w = *o; v.x += w.x; v.y += w.y; }
        *o = v;
      }
      if (okb) {
        float2* o = reinterpret_cast<float2*>(out + rb * N + y);
        float2 v = make_float2(acc[2], acc[3]);
        if (ACCUM) { const float2 w = *o; v.x += w.x; v.y += w.y; }
        *o = v;
      }
    }
  }
}

// Pointwise (1x1) layer on the tensor cores: for 16 pixels of one sample (a tile)
// D (pixels x cout) = X^T (pixels x cin) W^T (cin x cout), the activations split into
// bf16 hi + lo (two mma.sync each), the weights used as they are stored (bf16).  Same
// result as k_pw: Y[b][o][p] = bias[o] + sum_c W[o][c] X[b][c][p] (+ Y when ACCUM),
// Yact = gelu(Y) when GELU; TRANS uses W^T.  KT = ceil(cin/16) k-blocks, NT =
// ceil(cout/8) n-tiles (cout <= 64).  Each warp loads its weight fragments once and
// runs kPwTiles consecutive tiles.
constexpr int kPwTiles = 8;
template <int KT, int NT, bool TRANS, bool ACCUM, bool GELU>
__global__ void __launch_bounds__(128) k_pw_tc(const float* __restrict__ X, int cin, const bf16* __restrict__ Wt,
                                               const bf16* __restrict__ bias, float* __restrict__ Y,
                                               float* __restrict__ Yact, int cout, size_t P) {
  const int lane = threadIdx.x % 32, g = lane / 4, t = lane % 4;
  const int b = blockIdx.y;
  const size_t tiles = (P + 15) / 16;
  const size_t tile0 = ((size_t)blockIdx.x * 4 + threadIdx.x / 32) * kPwTiles;
  if (tile0 >= tiles) return;
  // B[c][o] = W[o][c]: TRANS reads Wt[c][o] (stored [cin][cout]), else Wt[o][c]
  auto wbits = [&](int c, int o) -> unsigned {
    if (c >= cin || o >= cout) return 0u;
    const bf16 w = TRANS ? Wt[(size_t)c * cout + o] : Wt[(size_t)o * cin + c];
    return (unsigned)__bfloat16_as_ushort(w);
  };
  unsigned wf[KT][NT][2];
#pragma unroll
  for (int kb = 0; kb < KT; ++kb)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int n = 8 * nt + g, c0 = 16 * kb + 2 * t, c1 = c0 + 8;
      wf[kb][nt][0] = wbits(c0, n) | (wbits(c0 + 1, n) << 16);
      wf[kb][nt][1] = wbits(c1, n) | (wbits(c1 + 1, n) << 16);
    }
  float bv[NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int o = 8 * nt + 2 * t + e;
      bv[nt][e] = (bias != nullptr && o < cout) ? b2f(bias[o]) : 0.f;
    }
  const float* xb = X + (size_t)b * cin * P;
  const size_t tile1 = tile0 + kPwTiles < tiles ? tile0 + kPwTiles : tiles;
  for (size_t tile = tile0; tile < tile1; ++tile) {
    const size_t pa = tile * 16 + g, pb = pa + 8;
    const bool oka = pa < P, okb = pb < P;
    auto xv = [&](int c, size_t p, bool ok) -> float { return (ok && c < cin) ? xb[(size_t)c * P + p] : 0.f; };
    unsigned ah[KT][4], al[KT][4];
#pragma unroll
    for (int kb = 0; kb < KT; ++kb) {
      const int c0 = 16 * kb + 2 * t, c1 = c0 + 8;
      split2(xv(c0, pa, oka), xv(c0 + 1, pa, oka), ah[kb][0], al[kb][0]);
      split2(xv(c0, pb, okb), xv(c0 + 1, pb, okb), ah[kb][1], al[kb][1]);
      split2(xv(c1, pa, oka), xv(c1 + 1, pa, oka), ah[kb][2], al[kb][2]);
      split2(xv(c1, pb, okb), xv(c1 + 1, pb, okb), ah[kb][3], al[kb][3]);
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kb = 0; kb < KT; ++kb) {
        mma_bf16(acc, ah[kb], wf[kb][nt][0], wf[kb][nt][1]);
        mma_bf16(acc, al[kb], wf[kb][nt][0], wf[kb][nt][1]);
      }
      // acc[0], acc[1]: pixel pa, outputs o0, o0 + 1; acc[2], acc[3]: pixel pb
      const int o0 = 8 * nt + 2 * t;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = o0 + (e & 1);
        const size_t p = (e < 2) ? pa : pb;
        const bool ok = (e < 2) ? oka : okb;
        if (!ok || o >= cout) continue;
        float v = acc[e] + bv[nt][e & 1];
        float* y = Y + ((size_t)b * cout + o) * P + p;
        if (ACCUM) v += *y;
        *y = v;
        if (GELU) Yact[((size_t)b * cout + o) * P + p] = gelu_f(v);
      }
    }
  }
}

// ---- fused Fourier layer (forward) --------------------------------------------
// One kernel for z = W v + b + S(v) and v' = gelu(z): for 16 pixels y of one row x of
// one sample, both contractions go into the same accumulator (pixels x cout):
//   W v:  A = v^T (pixels x cin, split hi/lo), B = W^T (bf16 as stored),
//   S(v): A = Tf (pixels y x 2m: the inverse y-transform's e^{+i k y} terms, which are
//         the forward twiddles read as Re/Im pairs), B = (c_k / N^2) A_row (2m x cout:
//         the x-inverse of the mixed modes of this row, split hi/lo), three products.
// The inverse y-transform's output never goes to memory.  The pixel-operand Tf is
// stored split and in A-fragment order (k_frag_a); the row operand is gathered once
// per warp and row.
// fragment-ordered split copy of A (M x K, element (r, k) at Am[r ldr + k]): for m-tile
// mt and k-block kb, lane l holds uint4 hi (a0..a3) and uint4 lo (a0..a3) with a0 =
// (A[16 mt + g][16 kb + 2t], A[.][+1]), a1 = row + 8, a2 = col + 8, a3 = both
__global__ void k_frag_a(const float* __restrict__ Am, int M, int K, size_t ldr, uint4* __restrict__ out) {
  const int MT = (M + 15) / 16, KB = (K + 15) / 16;
  FOR_N(i, (size_t)MT * KB * 32) {
    const int lane = (int)(i % 32), kb = (int)((i / 32) % KB), mt = (int)(i / (32 * (size_t)KB));
    const int g = lane / 4, t = lane % 4;
    unsigned h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 16 * mt + g + 8 * (e & 1), k = 16 * kb + 2 * t + 8 * (e >> 1);
      const float x0 = (r < M && k < K) ? Am[(size_t)r * ldr + k] : 0.f;
      const float x1 = (r < M && k + 1 < K) ? Am[(size_t)r * ldr + k + 1] : 0.f;
      split2(x0, x1, h[e], l[e]);
    }
    out[2 * i] = make_uint4(h[0], h[1], h[2], h[3]);
    out[2 * i + 1] = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// NT n-tiles of the outputs (width W = 8 NT), KT = ceil(W / 16) k-blocks of the channel
// contraction, KS k-blocks of the modes (2m <= 16 KS).  Warp w of the grid takes row
// (b, x) = w / chunks and the y-tiles [chunk * tpw, (chunk + 1) * tpw).  Offsets
// within one sample are 32-bit (W N^2 < 2^31).
template <int KT, int NT, int KS>
__global__ void __launch_bounds__(128) k_layer_tc(const float* __restrict__ V, const bf16* __restrict__ Ww,
                                                  const bf16* __restrict__ bias, const float* __restrict__ A,
                                                  const float* __restrict__ cs, const uint4* __restrict__ TfA,
                                                  float* __restrict__ Z, float* __restrict__ Vout, int N, int n2m,
                                                  size_t rows, int tpw, int gelu) {
  constexpr int W = 8 * NT;
  const int lane = threadIdx.x % 32, g = lane / 4, t = lane % 4;
  const int YT = (N + 15) / 16, chunks = (YT + tpw - 1) / tpw;
  const size_t w = (size_t)blockIdx.x * 4 + threadIdx.x / 32;
  const size_t row = w / chunks;
  if (row >= rows) return;
  const int chunk = (int)(w % chunks);
  const size_t b = row / N;
  const int x = (int)(row % N);
  const unsigned P = (unsigned)N * (unsigned)N;
  // B operands: W^T as stored (bf16), the row's mode coefficients split
  unsigned wf[KT][NT][2];
#pragma unroll
  for (int kb = 0; kb < KT; ++kb)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int o = 8 * nt + g;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int c = 16 * kb + 2 * t + 8 * hh;
        const bool cv = 16 * kb + 8 * hh < W;   // c < W for every lane, or for none
        const unsigned lo = cv ? (unsigned)__bfloat16_as_ushort(Ww[o * W + c]) : 0u;
        const unsigned hi = cv ? (unsigned)__bfloat16_as_ushort(Ww[o * W + c + 1]) : 0u;
        wf[kb][nt][hh] = lo | (hi << 16);
      }
    }
  unsigned sfh[KS][NT][2], sfl[KS][NT][2];
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int o = 8 * nt + g;
      const float* ar = A + ((b * W + o) * N + x) * n2m;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int k = 16 * ks + 2 * t + 8 * hh;
        const float x0 = k < n2m ? ar[k] * cs[k / 2] : 0.f;
        const float x1 = k + 1 < n2m ? ar[k + 1] * cs[(k + 1) / 2] : 0.f;
        split2(x0, x1, sfh[ks][nt][hh], sfl[ks][nt][hh]);
      }
    }
  float bv[NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) bv[nt][e] = bias != nullptr ? b2f(bias[8 * nt + 2 * t + e]) : 0.f;
  // this sample's planes, offset to row x
  const float* vb = V + b * W * (size_t)P + (size_t)x * N;
  const size_t ob = b * W * (size_t)P + (size_t)x * N;
  float* zb = Z != nullptr ? Z + ob : nullptr;
  float* ub = Vout + ob;
  const int yt0 = chunk * tpw, yt1 = min(YT, yt0 + tpw);
  auto tile = [&](int yt, auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
    const int ya = 16 * yt + g, yb = ya + 8;
    const bool oka = FULL || ya < N, okb = FULL || yb < N;
    unsigned ah[KT][4], al[KT][4];
#pragma unroll
    for (int kb = 0; kb < KT; ++kb) {
      float xv[4][2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const bool cv = 16 * kb + 8 * hh < W;
          const float* pc = vb + (unsigned)(16 * kb + 2 * t + 8 * hh + e) * P;
          xv[2 * hh][e] = (cv && oka) ? pc[ya] : 0.f;
          xv[2 * hh + 1][e] = (cv && okb) ? pc[yb] : 0.f;
        }
#pragma unroll
      for (int r = 0; r < 4; ++r) split2(xv[r][0], xv[r][1], ah[kb][r], al[kb][r]);
    }
    unsigned th[KS][4], tl[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const uint4* tp = TfA + (((size_t)yt * KS + ks) * 32 + lane) * 2;
      const uint4 h4 = __ldg(tp), l4 = __ldg(tp + 1);
      th[ks][0] = h4.x; th[ks][1] = h4.y; th[ks][2] = h4.z; th[ks][3] = h4.w;
      tl[ks][0] = l4.x; tl[ks][1] = l4.y; tl[ks][2] = l4.z; tl[ks][3] = l4.w;
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kb = 0; kb < KT; ++kb) {
        mma_bf16(acc, ah[kb], wf[kb][nt][0], wf[kb][nt][1]);
        mma_bf16(acc, al[kb], wf[kb][nt][0], wf[kb][nt][1]);
      }
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        mma_bf16(acc, th[ks], sfh[ks][nt][0], sfh[ks][nt][1]);
        mma_bf16(acc, th[ks], sfl[ks][nt][0], sfl[ks][nt][1]);
        mma_bf16(acc, tl[ks], sfh[ks][nt][0], sfh[ks][nt][1]);
      }
      // acc[0], acc[1]: pixel ya, outputs o0, o0 + 1; acc[2], acc[3]: pixel yb
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const unsigned oo = (unsigned)(8 * nt + 2 * t + e) * P;
        const float va = acc[e] + bv[nt][e], vb2 = acc[2 + e] + bv[nt][e];
        if (zb != nullptr) {
          if (oka) zb[oo + ya] = va;
          if (okb) zb[oo + yb] = vb2;
        }
        float wa = va, wb = vb2;
        if (gelu) gelu2(wa, wb);
        if (oka) ub[oo + ya] = wa;
        if (okb) ub[oo + yb] = wb;
      }
    }
  };
  if (N % 16 == 0) {
    for (int yt = yt0; yt < yt1; ++yt) tile(yt, std::true_type{});
  } else {
    for (int yt = yt0; yt < yt1; ++yt) tile(yt, std::false_type{});
  }
}

// 16-byte asynchronous global -> shared copies (L2 only), committed in groups
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// The fused layer for N a multiple of 16, with the activations of the next y-tiles
// copied to shared memory (cp.async, kLayerStages stages per warp: the next tile in
// flight while one is contracted; four stages measured no faster, the kernel being
// bound by its instruction issue): each warp stages its W channels x 16 pixels (W
// 64-byte rows, row stride 20 floats, which makes the fragment reads conflict-free).
// Same arithmetic and order as k_layer_tc.
constexpr int kLayerRow = 20, kLayerStages = 2;
template <int KT, int NT, int KS>
__global__ void __launch_bounds__(128, 4) k_layer_tc_pipe(const float* __restrict__ V, const bf16* __restrict__ Ww,
                                                       const bf16* __restrict__ bias, const float* __restrict__ A,
                                                       const float* __restrict__ cs, const uint4* __restrict__ TfA,
                                                       float* __restrict__ Z, float* __restrict__ Vout, int N, int n2m,
                                                       size_t rows, int tpw, int gelu) {
  constexpr int W = 8 * NT, STAGE = W * kLayerRow, S = kLayerStages;
  __shared__ __align__(16) float sbuf[4][S][STAGE];
  const int lane = threadIdx.x % 32, g = lane / 4, t = lane % 4, wid = threadIdx.x / 32;
  const int YT = N / 16, chunks = (YT + tpw - 1) / tpw;
  const size_t w = (size_t)blockIdx.x * 4 + wid;
  const size_t row = w / chunks;
  if (row >= rows) return;
  const int chunk = (int)(w % chunks);
  const size_t b = row / N;
  const int x = (int)(row % N);
  const unsigned P = (unsigned)N * (unsigned)N;
  unsigned wf[KT][NT][2];
#pragma unroll
  for (int kb = 0; kb < KT; ++kb)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int o = 8 * nt + g;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int c = 16 * kb + 2 * t + 8 * hh;
        const bool cv = 16 * kb + 8 * hh < W;
        const unsigned lo = cv ? (unsigned)__bfloat16_as_ushort(Ww[o * W + c]) : 0u;
        const unsigned hi = cv ? (unsigned)__bfloat16_as_ushort(Ww[o * W + c + 1]) : 0u;
        wf[kb][nt][hh] = lo | (hi << 16);
      }
    }
  unsigned sfh[KS][NT][2], sfl[KS][NT][2];
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int o = 8 * nt + g;
      const float* ar = A + ((b * W + o) * N + x) * n2m;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int k = 16 * ks + 2 * t + 8 * hh;
        const float x0 = k < n2m ? ar[k] * cs[k / 2] : 0.f;
        const float x1 = k + 1 < n2m ? ar[k + 1] * cs[(k + 1) / 2] : 0.f;
        split2(x0, x1, sfh[ks][nt][hh], sfl[ks][nt][hh]);
      }
    }
  float bv[NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) bv[nt][e] = bias != nullptr ? b2f(bias[8 * nt + 2 * t + e]) : 0.f;
  const float* vb = V + b * W * (size_t)P + (size_t)x * N;
  const size_t ob = b * W * (size_t)P + (size_t)x * N;
  float* zb = Z != nullptr ? Z + ob : nullptr;
  float* ub = Vout + ob;
  float(*buf)[STAGE] = sbuf[wid];
  // tile yt -> stage st: W rows of 16 floats, four 16-byte pieces each
  auto prefetch = [&](int yt, int st) {
#pragma unroll
    for (int j = lane; j < 4 * W; j += 32) {
      const int c = j >> 2, part = j & 3;
      cp_async16(&buf[st][c * kLayerRow + 4 * part], vb + (unsigned)c * P + 16 * yt + 4 * part);
    }
    cp_async_commit();
  };
  const int yt0 = chunk * tpw, yt1 = min(YT, yt0 + tpw);
  // one commit group per tile (empty past the chunk's end): before the contraction of
  // tile yt0 + i, S + i groups are committed and waiting until at most S - 1 are
  // pending completes the first i + 1
#pragma unroll
  for (int i = 0; i < S - 1; ++i) {
    if (yt0 + i < yt1) prefetch(yt0 + i, i);
    else cp_async_commit();
  }
  for (int yt = yt0; yt < yt1; ++yt) {
    const int i = yt - yt0;
    if (yt + S - 1 < yt1) prefetch(yt + S - 1, (i + S - 1) % S);
    else cp_async_commit();
    cp_async_wait<S - 1>();
    __syncwarp();
    const float* sb = buf[i % S];
    const int ya = 16 * yt + g, yb = ya + 8;
    unsigned ah[KT][4], al[KT][4];
#pragma unroll
    for (int kb = 0; kb < KT; ++kb) {
      float xv[4][2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const bool cv = 16 * kb + 8 * hh < W;
          const int c = 16 * kb + 2 * t + 8 * hh + e;
          xv[2 * hh][e] = cv ? sb[c * kLayerRow + g] : 0.f;
          xv[2 * hh + 1][e] = cv ? sb[c * kLayerRow + g + 8] : 0.f;
        }
#pragma unroll
      for (int r = 0; r < 4; ++r) split2(xv[r][0], xv[r][1], ah[kb][r], al[kb][r]);
    }
    __syncwarp();   // every lane has read the stage before it is refilled
    unsigned th[KS][4], tl[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const uint4* tp = TfA + (((size_t)yt * KS + ks) * 32 + lane) * 2;
      const uint4 h4 = __ldg(tp), l4 = __ldg(tp + 1);
      th[ks][0] = h4.x; th[ks][1] = h4.y; th[ks][2] = h4.z; th[ks][3] = h4.w;
      tl[ks][0] = l4.x; tl[ks][1] = l4.y; tl[ks][2] = l4.z; tl[ks][3] = l4.w;
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kb = 0; kb < KT; ++kb) {
        mma_bf16(acc, ah[kb], wf[kb][nt][0], wf[kb][nt][1]);
        mma_bf16(acc, al[kb], wf[kb][nt][0], wf[kb][nt][1]);
      }
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        mma_bf16(acc, th[ks], sfh[ks][nt][0], sfh[ks][nt][1]);
        mma_bf16(acc, th[ks], sfl[ks][nt][0], sfl[ks][nt][1]);
        mma_bf16(acc, tl[ks], sfh[ks][nt][0], sfh[ks][nt][1]);
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const unsigned oo = (unsigned)(8 * nt + 2 * t + e) * P;
        const float va = acc[e] + bv[nt][e], vb2 = acc[2 + e] + bv[nt][e];
        if (zb != nullptr) {
          zb[oo + ya] = va;
          zb[oo + yb] = vb2;
        }
        float wa = va, wb = vb2;
        if (gelu) gelu2(wa, wb);
        ub[oo + ya] = wa;
        ub[oo + yb] = wb;
      }
    }
  }
  cp_async_wait<0>();
}

// Fused projection (inference): out[b][p] = q2 + sum_j Q2[j] gelu(q1[j] + sum_c Q1[j][c]
// v[b][c][p]), the hidden layer in registers: the Q1 product as in k_pw_tc, the Q2 dot
// product in float over each lane's outputs and the four lanes of a pixel (shuffles).
// Offsets within one sample are 32-bit (cin N^2 < 2^32).
template <int KT, int NT>
__global__ void __launch_bounds__(128) k_proj_tc(const float* __restrict__ X, int cin, const bf16* __restrict__ Q1,
                                                 const bf16* __restrict__ q1, const bf16* __restrict__ Q2,
                                                 const bf16* __restrict__ q2, int H, float* __restrict__ out, unsigned P,
                                                 int tpw) {
  const int lane = threadIdx.x % 32, g = lane / 4, t = lane % 4;
  const int b = blockIdx.y;
  const unsigned tiles = (P + 15) / 16;
  const size_t tile0 = ((size_t)blockIdx.x * 4 + threadIdx.x / 32) * tpw;
  if (tile0 >= tiles) return;
  unsigned wf[KT][NT][2];
#pragma unroll
  for (int kb = 0; kb < KT; ++kb)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int j = 8 * nt + g;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int c = 16 * kb + 2 * t + 8 * hh;
        const unsigned lo = (j < H && c < cin) ? (unsigned)__bfloat16_as_ushort(Q1[j * cin + c]) : 0u;
        const unsigned hi = (j < H && c + 1 < cin) ? (unsigned)__bfloat16_as_ushort(Q1[j * cin + c + 1]) : 0u;
        wf[kb][nt][hh] = lo | (hi << 16);
      }
    }
  float qb[NT][2], qw[NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = 8 * nt + 2 * t + e;
      qb[nt][e] = j < H ? b2f(q1[j]) : 0.f;
      qw[nt][e] = j < H ? b2f(Q2[j]) : 0.f;
    }
  const float bias2 = b2f(q2[0]);
  const float* xb = X + (size_t)b * cin * P;
  float* ob = out + (size_t)b * P;
  const unsigned t1 = (unsigned)min((size_t)tiles, tile0 + tpw);
  auto tile = [&](unsigned tl, auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
    const unsigned pa = tl * 16 + g, pb = pa + 8;
    const bool oka = FULL || pa < P, okb = FULL || pb < P;
    unsigned ah[KT][4], al[KT][4];
#pragma unroll
    for (int kb = 0; kb < KT; ++kb) {
      float xv[4][2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c = 16 * kb + 2 * t + 8 * hh + e;
          const float* pc = xb + (unsigned)c * P;
          xv[2 * hh][e] = (c < cin && oka) ? pc[pa] : 0.f;
          xv[2 * hh + 1][e] = (c < cin && okb) ? pc[pb] : 0.f;
        }
#pragma unroll
      for (int r = 0; r < 4; ++r) split2(xv[r][0], xv[r][1], ah[kb][r], al[kb][r]);
    }
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kb = 0; kb < KT; ++kb) {
        mma_bf16(acc, ah[kb], wf[kb][nt][0], wf[kb][nt][1]);
        mma_bf16(acc, al[kb], wf[kb][nt][0], wf[kb][nt][1]);
      }
      float h0 = acc[0] + qb[nt][0], h1 = acc[1] + qb[nt][1], h2 = acc[2] + qb[nt][0], h3 = acc[3] + qb[nt][1];
      gelu2(h0, h1);
      gelu2(h2, h3);
      sa += qw[nt][0] * h0 + qw[nt][1] * h1;
      sb += qw[nt][0] * h2 + qw[nt][1] * h3;
    }
    sa += __shfl_xor_sync(0xffffffffu, sa, 1);
    sa += __shfl_xor_sync(0xffffffffu, sa, 2);
    sb += __shfl_xor_sync(0xffffffffu, sb, 1);
    sb += __shfl_xor_sync(0xffffffffu, sb, 2);
    if (t == 0) {
      if (oka) ob[pa] = sa + bias2;
      if (okb) ob[pb] = sb + bias2;
    }
  };
  if (P % 16 == 0) {
    for (unsigned tl = (unsigned)tile0; tl < t1; ++tl) tile(tl, std::true_type{});
  } else {
    for (unsigned tl = (unsigned)tile0; tl < t1; ++tl) tile(tl, std::false_type{});
  }
}

// c_k / N^2, the weights of the gradient of the inverse transform, for the current N
__global__ void k_cky_scaled(const float* __restrict__ c, float* __restrict__ cs, int m, float inv) {
  FOR_N(k, (size_t)m) cs[k] = c[k] * inv;
}

constexpr int G1_BM = 128, G1_BN = 32, G1_BK = 32;   // forward: 256 threads, 4 x 4 outputs each
// C[r][j] = sum_y V[r][y] Tf[y][j] for rows r < rows, j < n2m (= 2m)
__global__ void __launch_bounds__(256) k_dft_y_gemm(const float* __restrict__ V, const float* __restrict__ Tf,
                                                    float* __restrict__ C, size_t rows, int N, int n2m) {
  __shared__ __align__(16) float Vs[G1_BK][G1_BM + 4];
  __shared__ __align__(16) float Ts[G1_BK][G1_BN];
  const int tid = threadIdx.x;
  const size_t r0 = (size_t)blockIdx.x * G1_BM;
  const int c0 = blockIdx.y * G1_BN;
  const int tr = (tid / 8) * 4, tc = (tid % 8) * 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < N; k0 += G1_BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {   // V tile, 128 rows x 32 k, stored k-major
      const int f = tid + 256 * q, row = f / 8, kq = (f % 8) * 4;
      const size_t r = r0 + row;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = k0 + kq + e;
        Vs[kq + e][row] = (r < rows && k < N) ? V[r * N + k] : 0.f;
      }
    }
    {   // Tf tile, 32 k x 32 columns
      const int k = tid / 8, cq = (tid % 8) * 4;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = c0 + cq + e;
        Ts[k][cq + e] = (k0 + k < N && col < n2m) ? Tf[(size_t)(k0 + k) * n2m + col] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < G1_BK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&Vs[kk][tr]);
      const float4 b = *reinterpret_cast<const float4*>(&Ts[kk][tc]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const size_t r = r0 + tr + i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + tc + j;
      if (col < n2m) C[r * n2m + col] = acc[i][j];
    }
  }
}

constexpr int G2_BM = 64, G2_BN = 128, G2_BK = 32;   // inverse: 256 threads, 4 x 8 outputs each
// out[r][y] (+)= sum_k A[r][k] cs(k) Ti[k][y], k < n2m, cs(k) = scale * (c ? c[k/2] : 1)
template <bool ACCUM>
__global__ void __launch_bounds__(256) k_idft_y_gemm(const float* __restrict__ A, const float* __restrict__ Ti,
                                                     const float* __restrict__ c, float scale,
                                                     float* __restrict__ out, size_t rows, int N, int n2m) {
  __shared__ float As[G2_BK][G2_BM + 1];
  __shared__ __align__(16) float Us[G2_BK][G2_BN];
  const int tid = threadIdx.x;
  const size_t r0 = (size_t)blockIdx.x * G2_BM;
  const int c0 = blockIdx.y * G2_BN;
  const int tr = (tid / 16) * 4, tc = (tid % 16) * 8;
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < n2m; k0 += G2_BK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {   // A tile, 64 rows x 32 k (scaled), stored k-major
      const int f = tid + 256 * q, row = f / 32, k = f % 32;
      const size_t r = r0 + row;
      const int kg = k0 + k;
      float val = 0.f;
      if (r < rows && kg < n2m) val = A[r * n2m + kg] * (scale * (c != nullptr ? c[kg / 2] : 1.f));
      As[k][row] = val;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {  // Ti tile, 32 k x 128 y
      const int f = tid + 256 * q, k = f / 128, cc = f % 128;
      const int y = c0 + cc;
      Us[k][cc] = (k0 + k < n2m && y < N) ? Ti[(size_t)(k0 + k) * N + y] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < G2_BK; ++kk) {
      float av[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tr + i];
      const float4 b0 = *reinterpret_cast<const float4*>(&Us[kk][tc]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Us[kk][tc + 4]);
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const size_t r = r0 + tr + i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int y = c0 + tc + j;
      if (y < N) {
        float* o = out + r * N + y;
        if (ACCUM) *o += acc[i][j];
        else *o = acc[i][j];
      }
    }
  }
}

// Xh[q][kxi][ky] = s[ky] sum_x A[q][x][ky] e^{-2 pi i kx x/N}: block (q, kxi); thread
// (slice, ky) adds every S-th x from its slice, then the slices are added in order
__global__ void __launch_bounds__(256) k_dft_x_par(const float2* __restrict__ A, float2* __restrict__ Xh,
                                                   const float2* __restrict__ tw, const float* __restrict__ wky,
                                                   int N, int m) {
  __shared__ float2 red[256];
  const size_t q = blockIdx.x;
  const int kxi = blockIdx.y;
  const int kx = kx_of(kxi, m, N);
  const int S = 256 / m;
  const int ky = threadIdx.x % m, slice = threadIdx.x / m;
  float re = 0.f, im = 0.f;
  if (slice < S) {
    const float2* a = A + q * (size_t)N * m + ky;
    // twiddle index kx x mod N, stepped by kx S mod N
    int idx = (int)(((long long)kx * slice) % N);
    const int step = (int)(((long long)kx * S) % N);
    for (int x = slice; x < N; x += S) {
      const float2 w = tw[idx];
      const float2 v = a[(size_t)x * m];
      re += v.x * w.x - v.y * w.y;
      im += v.x * w.y + v.y * w.x;
      idx += step;
      if (idx >= N) idx -= N;
    }
  }
  red[threadIdx.x] = make_float2(re, im);
  __syncthreads();
  if (threadIdx.x < m) {
    float2 t = red[threadIdx.x];
    for (int sl = 1; sl < S; ++sl) {
      const float2 u = red[sl * m + threadIdx.x];
      t.x += u.x;
      t.y += u.y;
    }
    const float sc = wky != nullptr ? wky[threadIdx.x] : 1.f;
    Xh[(q * 2 * m + kxi) * m + threadIdx.x] = make_float2(t.x * sc, t.y * sc);
  }
}

// Y[b][o][mode] = sum_i X[b][i][mode] R[i][o][mode]
__global__ void k_mix(const float2* __restrict__ X, const bf16* __restrict__ Rre, const bf16* __restrict__ Rim,
                      float2* __restrict__ Y, int W, int nm, int B) {
  FOR_N(e, (size_t)B * W * nm) {
    const int mode = (int)(e % nm);
    const int o = (int)((e / nm) % W);
    const int b = (int)(e / ((size_t)nm * W));
    float re = 0.f, im = 0.f;
    for (int i = 0; i < W; ++i) {
      const float2 x = X[((size_t)b * W + i) * nm + mode];
      const size_t r = ((size_t)i * W + o) * nm + mode;
      const float rr = b2f(Rre[r]), ri = b2f(Rim[r]);
      re += x.x * rr - x.y * ri;
      im += x.x * ri + x.y * rr;
    }
    Y[e] = make_float2(re, im);
  }
}

// dR[i][o][mode] = sum_b conj(X[b][i][mode]) dY[b][o][mode]
__global__ void k_mix_wgrad(const float2* __restrict__ X, const float2* __restrict__ dY, float* __restrict__ gre,
                            float* __restrict__ gim, int W, int nm, int B) {
  FOR_N(e, (size_t)W * W * nm) {
    const int mode = (int)(e % nm);
    const int o = (int)((e / nm) % W);
    const int i = (int)(e / ((size_t)nm * W));
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; ++b) {
      const float2 x = X[((size_t)b * W + i) * nm + mode];
      const float2 d = dY[((size_t)b * W + o) * nm + mode];
      re += x.x * d.x + x.y * d.y;
      im += x.x * d.y - x.y * d.x;
    }
    gre[e] = re;
    gim[e] = im;
  }
}

// dX[b][i][mode] = sum_o conj(R[i][o][mode]) dY[b][o][mode]
__global__ void k_mix_dgrad(const float2* __restrict__ dY, const bf16* __restrict__ Rre, const bf16* __restrict__ Rim,
                            float2* __restrict__ dX, int W, int nm, int B) {
  FOR_N(e, (size_t)B * W * nm) {
    const int mode = (int)(e % nm);
    const int i = (int)((e / nm) % W);
    const int b = (int)(e / ((size_t)nm * W));
    float re = 0.f, im = 0.f;
    for (int o = 0; o < W; ++o) {
      const float2 d = dY[((size_t)b * W + o) * nm + mode];
      const size_t r = ((size_t)i * W + o) * nm + mode;
      const float rr = b2f(Rre[r]), ri = b2f(Rim[r]);
      re += rr * d.x + ri * d.y;
      im += rr * d.y - ri * d.x;
    }
    dX[e] = make_float2(re, im);
  }
}

// loss = mean (out - t)^2 (block partials), d_out = 2 (out - t) / n
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ t, float* __restrict__ dout,
                      double* __restrict__ part, size_t n) {
  double s = 0.0;
  FOR_N(i, n) {
    const float d = out[i] - t[i];
    dout[i] = 2.f * d / (float)n;
    s += (double)d * d;
  }
  __shared__ double sh[FT];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = FT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, bf16* __restrict__ wb, size_t n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
  FOR_N(i, n) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float wn = w[i] - lr * (a * c1) / (sqrtf(v * c2) + eps);
    w[i] = wn;
    wb[i] = __float2bfloat16(wn);
  }
}

__global__ void k_to_bf16(const float* __restrict__ w, bf16* __restrict__ wb, size_t n) {
  FOR_N(i, n) wb[i] = __float2bfloat16(w[i]);
}

__global__ void k_bf16_to_f32(const bf16* __restrict__ wb, float* __restrict__ w, size_t n) {
  FOR_N(i, n) w[i] = b2f(wb[i]);
}

// p_init[b][p] = pbar[b] * max(out[b][p], 0)
__global__ void k_fno_pressure(const float* __restrict__ out, const double* __restrict__ pbar, float q_min,
                               float* __restrict__ p, size_t P, int B) {
  FOR_N(i, (size_t)B * P) {
    const float q = out[i];
    p[i] = q > q_min ? (float)pbar[i / P] * q : 0.f;
  }
}

// q[b][p] = p[b][p] / pbar[b]  (training targets)
__global__ void k_fno_target(const float* __restrict__ p, const double* __restrict__ pbar, float* __restrict__ q,
                             size_t P, int B) {
  FOR_N(i, (size_t)B * P) q[i] = (float)((double)p[i] / pbar[i / P]);
}

__global__ void k_twiddle_f(float2* __restrict__ tw, int N) {
  FOR_N(k, (size_t)N) {
    double s, c;
    sincospi(2.0 * (double)k / (double)N, &s, &c);
    tw[k] = make_float2((float)c, (float)(-s));
  }
}

}  // namespace
}  // namespace bem

// ===========================================================================
using namespace bem;

struct bem_fno_s {
  bem_fno_desc d;
  int dev = 0;
  size_t o_Pw, o_Pb, o_Rre, o_Rim, o_Ww, o_Wb, o_Q1w, o_Q1b, o_Q2w, o_Q2b, P;
  float* w = nullptr;       // master weights
  bf16* wb = nullptr;       // bf16 copy used by the kernels
  float* g = nullptr;       // gradients
  float* m1 = nullptr;
  float* m2 = nullptr;
  int step = 0;
  // activations and scratch, sized for (B, N) of the largest call so far
  int capB = 0, capN = 0, twN = 0;
  bool cap_train = false;
  std::vector<float*> v, z;
  std::vector<float2*> Xh;
  float *a = nullptr, *h = nullptr, *out = nullptr, *dout = nullptr;
  float *dv = nullptr, *dz = nullptr, *dt = nullptr, *mom = nullptr, *part = nullptr, *cky = nullptr, *cky_s = nullptr;
  double* mom_part = nullptr;   // per-chunk sums of the height moments
  float2 *A = nullptr, *Y = nullptr, *dY = nullptr, *tw = nullptr;
  float *Tf = nullptr, *Ti = nullptr;   // twiddle matrices of the y transforms (N x 2m, 2m x N)
  uint4 *TfB = nullptr, *TiB = nullptr; // the same split into bf16 hi/lo, in mma fragment order
  uint4* TfA = nullptr;                 // Tf split, in A-fragment order (fused layer kernel)
  double* lpart = nullptr;
  std::vector<void*> owned;
  size_t n_persistent = 0;   // leading entries of owned that live as long as the handle
};

namespace {

template <typename P>
cudaError_t alloc(bem_fno_s* f, P** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(P));
  if (e == cudaSuccess) f->owned.push_back(*p);
  return e;
}

// the tensor-core y transforms hold up to 8 n-tiles of 2m columns (m <= 32)
bool tc_ok(const bem_fno_s* f) { return 2 * f->d.modes <= 8 * TC_NT_MAX; }
// the fused layer kernel: width 8, 16 or 32 (its register tiles), the same modes
bool fused_ok(const bem_fno_s* f) {
  const int W = f->d.width;
  return tc_ok(f) && (W == 8 || W == 16 || W == 32);
}
// the fused projection: input width <= 32, hidden width <= 64
bool proj_ok(const bem_fno_s* f) { return f->d.width <= 32 && f->d.hidden <= 64; }

constexpr int kMaxSamples = 4096;
// frees the activation buffers: everything allocated after the handle's persistent
// buffers (parameters, optimiser state, moments), whose count is recorded at creation
void free_acts(bem_fno_s* f) {
  for (size_t i = f->n_persistent; i < f->owned.size(); ++i) cudaFree(f->owned[i]);
  f->owned.resize(std::min<size_t>(f->owned.size(), f->n_persistent));
  f->v.clear();
  f->z.clear();
  f->Xh.clear();
  f->capB = f->capN = f->twN = 0;
}

// twiddles, the y-transform matrices and the gradient weights c_k / N^2 for grid N
void set_twiddles(bem_fno_s* f, int N, cudaStream_t s) {
  const int m = f->d.modes;
  k_twiddle_f<<<blocks_for(N), FT, 0, s>>>(f->tw, N);
  k_twiddle_mats<<<blocks_for((size_t)N * m), FT, 0, s>>>(f->tw, f->Tf, f->Ti, N, m);
  k_cky_scaled<<<1, 32, 0, s>>>(f->cky, f->cky_s, m, (float)(1.0 / ((double)N * N)));
  note_launches(3);
  if (tc_ok(f)) {
    const int n2m = 2 * m;
    // forward B = Tf (K = N, columns n2m), inverse B = Ti (K = n2m, columns N)
    k_frag_b<<<blocks_for((size_t)((N + 15) / 16) * ((n2m + 7) / 8) * 32), FT, 0, s>>>(f->Tf, N, n2m, n2m, 1, f->TfB);
    k_frag_b<<<blocks_for((size_t)((n2m + 15) / 16) * ((N + 7) / 8) * 32), FT, 0, s>>>(f->Ti, n2m, N, N, 1, f->TiB);
    note_launches(2);
  }
  if (fused_ok(f)) {
    const int n2m = 2 * m;
    k_frag_a<<<blocks_for((size_t)((N + 15) / 16) * ((n2m + 15) / 16) * 32), FT, 0, s>>>(f->Tf, N, n2m, n2m, f->TfA);
    note_launches(1);
  }
  f->twN = N;
}

bem_status ensure(bem_fno_s* f, int B, int N, bool train, cudaStream_t s) {
  if (B <= f->capB && N <= f->capN && (!train || f->cap_train)) {
    if (f->twN != N) set_twiddles(f, N, s);
    return BEM_OK;
  }
  free_acts(f);
  const int W = f->d.width, m = f->d.modes, L = f->d.layers, H = f->d.hidden;
  const size_t P = (size_t)N * N;
  const size_t nm = 2 * (size_t)m * m;
  const int nv = train ? L + 1 : 2, nz = train ? L : 1;
  cudaError_t e = cudaSuccess;
  f->v.resize(nv);
  f->z.resize(nz);
  f->Xh.resize(train ? L : 1);
  for (int i = 0; i < nv && e == cudaSuccess; ++i) e = alloc(f, &f->v[i], (size_t)B * W * P);
  for (int i = 0; i < nz && e == cudaSuccess; ++i) e = alloc(f, &f->z[i], (size_t)B * W * P);
  for (size_t i = 0; i < f->Xh.size() && e == cudaSuccess; ++i) e = alloc(f, &f->Xh[i], (size_t)B * W * nm);
  if (e == cudaSuccess) e = alloc(f, &f->a, (size_t)B * H * P);
  if (e == cudaSuccess) e = alloc(f, &f->h, (size_t)B * H * P);
  if (e == cudaSuccess) e = alloc(f, &f->out, (size_t)B * P);
  if (e == cudaSuccess) e = alloc(f, &f->dout, (size_t)B * P);
  const size_t big = (size_t)B * std::max(W, H) * P;
  if (e == cudaSuccess && train) e = alloc(f, &f->dv, big);
  if (e == cudaSuccess && train) e = alloc(f, &f->dz, big);
  if (e == cudaSuccess && train) e = alloc(f, &f->dt, big);
  if (e == cudaSuccess) e = alloc(f, &f->A, (size_t)B * W * N * m);
  if (e == cudaSuccess) e = alloc(f, &f->Y, (size_t)B * W * nm);
  if (e == cudaSuccess) e = alloc(f, &f->dY, (size_t)B * W * nm);
  if (e == cudaSuccess) e = alloc(f, &f->tw, (size_t)N);
  if (e == cudaSuccess) e = alloc(f, &f->Tf, (size_t)2 * m * N);
  if (e == cudaSuccess) e = alloc(f, &f->Ti, (size_t)2 * m * N);
  if (e == cudaSuccess && tc_ok(f))
    e = alloc(f, &f->TfB, (size_t)((N + 15) / 16) * ((2 * m + 7) / 8) * 32);
  if (e == cudaSuccess && tc_ok(f))
    e = alloc(f, &f->TiB, (size_t)((2 * m + 15) / 16) * ((N + 7) / 8) * 32);
  if (e == cudaSuccess && fused_ok(f))
    e = alloc(f, &f->TfA, (size_t)((N + 15) / 16) * ((2 * m + 15) / 16) * 64);
  const size_t nblk = (size_t)B * ((P + FT - 1) / FT);
  const size_t maxout = (size_t)std::max(W, H) * std::max({W, H, 7}) + std::max(W, H);
  if (e == cudaSuccess && train) e = alloc(f, &f->part, nblk * maxout);
  if (e == cudaSuccess) e = alloc(f, &f->lpart, (size_t)4096);
  if (e == cudaSuccess) e = alloc(f, &f->cky, (size_t)m);
  if (e == cudaSuccess) e = alloc(f, &f->cky_s, (size_t)m);
  if (e != cudaSuccess) {
    free_acts(f);
    return cuda_fail(e, "cudaMalloc(fno activations)");
  }
  f->capB = B;
  f->capN = N;
  f->cap_train = train;
  std::vector<float> c(m);
  for (int k = 0; k < m; ++k) c[k] = k == 0 ? 1.f : 2.f;
  BEM_CUDA_TRY(cudaMemcpyAsync(f->cky, c.data(), m * sizeof(float), cudaMemcpyHostToDevice, s));
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  set_twiddles(f, N, s);
  return BEM_OK;
}

// pointwise layer dispatch on the (compile-time) input width
template <int KT, int NT, bool TRANS, bool ACCUM, bool GELU>
void pw_tc_launch(const float* X, int cin, const bf16* Wt, const bf16* bias, float* Y, float* Yact, int cout,
                  size_t P, int B, cudaStream_t s) {
  const size_t warps = ((P + 15) / 16 + kPwTiles - 1) / kPwTiles;
  const dim3 grid((unsigned)((warps + 3) / 4), B);
  k_pw_tc<KT, NT, TRANS, ACCUM, GELU><<<grid, 128, 0, s>>>(X, cin, Wt, bias, Y, Yact, cout, P);
}

template <int KT, bool TRANS, bool ACCUM, bool GELU>
void pw_tc_nt(const float* X, int cin, const bf16* Wt, const bf16* bias, float* Y, float* Yact, int cout, size_t P,
              int B, cudaStream_t s) {
  switch ((cout + 7) / 8) {
    case 1: pw_tc_launch<KT, 1, TRANS, ACCUM, GELU>(X, cin, Wt, bias, Y, Yact, cout, P, B, s); break;
    case 2: pw_tc_launch<KT, 2, TRANS, ACCUM, GELU>(X, cin, Wt, bias, Y, Yact, cout, P, B, s); break;
    case 4: pw_tc_launch<KT, 4, TRANS, ACCUM, GELU>(X, cin, Wt, bias, Y, Yact, cout, P, B, s); break;
    default: pw_tc_launch<KT, 8, TRANS, ACCUM, GELU>(X, cin, Wt, bias, Y, Yact, cout, P, B, s); break;
  }
}

template <bool TRANS, bool ACCUM, bool GELU>
void pw(const float* X, int cin, const bf16* Wt, const bf16* bias, float* Y, float* Yact, int cout, size_t P, int B,
        cudaStream_t s) {
  // the tensor-core form wherever a contraction has something to contract (cin >= 7)
  if (cin >= 7 && cout <= 64) {
    if (cin <= 16) pw_tc_nt<1, TRANS, ACCUM, GELU>(X, cin, Wt, bias, Y, Yact, cout, P, B, s);
    else if (cin <= 32) pw_tc_nt<2, TRANS, ACCUM, GELU>(X, cin, Wt, bias, Y, Yact, cout, P, B, s);
    else pw_tc_nt<4, TRANS, ACCUM, GELU>(X, cin, Wt, bias, Y, Yact, cout, P, B, s);
    note_launches(1);
    return;
  }
  dim3 grid((unsigned)((P + FT - 1) / FT), B);
  const size_t sm = (size_t)cout * cin * sizeof(float);
  switch (cin) {
    case 1: k_pw<1, TRANS, ACCUM, GELU><<<grid, FT, sm, s>>>(X, Wt, bias, Y, Yact, cout, P); break;
    case 7: k_pw<7, TRANS, ACCUM, GELU><<<grid, FT, sm, s>>>(X, Wt, bias, Y, Yact, cout, P); break;
    case 8: k_pw<8, TRANS, ACCUM, GELU><<<grid, FT, sm, s>>>(X, Wt, bias, Y, Yact, cout, P); break;
    case 16: k_pw<16, TRANS, ACCUM, GELU><<<grid, FT, sm, s>>>(X, Wt, bias, Y, Yact, cout, P); break;
    case 32: k_pw<32, TRANS, ACCUM, GELU><<<grid, FT, sm, s>>>(X, Wt, bias, Y, Yact, cout, P); break;
    case 64: k_pw<64, TRANS, ACCUM, GELU><<<grid, FT, sm, s>>>(X, Wt, bias, Y, Yact, cout, P); break;
    default: break;
  }
  note_launches(1);
}

bool width_ok(int c) { return c == 1 || c == 7 || c == 8 || c == 16 || c == 32 || c == 64; }

void wgrad(const float* dY, int cout, const float* X, int cin, float* gw, float* gb, float* part, size_t P, int B,
           cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr)) cudaFuncSetAttribute(k_pw_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  dim3 grid((unsigned)((P + FT - 1) / FT), B);
  const size_t sm = (size_t)(cout + cin) * FT * sizeof(float);
  k_pw_wgrad<<<grid, FT, sm, s>>>(dY, X, part, cout, cin, P);
  const int nblk = (int)(grid.x * grid.y);
  k_pw_wgrad_sum<<<blocks_for((size_t)cout * cin + cout), FT, 0, s>>>(part, nblk, cout, cin, gw, gb);
  note_launches(2);
}

// spectral branch: out (=|+=) idft( R * dft(vin) ), caching dft(vin) in Xh
// A (rows x m complex) = truncated DFT along y of the rows of v
void dft_y(bem_fno_s* f, const float* v, size_t rows, int N, cudaStream_t s) {
  const int n2m = 2 * f->d.modes;
  if (tc_ok(f)) {
    const unsigned grid = (unsigned)((rows + 127) / 128);
    float* C = reinterpret_cast<float*>(f->A);
    switch ((n2m + 7) / 8) {
      case 1: k_dft_y_tc<1><<<grid, 128, 0, s>>>(v, f->TfB, C, rows, N, n2m); break;
      case 2: k_dft_y_tc<2><<<grid, 128, 0, s>>>(v, f->TfB, C, rows, N, n2m); break;
      case 3: k_dft_y_tc<3><<<grid, 128, 0, s>>>(v, f->TfB, C, rows, N, n2m); break;
      case 4: k_dft_y_tc<4><<<grid, 128, 0, s>>>(v, f->TfB, C, rows, N, n2m); break;
      case 5: k_dft_y_tc<5><<<grid, 128, 0, s>>>(v, f->TfB, C, rows, N, n2m); break;
      case 6: k_dft_y_tc<6><<<grid, 128, 0, s>>>(v, f->TfB, C, rows, N, n2m); break;
      case 7: k_dft_y_tc<7><<<grid, 128, 0, s>>>(v, f->TfB, C, rows, N, n2m); break;
      default: k_dft_y_tc<8><<<grid, 128, 0, s>>>(v, f->TfB, C, rows, N, n2m); break;
    }
    return;
  }
  const dim3 grid((unsigned)((rows + G1_BM - 1) / G1_BM), (unsigned)((n2m + G1_BN - 1) / G1_BN));
  k_dft_y_gemm<<<grid, 256, 0, s>>>(v, f->Tf, reinterpret_cast<float*>(f->A), rows, N, n2m);
}

// out (rows x N) (+)= inverse truncated transform along y of A with weights c, scale
template <bool ACCUM>
void idft_y(bem_fno_s* f, float* out, const float* c, float scale, size_t rows, int N, cudaStream_t s) {
  const int n2m = 2 * f->d.modes;
  if (tc_ok(f)) {
    const dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((N + TC_IY - 1) / TC_IY));
    k_idft_y_tc<ACCUM><<<grid, 128, 0, s>>>(reinterpret_cast<const float*>(f->A), f->TiB, c, scale, out, rows, N, n2m);
    return;
  }
  const dim3 grid((unsigned)((rows + G2_BM - 1) / G2_BM), (unsigned)((N + G2_BN - 1) / G2_BN));
  k_idft_y_gemm<ACCUM><<<grid, 256, 0, s>>>(reinterpret_cast<const float*>(f->A), f->Ti, c, scale, out, rows, N,
                                            n2m);
}

// spectral branch up to the inverse along x: A[(b, o, x)][2m] holds the mixed modes
// of every row, caching dft(vin) in Xh
void spectral_modes(bem_fno_s* f, int l, const float* vin, float2* Xh, int B, int N, cudaStream_t s) {
  const int W = f->d.width, m = f->d.modes;
  const size_t bc = (size_t)B * W, nm = 2 * (size_t)m * m;
  dft_y(f, vin, bc * N, N, s);
  k_dft_x_par<<<dim3((unsigned)bc, 2 * m), 256, 0, s>>>(f->A, Xh, f->tw, nullptr, N, m);
  const bf16* Rre = f->wb + f->o_Rre + (size_t)l * W * W * nm;
  const bf16* Rim = f->wb + f->o_Rim + (size_t)l * W * W * nm;
  k_mix<<<blocks_for(bc * nm), FT, 0, s>>>(Xh, Rre, Rim, f->Y, W, (int)nm, B);
  k_idft_x<<<blocks_for(bc * N * ((m + 3) / 4)), FT, 0, s>>>(f->Y, f->A, f->tw, N, m, bc);
  note_launches(4);
}

void spectral_fwd(bem_fno_s* f, int l, const float* vin, float2* Xh, float* out, int B, int N, cudaStream_t s) {
  spectral_modes(f, l, vin, Xh, B, N, s);
  idft_y<false>(f, out, f->cky, 1.f / ((float)N * N), (size_t)B * f->d.width * N, N, s);
  note_launches(1);
}

template <int KT, int NT, int KS>
void layer_launch(bem_fno_s* f, const float* vin, const bf16* Ww, const bf16* Wb, float* z, float* vout, bool gelu,
                  int B, int N, cudaStream_t s) {
  const int YT = (N + 15) / 16, tpw = std::min(YT, 32), chunks = (YT + tpw - 1) / tpw;
  const size_t rows = (size_t)B * N, warps = rows * chunks;
  if (N % 16 == 0) {   // whole 16-pixel tiles, 16-byte aligned rows: the staged form
    k_layer_tc_pipe<KT, NT, KS><<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(
        vin, Ww, Wb, reinterpret_cast<const float*>(f->A), f->cky_s, f->TfA, z, vout, N, 2 * f->d.modes, rows, tpw,
        gelu ? 1 : 0);
    return;
  }
  k_layer_tc<KT, NT, KS><<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(
      vin, Ww, Wb, reinterpret_cast<const float*>(f->A), f->cky_s, f->TfA, z, vout, N, 2 * f->d.modes, rows, tpw,
      gelu ? 1 : 0);
}

template <int KT, int NT>
void layer_ks(bem_fno_s* f, const float* vin, const bf16* Ww, const bf16* Wb, float* z, float* vout, bool gelu, int B,
              int N, cudaStream_t s) {
  switch ((2 * f->d.modes + 15) / 16) {
    case 1: layer_launch<KT, NT, 1>(f, vin, Ww, Wb, z, vout, gelu, B, N, s); break;
    case 2: layer_launch<KT, NT, 2>(f, vin, Ww, Wb, z, vout, gelu, B, N, s); break;
    case 3: layer_launch<KT, NT, 3>(f, vin, Ww, Wb, z, vout, gelu, B, N, s); break;
    default: layer_launch<KT, NT, 4>(f, vin, Ww, Wb, z, vout, gelu, B, N, s); break;
  }
}

// z = W vin + b + S(vin) (stored when z is given), vout = gelu(z) or z, in one pass
// over the pixels after the spectral branch's mode work (fused_ok)
void layer_fused(bem_fno_s* f, int l, const float* vin, float2* Xh, float* z, float* vout, bool gelu, int B, int N,
                 cudaStream_t s) {
  const int W = f->d.width;
  spectral_modes(f, l, vin, Xh, B, N, s);
  const bf16* Ww = f->wb + f->o_Ww + (size_t)l * W * W;
  const bf16* Wb = f->wb + f->o_Wb + (size_t)l * W;
  if (W == 8) layer_ks<1, 1>(f, vin, Ww, Wb, z, vout, gelu, B, N, s);
  else if (W == 16) layer_ks<1, 2>(f, vin, Ww, Wb, z, vout, gelu, B, N, s);
  else layer_ks<2, 4>(f, vin, Ww, Wb, z, vout, gelu, B, N, s);
  note_launches(1);
}

template <int KT, int NT>
void proj_launch(bem_fno_s* f, const float* v, int B, int N, cudaStream_t s) {
  const size_t P = (size_t)N * N, tiles = (P + 15) / 16;
  const int tpw = 8;
  const size_t warps = (tiles + tpw - 1) / tpw;
  k_proj_tc<KT, NT><<<dim3((unsigned)((warps + 3) / 4), B), 128, 0, s>>>(
      v, f->d.width, f->wb + f->o_Q1w, f->wb + f->o_Q1b, f->wb + f->o_Q2w, f->wb + f->o_Q2b, f->d.hidden, f->out,
      (unsigned)P, tpw);
}

template <int KT>
void proj_nt(bem_fno_s* f, const float* v, int B, int N, cudaStream_t s) {
  const int nt = (f->d.hidden + 7) / 8;
  if (nt <= 1) proj_launch<KT, 1>(f, v, B, N, s);
  else if (nt <= 2) proj_launch<KT, 2>(f, v, B, N, s);
  else if (nt <= 4) proj_launch<KT, 4>(f, v, B, N, s);
  else proj_launch<KT, 8>(f, v, B, N, s);
}

// out = Q2 gelu(Q1 v + q1) + q2 without storing the hidden layer (inference, proj_ok)
void proj_fused(bem_fno_s* f, const float* v, int B, int N, cudaStream_t s) {
  if (f->d.width <= 16) proj_nt<1>(f, v, B, N, s);
  else proj_nt<2>(f, v, B, N, s);
  note_launches(1);
}

bem_status forward(bem_fno_s* f, int B, int N, const float* x, bool train, cudaStream_t s) {
  const int W = f->d.width, L = f->d.layers, H = f->d.hidden;
  const size_t P = (size_t)N * N;
  pw<false, false, false>(x, 7, f->wb + f->o_Pw, f->wb + f->o_Pb, f->v[0], nullptr, W, P, B, s);
  for (int l = 0; l < L; ++l) {
    float* vin = train ? f->v[l] : f->v[l & 1];
    float* z = train ? f->z[l] : f->z[0];
    float2* Xh = train ? f->Xh[l] : f->Xh[0];
    float* vout = train ? f->v[l + 1] : f->v[(l + 1) & 1];
    if (fused_ok(f) && (size_t)W * P < (size_t(1) << 32)) {   // 32-bit offsets within a sample
      // z is kept only for the backward pass
      layer_fused(f, l, vin, Xh, train ? z : nullptr, vout, l < L - 1, B, N, s);
      continue;
    }
    spectral_fwd(f, l, vin, Xh, z, B, N, s);
    const bf16* Ww = f->wb + f->o_Ww + (size_t)l * W * W;
    const bf16* Wb = f->wb + f->o_Wb + (size_t)l * W;
    if (l < L - 1) {
      pw<false, true, true>(vin, W, Ww, Wb, z, vout, W, P, B, s);
    } else {
      pw<false, true, false>(vin, W, Ww, Wb, z, nullptr, W, P, B, s);
      BEM_CUDA_TRY(cudaMemcpyAsync(vout, z, (size_t)B * W * P * sizeof(float), cudaMemcpyDeviceToDevice, s));
    }
  }
  float* vL = train ? f->v[L] : f->v[L & 1];
  if (!train && proj_ok(f) && (size_t)W * P < (size_t(1) << 32)) {
    proj_fused(f, vL, B, N, s);
  } else {
    pw<false, false, true>(vL, W, f->wb + f->o_Q1w, f->wb + f->o_Q1b, f->a, f->h, H, P, B, s);
    pw<false, false, false>(f->h, H, f->wb + f->o_Q2w, f->wb + f->o_Q2b, f->out, nullptr, 1, P, B, s);
  }
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

bem_status backward(bem_fno_s* f, int B, int N, const float* x, const float* target, double* loss, cudaStream_t s) {
  const int W = f->d.width, m = f->d.modes, L = f->d.layers, H = f->d.hidden;
  const size_t P = (size_t)N * N, nm = 2 * (size_t)m * m, bc = (size_t)B * W;
  const int lb = std::min(blocks_for((size_t)B * P), 4096);
  k_mse<<<lb, FT, 0, s>>>(f->out, target, f->dout, f->lpart, (size_t)B * P);
  note_launches(1);
  std::vector<double> lp(lb);
  BEM_CUDA_TRY(cudaMemcpyAsync(lp.data(), f->lpart, lb * sizeof(double), cudaMemcpyDeviceToHost, s));
  // projection
  wgrad(f->dout, 1, f->h, H, f->g + f->o_Q2w, f->g + f->o_Q2b, f->part, P, B, s);
  pw<true, false, false>(f->dout, 1, f->wb + f->o_Q2w, nullptr, f->dt, nullptr, H, P, B, s);   // d_h
  k_gelu_bwd<<<blocks_for((size_t)B * H * P), FT, 0, s>>>(f->dt, f->a, f->dz, (size_t)B * H * P);   // d_a
  note_launches(1);
  wgrad(f->dz, H, f->v[L], W, f->g + f->o_Q1w, f->g + f->o_Q1b, f->part, P, B, s);
  pw<true, false, false>(f->dz, H, f->wb + f->o_Q1w, nullptr, f->dv, nullptr, W, P, B, s);     // d_v
  for (int l = L - 1; l >= 0; --l) {
    const float* dz = f->dv;
    if (l < L - 1) {
      k_gelu_bwd<<<blocks_for(bc * P), FT, 0, s>>>(f->dv, f->z[l], f->dz, bc * P);
      note_launches(1);
      dz = f->dz;
    }
    wgrad(dz, W, f->v[l], W, f->g + f->o_Ww + (size_t)l * W * W, f->g + f->o_Wb + (size_t)l * W, f->part, P, B, s);
    // pointwise branch of d_vin into dt
    pw<true, false, false>(dz, W, f->wb + f->o_Ww + (size_t)l * W * W, nullptr, f->dt, nullptr, W, P, B, s);
    // spectral branch: dY = (c/N^2) dft(dz); dR = sum_b conj(Xh) dY; dXh = sum_o conj(R) dY
    dft_y(f, dz, bc * N, N, s);
    k_dft_x_par<<<dim3((unsigned)bc, 2 * m), 256, 0, s>>>(f->A, f->dY, f->tw, f->cky_s, N, m);
    const bf16* Rre = f->wb + f->o_Rre + (size_t)l * W * W * nm;
    const bf16* Rim = f->wb + f->o_Rim + (size_t)l * W * W * nm;
    k_mix_wgrad<<<blocks_for((size_t)W * W * nm), FT, 0, s>>>(f->Xh[l], f->dY, f->g + f->o_Rre + (size_t)l * W * W * nm,
                                                          f->g + f->o_Rim + (size_t)l * W * W * nm, W, (int)nm, B);
    k_mix_dgrad<<<blocks_for(bc * nm), FT, 0, s>>>(f->dY, Rre, Rim, f->Y, W, (int)nm, B);
    // d_vin += Re(sum dXh e^{+i theta}) (adjoint of the forward transform)
    k_idft_x<<<blocks_for(bc * N * ((m + 3) / 4)), FT, 0, s>>>(f->Y, f->A, f->tw, N, m, bc);
    idft_y<true>(f, f->dt, nullptr, 1.f, bc * N, N, s);
    note_launches(6);
    std::swap(f->dv, f->dt);
  }
  wgrad(f->dv, W, x, 7, f->g + f->o_Pw, f->g + f->o_Pb, f->part, P, B, s);
  BEM_CUDA_TRY(cudaGetLastError());
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  double sum = 0.0;
  for (double v : lp) sum += v;
  *loss = sum / (double)((size_t)B * P);
  return BEM_OK;
}

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

bem_status bem_fno_create(const bem_fno_desc* desc, bem_fno* out) {
  if (desc == nullptr || out == nullptr) { set_error("NULL argument"); return BEM_EINVAL; }
  *out = nullptr;
  if (!width_ok(desc->width) || !width_ok(desc->hidden) || desc->modes < 1 || desc->layers < 1 ||
      desc->layers > 16) {
    set_error("FNO widths must be one of 1, 7, 8, 16, 32, 64; modes >= 1; 1 <= layers <= 16");
    return BEM_EINVAL;
  }
  bem_fno_s* f = new bem_fno_s();
  f->d = *desc;
  cudaGetDevice(&f->dev);
  const size_t W = desc->width, m = desc->modes, L = desc->layers, H = desc->hidden;
  const size_t nm = 2 * m * m;
  size_t off = 0;
  f->o_Pw = off; off += W * 7;
  f->o_Pb = off; off += W;
  f->o_Rre = off; off += L * W * W * nm;
  f->o_Rim = off; off += L * W * W * nm;
  f->o_Ww = off; off += L * W * W;
  f->o_Wb = off; off += L * W;
  f->o_Q1w = off; off += H * W;
  f->o_Q1b = off; off += H;
  f->o_Q2w = off; off += H;
  f->o_Q2b = off; off += 1;
  f->P = off;
  cudaError_t e = alloc(f, &f->w, f->P);
  if (e == cudaSuccess) e = alloc(f, &f->wb, f->P);
  if (e == cudaSuccess) e = alloc(f, &f->g, f->P);
  if (e == cudaSuccess) e = alloc(f, &f->m1, f->P);
  if (e == cudaSuccess) e = alloc(f, &f->m2, f->P);
  if (e == cudaSuccess) e = alloc(f, &f->mom, (size_t)4 * kMaxSamples);
  if (e == cudaSuccess) e = alloc(f, &f->mom_part, (size_t)2 * kMomChunks * kMaxSamples);
  f->n_persistent = f->owned.size();
  if (e != cudaSuccess) {
    for (void* p : f->owned) cudaFree(p);
    delete f;
    return cuda_fail(e, "cudaMalloc(fno parameters)");
  }
  e = cudaMemset(f->w, 0, f->P * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(f->wb, 0, f->P * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMemset(f->g, 0, f->P * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(f->m1, 0, f->P * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(f->m2, 0, f->P * sizeof(float));
  if (e != cudaSuccess) {
    for (void* p : f->owned) cudaFree(p);
    delete f;
    return cuda_fail(e, "cudaMemset(fno parameters)");
  }
  *out = f;
  return BEM_OK;
}

bem_status bem_fno_destroy(bem_fno f) {
  if (f == nullptr) return BEM_OK;
  cudaDeviceSynchronize();
  for (void* p : f->owned) cudaFree(p);
  delete f;
  return BEM_OK;
}

int64_t bem_fno_param_count(bem_fno f) { return f == nullptr ? -1 : (int64_t)f->P; }

bem_status bem_fno_set_params(bem_fno f, const float* w, int64_t count, void* cuda_stream) {
  if (f == nullptr || w == nullptr || count != (int64_t)f->P) { set_error("bad parameter vector"); return BEM_EINVAL; }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  BEM_CUDA_TRY(cudaMemcpyAsync(f->w, w, f->P * sizeof(float), cudaMemcpyDefault, s));
  k_to_bf16<<<blocks_for(f->P), FT, 0, s>>>(f->w, f->wb, f->P);
  note_launches(1);
  BEM_CUDA_TRY(cudaMemsetAsync(f->m1, 0, f->P * sizeof(float), s));
  BEM_CUDA_TRY(cudaMemsetAsync(f->m2, 0, f->P * sizeof(float), s));
  f->step = 0;
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status bem_fno_get_params(bem_fno f, float* w, int64_t count, int32_t rounded, void* cuda_stream) {
  if (f == nullptr || w == nullptr || count != (int64_t)f->P) { set_error("bad parameter vector"); return BEM_EINVAL; }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (rounded) {
    // the bf16 values the kernels use, widened to float (staged through the gradient buffer)
    k_bf16_to_f32<<<blocks_for(f->P), FT, 0, s>>>(f->wb, f->g, f->P);
    note_launches(1);
    BEM_CUDA_TRY(cudaMemcpyAsync(w, f->g, f->P * sizeof(float), cudaMemcpyDefault, s));
  } else {
    BEM_CUDA_TRY(cudaMemcpyAsync(w, f->w, f->P * sizeof(float), cudaMemcpyDefault, s));
  }
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status bem_fno_get_state(bem_fno f, float* m1, float* m2, int64_t count, int32_t* step, void* cuda_stream) {
  if (f == nullptr || m1 == nullptr || m2 == nullptr || step == nullptr || count != (int64_t)f->P) {
    set_error("bad optimiser state arguments");
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  BEM_CUDA_TRY(cudaMemcpyAsync(m1, f->m1, f->P * sizeof(float), cudaMemcpyDefault, s));
  BEM_CUDA_TRY(cudaMemcpyAsync(m2, f->m2, f->P * sizeof(float), cudaMemcpyDefault, s));
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  *step = f->step;
  return BEM_OK;
}

bem_status bem_fno_set_state(bem_fno f, const float* m1, const float* m2, int64_t count, int32_t step,
                             void* cuda_stream) {
  if (f == nullptr || m1 == nullptr || m2 == nullptr || count != (int64_t)f->P || step < 0) {
    set_error("bad optimiser state arguments");
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  BEM_CUDA_TRY(cudaMemcpyAsync(f->m1, m1, f->P * sizeof(float), cudaMemcpyDefault, s));
  BEM_CUDA_TRY(cudaMemcpyAsync(f->m2, m2, f->P * sizeof(float), cudaMemcpyDefault, s));
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  f->step = step;
  return BEM_OK;
}

bem_status bem_fno_features(bem_fno f, int32_t B, int32_t N, const float* heights, const double* params, float* x,
                            void* cuda_stream) {
  if (f == nullptr || heights == nullptr || params == nullptr || x == nullptr || B < 1 || N < 2) {
    set_error("invalid FNO feature arguments");
    return BEM_EINVAL;
  }
  if (!is_dev(heights) || !is_dev(params) || !is_dev(x)) { set_error("FNO arrays must be device arrays"); return BEM_EINVAL; }
  if (B > kMaxSamples) { set_error("at most 4096 samples per feature call"); return BEM_EINVAL; }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t P = (size_t)N * N;
  k_fno_moments_part<<<dim3(kMomChunks, B), FT, 0, s>>>(heights, f->mom_part, P);
  k_fno_moments<<<B, 32, 0, s>>>(f->mom_part, params, f->mom, P);
  k_fno_features<<<blocks_for((size_t)B * P), FT, 0, s>>>(heights, f->mom, params, x, N, B);
  note_launches(3);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

bem_status bem_fno_forward(bem_fno f, int32_t B, int32_t N, const float* x, float* out, void* cuda_stream) {
  if (f == nullptr || x == nullptr || out == nullptr || B < 1 || N < 2 * f->d.modes || N % 2 != 0) {
    set_error("invalid FNO forward arguments (N must be even and at least twice the retained modes)");
    return BEM_EINVAL;
  }
  if (!is_dev(x) || !is_dev(out)) { set_error("FNO arrays must be device arrays"); return BEM_EINVAL; }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  bem_status st = ensure(f, B, N, f->cap_train && B <= f->capB && N <= f->capN, s);
  if (st != BEM_OK) return st;
  st = forward(f, B, N, x, f->cap_train, s);
  if (st != BEM_OK) return st;
  BEM_CUDA_TRY(cudaMemcpyAsync(out, f->out, (size_t)B * N * N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return BEM_OK;
}

bem_status bem_fno_gradients(bem_fno f, int32_t B, int32_t N, const float* x, const float* target, float* grad,
                             double* loss, void* cuda_stream) {
  if (f == nullptr || x == nullptr || target == nullptr || loss == nullptr || B < 1 || N < 2 * f->d.modes ||
      N % 2 != 0) {
    set_error("invalid FNO gradient arguments (N must be even and at least twice the retained modes)");
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  bem_status st = ensure(f, B, N, true, s);
  if (st != BEM_OK) return st;
  st = forward(f, B, N, x, true, s);
  if (st != BEM_OK) return st;
  st = backward(f, B, N, x, target, loss, s);
  if (st != BEM_OK) return st;
  if (grad != nullptr) {
    BEM_CUDA_TRY(cudaMemcpyAsync(grad, f->g, f->P * sizeof(float), cudaMemcpyDefault, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return BEM_OK;
}

bem_status bem_fno_train_step(bem_fno f, int32_t B, int32_t N, const float* x, const float* target, float lr,
                              double* loss, void* cuda_stream) {
  bem_status st = bem_fno_gradients(f, B, N, x, target, nullptr, loss, cuda_stream);
  if (st != BEM_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  f->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f / (1.f - powf(b1, (float)f->step)), c2 = 1.f / (1.f - powf(b2, (float)f->step));
  k_adam<<<blocks_for(f->P), FT, 0, s>>>(f->w, f->g, f->m1, f->m2, f->wb, f->P, lr, b1, b2, c1, c2, 1e-8f);
  note_launches(1);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

bem_status bem_fno_pressure(bem_fno f, int32_t B, int32_t N, const float* out, const double* pbar, float q_min,
                            float* p, void* cuda_stream) {
  if (f == nullptr || out == nullptr || pbar == nullptr || p == nullptr || B < 1 || !(q_min >= 0.f)) {
    set_error("invalid FNO pressure arguments");
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_fno_pressure<<<blocks_for((size_t)B * N * N), FT, 0, s>>>(out, pbar, q_min, p, (size_t)N * N, B);
  note_launches(1);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

bem_status bem_fno_target(bem_fno f, int32_t B, int32_t N, const float* p, const double* pbar, float* q,
                          void* cuda_stream) {
  if (f == nullptr || p == nullptr || pbar == nullptr || q == nullptr || B < 1) {
    set_error("invalid FNO target arguments");
    return BEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_fno_target<<<blocks_for((size_t)B * N * N), FT, 0, s>>>(p, pbar, q, (size_t)N * N, B);
  note_launches(1);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

}  // extern "C"
