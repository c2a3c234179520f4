// The surface operator u = K p (Eq. 1) evaluated as in Eq. (11) on a 2N x 2N period.
//
// Three passes, all zero-padding aware (the padded half is never stored):
//  1. row pass    : per row r < N, the length-2N real FFT of (p[r, 0..N-1], 0...),
//                   kept for frequencies j in [0, N] (Hermitian half).  The real row
//                   is packed as N/2 complex values z[m] = p[2m] + i p[2m+1]; the
//                   length-N complex FFT of the half-zero sequence z splits into two
//                   length-N/2 FFTs (even and odd outputs); the standard real-FFT
//                   recombination then gives X[j].
//  2. column pass : per frequency column j, the length-2N FFT of the N nonzero rows
//                   splits into FFT_N(y) (even wave numbers) and FFT_N(y e^{-2 pi i r/2N})
//                   (odd ones); each is multiplied by the compliance K^(|k|) of Eq. (9)
//                   (table scaled by 1/(2N)^2), inverse-transformed, and the two
//                   halves recombine into the first N rows of the inverse transform.
//  3. row inverse : the inverse real FFT of each row, evaluated only at the first N
//                   outputs (the window), via the same packing in reverse.
#include <math.h>

#include "bem_internal.cuh"
#include "fft.cuh"
#include "stack.cuh"

namespace bem {

// ---------------------------------------------------------------------------
// Compliance table (Eqs. 9, 10), evaluated in double on the device.
struct KernelParams {
  double c_pref;   // 2 (1 - nu1^2) / E1
  double A, B, C, D;
  double h;
  double kstep;    // 2 pi / (M delta)
  double dc;       // value at k = 0
  int N;
  int homog;       // h = inf: Eq. (4) with E1, nu1
};

__global__ void k_table64(double* __restrict__ t64, KernelParams P) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j > P.N) return;
  double val;
  if (i == 0 && j == 0) {
    val = P.dc;
  } else {
    const double k = P.kstep * sqrt((double)(i * i + j * j));
    if (P.homog) {
      val = P.c_pref / k;
    } else {
      const double x = k * P.h;
      const double e2 = exp(-2.0 * x);
      const double e4 = e2 * e2;
      const double num = P.A * e4 + P.B * x * e2 + P.D;
      const double den = -P.A * e4 - P.B * x * x * e2 + 2.0 * P.C * e2 + P.D;
      val = P.c_pref * num / (k * den);
    }
  }
  t64[(size_t)i * (P.N + 1) + j] = val;
}

// Compliance of a coating stack (stack.cuh) for every (i, j) in [0, N]^2; the
// k = 0 entry is the finite part computed on the host.
__global__ void k_table64_stack(double* __restrict__ t64, Stack st, double kstep, double dc, int N) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j > N) return;
  double val;
  if (i == 0 && j == 0) {
    val = dc;
  } else {
    const double k = kstep * sqrt((double)(i * i + j * j));
    val = stack_phi<double>(st, k) / k;
  }
  t64[(size_t)i * (N + 1) + j] = val;
}

// ---------------------------------------------------------------------------
// Open-plane operator of a homogeneous half-space.  The displacement at (x, y) of a
// uniform unit pressure on the square cell |xi|, |eta| <= delta/2 is Boussinesq's
// point-load solution 1/(pi E* r) (Eq. 4 in real space) integrated over the cell; the
// double integral of 1/r has the closed form (Love)
//   I(x, y) = F(x+h, y+h) - F(x+h, y-h) - F(x-h, y+h) + F(x-h, y-h),  h = delta/2,
//   F(s, t) = s asinh(t/|s|) + t asinh(s/|t|)   (a term is 0 where its s or t is 0).
// The window products only use offsets |dx|, |dy| <= N - 1, so the 2N-periodic
// wrap-around array W of the coefficients (zero at offset N) gives the open-plane
// convolution exactly; its 2-D DFT is real and even, K(i, j) = sum_{x, y} w_x w_y
// G(x, y) cos(pi i x / N) cos(pi j y / N) over x, y in [0, N] (w_0 = 1, w = 2
// inside, w_N = 0), i.e. K = C Gw C^T with C[i][x] = cos(pi i x / N): two double
// matrix products of order N + 1.
__device__ double love_f(double s, double t) {
  const double a = (s != 0.0) ? s * asinh(t / fabs(s)) : 0.0;
  const double b = (t != 0.0) ? t * asinh(s / fabs(t)) : 0.0;
  return a + b;
}

__global__ void k_open_coef(double* __restrict__ gw, int N, double delta, double inv_pi_es) {
  const size_t n1 = (size_t)N + 1, total = n1 * n1;
  const double h = 0.5 * delta;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n1), j = (int)(idx % n1);
    double v = 0.0;
    if (i < N && j < N) {
      const double x = i * delta, y = j * delta;
      const double I = love_f(x + h, y + h) - love_f(x + h, y - h) - love_f(x - h, y + h) + love_f(x - h, y - h);
      v = (i == 0 ? 1.0 : 2.0) * (j == 0 ? 1.0 : 2.0) * I * inv_pi_es;
    }
    gw[idx] = v;
  }
}

__global__ void k_cos_mat(double* __restrict__ cm, int N) {
  const size_t n1 = (size_t)N + 1, total = n1 * n1;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const long long i = (long long)(idx / n1), x = (long long)(idx % n1);
    cm[idx] = cospi((double)((i * x) % (2 * N)) / (double)N);
  }
}

// Cout[m][n] = sum_k A[m][k] B[n][k] for n x n row-major matrices (double; 64 x 64
// output tiles, 4 x 4 per thread, k in steps of 16 through shared memory)
__global__ void __launch_bounds__(256) k_dgemm_nt(const double* __restrict__ A, const double* __restrict__ B,
                                                  double* __restrict__ Cout, int n) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int r = e / 16, kk = e % 16;
      const int m = m0 + r, nn = n0 + r, k = k0 + kk;
      As[kk][r] = (m < n && k < n) ? A[(size_t)m * n + k] : 0.0;
      Bs[kk][r] = (nn < n && k < n) ? B[(size_t)nn * n + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] = fma(a[q], b[r], acc[q][r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int m = m0 + ty + 16 * q, nn = n0 + tx + 16 * r;
      if (m < n && nn < n) Cout[(size_t)m * n + nn] = acc[q][r];
    }
}

// The open-plane table into k->ws.table64; the handle's spectrum and solver vectors
// (unused until the first product) hold the intermediate matrices.
static bem_status build_open_table(bem_kernel_s* k, cudaStream_t s) {
  double E = 0.0, nu = 0.0;
  open_plane_homogeneous(k->desc, &E, &nu);
  const double es = E / (1.0 - nu * nu);
  const int n = k->N + 1;
  double* cm = (double*)k->ws.spec;
  double* gw = (double*)k->ws.vec;
  double* u = gw + (size_t)n * n;
  k_open_coef<<<256, 256, 0, s>>>(gw, k->N, k->desc.delta, 1.0 / (M_PI * es));
  k_cos_mat<<<256, 256, 0, s>>>(cm, k->N);
  const dim3 grid((n + 63) / 64, (n + 63) / 64);
  k_dgemm_nt<<<grid, 256, 0, s>>>(cm, gw, u, n);              // U = C Gw (Gw is symmetric)
  k_dgemm_nt<<<grid, 256, 0, s>>>(u, cm, k->ws.table64, n);   // K = U C^T
  note_launches(4);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

// The stack of a handle in the scaled form of stack.cuh.
static Stack stack_of(const bem_kernel_s* k) {
  Stack st{};
  st.n = k->n_layers;
  const double mu_ref = k->layers[0].E / (2.0 * (1.0 + k->layers[0].nu));
  st.mu_ref = mu_ref;
  for (int l = 0; l < st.n; ++l) {
    st.L[l].h = k->layers[l].h;
    st.L[l].q = k->layers[l].E / (2.0 * (1.0 + k->layers[l].nu)) / mu_ref;
    st.L[l].nu = k->layers[l].nu;
  }
  st.rigid = isinf(k->desc.E2) ? 1 : 0;
  st.qs = st.rigid ? 0.0 : k->desc.E2 / (2.0 * (1.0 + k->desc.nu2)) / mu_ref;
  st.nus = k->desc.nu2;
  return st;
}

// Blocked copy in the path precision, scaled by 1/M^2:
// table[(cb (N+1) + i) TC + tc] = K(i, cb TC + tc) / M^2 (0 past j = N).
template <typename T>
__global__ void k_table_block(const double* __restrict__ t64, T* __restrict__ tab, int N, double scale) {
  const int nblk = N / TC + 1;
  const size_t total = (size_t)nblk * (N + 1) * TC;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int tc = (int)(idx % TC);
    const size_t rest = idx / TC;
    const int i = (int)(rest % (N + 1));
    const int cb = (int)(rest / (N + 1));
    const int j = cb * TC + tc;
    tab[idx] = (j <= N) ? (T)(t64[(size_t)i * (N + 1) + j] * scale) : (T)0;
  }
}

// Square copy in the path precision, scaled by 1/M^2, rows padded to N + 4 entries.
// K depends on i^2 + j^2 only, so entry (i, j) is also entry (j, i): the values of
// frequency column j form row j here.
template <typename T>
__global__ void k_table_square(const double* __restrict__ t64, T* __restrict__ tab, int N, double scale) {
  const size_t total = (size_t)(N + 1) * (N + 4);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx / (N + 4), j = idx % (N + 4);
    tab[idx] = (j <= (size_t)N) ? (T)(t64[i * (N + 1) + j] * scale) : (T)0;
  }
}

// Float register path: the compliance in column pairs, scaled by 1/M^2:
// tab2[p (N + 1) + f] = (K(f, 2p), K(f, 2p + 1)), p in [0, N/2], f in [0, N]; the
// column N + 1 of the last pair does not exist and holds 0.
__global__ void k_table_pair(const double* __restrict__ t64, float2* __restrict__ tab, int N, double scale) {
  const size_t total = (size_t)(N / 2 + 1) * (N + 1);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t p = idx / (N + 1), f = idx % (N + 1);
    const size_t ja = 2 * p, jb = 2 * p + 1;
    const float a = (float)(t64[f * (N + 1) + ja] * scale);
    const float b = jb <= (size_t)N ? (float)(t64[f * (N + 1) + jb] * scale) : 0.f;
    tab[idx] = make_float2(a, b);
  }
}

template <typename T>
__global__ void k_twiddles(cplx<T>* __restrict__ tw, int M) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)M, &s, &c);
    tw[m] = mk((T)c, (T)(-s));
  }
}

// Normalised constants of Eq. (10): every constant is a quadratic form in
// a = E2 (1 + nu1), b = E1 (1 + nu2); dividing all four by (a + b)^2 leaves
// the ratio of Eq. (9) unchanged and stays finite for E2 = inf.
static void layered_constants(const bem_kernel_desc& d, double* A, double* B, double* C, double* D) {
  double al, be;
  if (isinf(d.E2)) {
    al = 1.0;
    be = 0.0;
  } else {
    const double a = d.E2 * (1.0 + d.nu1), b = d.E1 * (1.0 + d.nu2);
    al = a / (a + b);
    be = b / (a + b);
  }
  const double n1 = d.nu1, n2 = d.nu2;
  *A = ((3.0 - 4.0 * n1) * al - (3.0 - 4.0 * n2) * be) * (be - al);
  *B = 4.0 * (al + (3.0 - 4.0 * n2) * be) * (be - al);
  *C = (4.0 * n2 - 3.0) * be * be - 2.0 * (2.0 * n1 - 1.0) * (2.0 * n2 - 1.0) * al * be +
       (8.0 * n1 * n1 - 12.0 * n1 + 5.0) * al * al;
  *D = (al + (3.0 - 4.0 * n2) * be) * ((3.0 - 4.0 * n1) * al + be);
}

// Upper bound on the stage twiddle entries of a length-2^logl register FFT: the
// stage tables hold sum_{s>=1} R_s Ns_s = sum_{s>=1} Ns_{s+1} < 2L values.
int stage_tw_count(int logl) { return 2 << logl; }
// the paired tables hold at most Q planes of Ns records per stage (twp_planes(Q) <= Q
// for every radix used), and sum_{s>=1} Q_s Ns_s < 2L as above
int pair_tw_count(int logl) { return 2 << logl; }

size_t spec_bytes(const bem_kernel_s* k) {
  return (size_t)(k->N / TC + 1) * k->N * TC * 2 * k->elem;
}
size_t table_bytes(const bem_kernel_s* k) {
  // blocked layout (N < 16 path) or the square table (register path, rows of N + 4
  // so that every row starts on a 16-byte boundary), whichever is larger
  const size_t blocked = (size_t)(k->N / TC + 1) * (k->N + 1) * TC;
  const size_t square = (size_t)(k->N + 1) * (k->N + 4);
  return (blocked > square ? blocked : square) * k->elem;
}

bem_status build_table(bem_kernel_s* k, cudaStream_t s) {
  const bem_kernel_desc& d = k->desc;
  KernelParams P;
  P.N = k->N;
  P.c_pref = 2.0 * (1.0 - d.nu1 * d.nu1) / d.E1;
  P.h = d.h;
  P.kstep = 2.0 * M_PI / ((double)k->M * d.delta);
  P.homog = isinf(d.h) ? 1 : 0;
  layered_constants(d, &P.A, &P.B, &P.C, &P.D);
  // DC finite part: k K(k) = c F(kh), F = num/den; lim [K - F(0) c / k] = c h F'(0)
  // with num'(0) = B - 4A and den'(0) = 4A - 4C.
  if (P.homog || d.dc_mode == BEM_DC_ZERO) {
    P.dc = 0.0;
  } else {
    const double n0 = P.A + P.D, d0 = -P.A + 2.0 * P.C + P.D;
    const double dn = P.B - 4.0 * P.A, dd = 4.0 * P.A - 4.0 * P.C;
    P.dc = P.c_pref * d.h * (dn * d0 - n0 * dd) / (d0 * d0);
  }
  dim3 grid((k->N + 1 + 127) / 128, k->N + 1);
  if (d.op_kind == BEM_OP_OPEN) {
    bem_status st = build_open_table(k, s);
    if (st != BEM_OK) return st;
  } else if (k->n_layers > 0) {
    // stack: the long-wave expansion phi(eps) = phi(0) + phi'(0) eps by dual numbers
    const Stack st = stack_of(k);
    const double dc = (d.dc_mode == BEM_DC_ZERO) ? 0.0 : stack_phi<Dual>(st, Dual{0.0, 1.0}).d;
    if (!isfinite(dc)) {
      set_error("coating stack: non-finite long-wave compliance");
      return BEM_EINVAL;
    }
    k_table64_stack<<<grid, 128, 0, s>>>(k->ws.table64, st, P.kstep, dc, k->N);
  } else {
    k_table64<<<grid, 128, 0, s>>>(k->ws.table64, P);
  }
  note_launches(3);
  BEM_CUDA_TRY(cudaGetLastError());
  const double scale = 1.0 / ((double)k->M * (double)k->M);
  if (k->prec == BEM_FP64) {
    if (k->logN >= 4) k_table_square<double><<<256, 256, 0, s>>>(k->ws.table64, (double*)k->ws.table, k->N, scale);
    else k_table_block<double><<<256, 256, 0, s>>>(k->ws.table64, (double*)k->ws.table, k->N, scale);
    k_twiddles<double><<<(k->M + 255) / 256, 256, 0, s>>>((double2*)k->ws.tw, k->M);
    if (k->logN >= 4) reg_twiddles<double>(k, s);
  } else {
    if (k->logN >= 4) k_table_pair<<<256, 256, 0, s>>>(k->ws.table64, (float2*)k->ws.table, k->N, scale);
    else k_table_block<float><<<256, 256, 0, s>>>(k->ws.table64, (float*)k->ws.table, k->N, scale);
    k_twiddles<float><<<(k->M + 255) / 256, 256, 0, s>>>((float2*)k->ws.tw, k->M);
    if (k->logN >= 4) reg_twiddles<float>(k, s);
  }
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// Pass 1: rows, real -> half spectrum.  Block = TR rows.
template <typename T, int TR>
__global__ void __launch_bounds__(NTHREADS)
k_row_fwd(const T* __restrict__ p, cplx<T>* __restrict__ spec, const cplx<T>* __restrict__ tw, int logN,
          const int* __restrict__ skip) {
  using C = cplx<T>;
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logN, logH = logN - 1, H = N >> 1;
  C* a = reinterpret_cast<C*>(smem_raw);
  C* b = a + TR * N;
  const int r0 = blockIdx.x * TR;
  // sequences (rl, 0): z[m];  (rl, 1): z[m] e^{-2 pi i m/N}   (m < N/2)
  for (int idx = threadIdx.x; idx < TR * H; idx += blockDim.x) {
    const int rl = idx >> logH, m = idx & (H - 1);
    const C z = reinterpret_cast<const C*>(p + (size_t)(r0 + rl) * N)[m];
    a[(2 * rl) * H + m] = z;
    a[(2 * rl + 1) * H + m] = cmul(z, tw[2 * m]);
  }
  __syncthreads();
  const C* Z = block_fft<false>(a, b, logH, 2 * TR, tw, logN + 1);
  // X[j] = (Z[j] + Z*[N-j])/2 + e^{-2 pi i j/M} (Z[j] - Z*[N-j])/(2i),  j in [0, N]
  const int nblk = N / TC + 1;
  for (int idx = threadIdx.x; idx < nblk * TR * TC; idx += blockDim.x) {
    const int cb = idx / (TR * TC);
    const int q = idx - cb * (TR * TC);
    const int rl = q / TC, tc = q - rl * TC;
    const int j = cb * TC + tc;
    C X = mk((T)0, (T)0);
    if (j <= N) {
      const int j1 = j & (N - 1), j2 = (N - j) & (N - 1);
      const C za = Z[(2 * rl + (j1 & 1)) * H + (j1 >> 1)];
      const C zb = cconj(Z[(2 * rl + (j2 & 1)) * H + (j2 >> 1)]);
      const C E = cscale(cadd(za, zb), (T)0.5);
      const C O = cscale(cmul_mi(csub(za, zb)), (T)0.5);
      X = cadd(E, cmul(O, tw[j]));
    }
    spec[((size_t)cb * N + r0) * TC + q] = X;
  }
}

// Pass 2: columns, FFT -> x K^ -> IFFT, cropped to N rows.  Block = one column block.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
k_col(cplx<T>* __restrict__ spec, const T* __restrict__ table, const cplx<T>* __restrict__ tw, int logN,
      const int* __restrict__ skip) {
  using C = cplx<T>;
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logN, M = 2 * N;
  C* a = reinterpret_cast<C*>(smem_raw);
  C* b = a + 2 * N;
  const int cb = blockIdx.x;
  const int ncols = (cb == N / TC) ? 1 : TC;
  for (int tc = 0; tc < ncols; ++tc) {
    C* col = spec + (size_t)cb * N * TC + tc;
    const T* kt = table + (size_t)cb * (N + 1) * TC + tc;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const C y = col[(size_t)r * TC];
      a[r] = y;
      a[N + r] = cmul(y, tw[r]);
    }
    __syncthreads();
    C* V = block_fft<false>(a, b, logN, 2, tw, logN + 1);
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      const int ie = 2 * q, io = 2 * q + 1;
      const int fe = min(ie, M - ie), fo = min(io, M - io);
      V[q] = cscale(V[q], kt[(size_t)fe * TC]);
      V[N + q] = cscale(V[N + q], kt[(size_t)fo * TC]);
    }
    __syncthreads();
    C* W = block_fft<true>(V, (V == a) ? b : a, logN, 2, tw, logN + 1);
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      col[(size_t)r * TC] = cadd(W[r], cmulc(W[N + r], tw[r]));
    }
    __syncthreads();
  }
}

// Pass 3: rows, half spectrum -> real, first N outputs.  Block = TR rows.
template <typename T, int TR>
__global__ void __launch_bounds__(NTHREADS)
k_row_inv(const cplx<T>* __restrict__ spec, T* __restrict__ u, const cplx<T>* __restrict__ tw, int logN,
          const int* __restrict__ skip) {
  using C = cplx<T>;
  if (skip != nullptr && *skip == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logN, logH = logN - 1, H = N >> 1;
  C* a = reinterpret_cast<C*>(smem_raw);
  C* b = a + TR * N;
  const int r0 = blockIdx.x * TR;
  // Zi[j] = (Y[j] + Y*[N-j]) + i (Y[j] - Y*[N-j]) e^{+2 pi i j/M},  j in [0, N)
  for (int idx = threadIdx.x; idx < (N / TC) * TR * TC; idx += blockDim.x) {
    const int cb = idx / (TR * TC);
    const int q = idx - cb * (TR * TC);
    const int rl = q / TC, tc = q - rl * TC;
    const int j = cb * TC + tc;
    const int jr = N - j;
    const C y1 = spec[((size_t)cb * N + r0) * TC + q];
    const C y2 = cconj(spec[((size_t)(jr / TC) * N + r0 + rl) * TC + (jr % TC)]);
    const C e = cadd(y1, y2);
    const C o = cmul_pi(cmulc(csub(y1, y2), tw[j]));
    a[(2 * rl + (j & 1)) * H + (j >> 1)] = cadd(e, o);
  }
  __syncthreads();
  const C* z = block_fft<true>(a, b, logH, 2 * TR, tw, logN + 1);
  // z[m] = Ze[m] + e^{+2 pi i m/N} Zo[m];  u[r, 2m] = Re z, u[r, 2m+1] = Im z
  for (int idx = threadIdx.x; idx < TR * H; idx += blockDim.x) {
    const int rl = idx >> logH, m = idx & (H - 1);
    const C v = cadd(z[(2 * rl) * H + m], cmulc(z[(2 * rl + 1) * H + m], tw[2 * m]));
    reinterpret_cast<C*>(u + (size_t)(r0 + rl) * N)[m] = v;
  }
}

template <typename T> struct RowsPerBlock;
template <> struct RowsPerBlock<float> { static constexpr int value = 4; };
template <> struct RowsPerBlock<double> { static constexpr int value = 2; };

template <typename T>
static void set_smem_attrs() {
  using C = cplx<T>;
  constexpr int TR = RowsPerBlock<T>::value;
  static std::atomic<unsigned long long> done{0};
  if (!first_on_device(done)) return;
  const int max_row = 2 * TR * (1 << MAX_LOGN) * (int)sizeof(C);
  const int max_col = 4 * (1 << MAX_LOGN) * (int)sizeof(C);
  cudaFuncSetAttribute(k_row_fwd<T, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_row);
  cudaFuncSetAttribute(k_row_inv<T, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_row);
  cudaFuncSetAttribute(k_col<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_col);
}

template <typename T>
static void pass_impl(const bem_kernel_s* k, int pass, const T* p, T* u, cudaStream_t s, const int* skip) {
  using C = cplx<T>;
  constexpr int TR = RowsPerBlock<T>::value;
  set_smem_attrs<T>();
  const int N = k->N, logN = k->logN;
  const size_t smem_row = (size_t)2 * TR * N * sizeof(C);
  const size_t smem_col = (size_t)4 * N * sizeof(C);
  C* spec = (C*)k->ws.spec;
  const C* tw = (const C*)k->ws.tw;
  if (k->logN >= 4) {
    reg_pass<T>(k, pass, p, u, s, skip);
    note_launches(1);
    return;
  }
  if (pass == 0) k_row_fwd<T, TR><<<N / TR, NTHREADS, smem_row, s>>>(p, spec, tw, logN, skip);
  if (pass == 1) k_col<T><<<N / TC + 1, NTHREADS, smem_col, s>>>(spec, (const T*)k->ws.table, tw, logN, skip);
  if (pass == 2) k_row_inv<T, TR><<<N / TR, NTHREADS, smem_row, s>>>(spec, u, tw, logN, skip);
  note_launches(1);
}

static std::pair<cudaEvent_t, cudaEvent_t> timing_pair(const bem_kernel_s* k) {
  auto& tm = k->timing;
  if (!tm.pool.empty()) {
    auto e = tm.pool.back();
    tm.pool.pop_back();
    return e;
  }
  std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
  cudaEventCreate(&e.first);
  cudaEventCreate(&e.second);
  return e;
}

void harvest_pass_timing(const bem_kernel_s* k) {
  auto& tm = k->timing;
  for (int pass = 0; pass < 3; ++pass) {
    for (auto& e : tm.pending[pass]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) {
        tm.ms[pass] += ms;
        tm.n[pass] += 1;
      } else {
        cudaGetLastError();
      }
      tm.pool.push_back(e);
    }
    tm.pending[pass].clear();
  }
}

template <typename T>
void launch_matvec(const bem_kernel_s* k, const T* p, T* u, cudaStream_t s, const int* skip) {
  for (int pass = 0; pass < 3; ++pass) {
    if (k->timing.on) {
      auto e = timing_pair(k);
      cudaEventRecord(e.first, s);
      pass_impl<T>(k, pass, p, u, s, skip);
      cudaEventRecord(e.second, s);
      k->timing.pending[pass].push_back(e);
    } else {
      pass_impl<T>(k, pass, p, u, s, skip);
    }
  }
}

template <typename T>
void launch_pass(const bem_kernel_s* k, int pass, const T* p, T* u, cudaStream_t s) {
  pass_impl<T>(k, pass, p, u, s, nullptr);
}

template <typename T>
void prepare_passes(const bem_kernel_s* k) {
  if (k->logN >= 4) reg_prepare<T>(k);
  else set_smem_attrs<T>();
}

template void prepare_passes<float>(const bem_kernel_s*);
template void prepare_passes<double>(const bem_kernel_s*);
template void launch_pass<float>(const bem_kernel_s*, int, const float*, float*, cudaStream_t);
template void launch_pass<double>(const bem_kernel_s*, int, const double*, double*, cudaStream_t);
template void launch_matvec<float>(const bem_kernel_s*, const float*, float*, cudaStream_t, const int*);
template void launch_matvec<double>(const bem_kernel_s*, const double*, double*, cudaStream_t, const int*);

}  // namespace bem
