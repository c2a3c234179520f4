// Surface compliance of a stack of bonded elastic layers on an elastic (or rigid)
// substrate, in Fourier space: the multi-layer generalisation of Eqs. (9)/(10),
// which the paper derives for one layer from the Navier equations (Eq. 5) with
// boundary conditions (a)-(d) of Sec. 2.
//
// For a wave number k the plane-strain solutions of Eq. (5) in a layer are, with
// x = k z (z into the body), kappa = 3 - 4 nu, and the displacements written as
// (i U~, W) e^{i k s} along the in-plane direction s:
//   decaying  W = (a + b x) e^{-x},  U~ = (-a + (kappa - x) b) e^{-x}
//   growing   W = (c + d x') e^{x'},  U~ = (c + (kappa + x') d) e^{x'}
// and the tractions, divided by 2 mu_ref k (mu_ref: the shear modulus of the top
// layer, q = mu / mu_ref), are
//   decaying  tau = q (a + (x - 2(1 - nu)) b) e^{-x},  sig = q (-a + (1 - 2nu - x) b) e^{-x}
//   growing   tau = q (c + (2(1 - nu) + x') d) e^{x'},  sig = q (c + (1 - 2nu + x') d) e^{x'}.
// In a layer of thickness h the decaying part is measured from its top (x = 0..X,
// X = k h) and the growing part from its bottom (x' = x - X), so no factor exceeds 1.
//
// The state (U~, W, tau, sig) admitted by everything below an interface is a
// two-dimensional subspace, kept as the columns of a 4 x 2 matrix S:
//   substrate: its decaying solutions (rigid base: zero displacements, free tractions);
//   layer: the bottom state B_d (a, b) + B_g (c, d) must lie in span S, which fixes
//     (c, d) = G (a, b) by one 4 x 4 solve [B_g | -S] [G; w] = -B_d; the top state is
//     then (T_d + T_g G)(a, b), the new S.  B_d and T_g carry e^{-X}: a thick layer
//     decouples its two faces without any overflow.
// At the surface tau = 0 and sig = -1 (unit pressure, condition (c)) fix the two
// coefficients; K(k) = W(0) / (2 mu_ref k).
//
// phi(k) = k K(k) depends on k only through the X_j = k h_j.  Evaluated with dual
// numbers X_j = h_j eps it gives phi(0) (= 2/E_sub*, or 0 for a rigid base) and
// phi'(0), the finite part lim_{k->0} [K(k) - phi(0)/k] used for the k = 0 entry.
#pragma once

#include <math.h>

#include "bem.h"

namespace bem {

struct StackLayer {
  double h;    // thickness
  double q;    // shear modulus / that of the top layer
  double nu;
};

struct Stack {
  int n;                                // layers, surface first
  int rigid;                            // 1: rigid base
  double qs, nus;                       // substrate (when not rigid)
  double mu_ref;                        // shear modulus of the top layer
  StackLayer L[BEM_MAX_LAYERS];
};

// dual number v + d eps (eps^2 = 0)
struct Dual {
  double v, d;
};
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__host__ __device__ inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
__host__ __device__ inline Dual operator/(Dual a, Dual b) {
  return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
__host__ __device__ inline Dual expneg(Dual a) {
  const double e = exp(-a.v);
  return {e, -e * a.d};
}
__host__ __device__ inline double expneg(double a) { return exp(-a); }
__host__ __device__ inline double value(double a) { return a; }
__host__ __device__ inline double value(Dual a) { return a.v; }
template <typename R> __host__ __device__ inline R cst(double c);
template <> __host__ __device__ inline double cst<double>(double c) { return c; }
template <> __host__ __device__ inline Dual cst<Dual>(double c) { return {c, 0.0}; }

// Solves A X = B for the 4 x 4 A and 4 x 2 B (both overwritten), partial pivoting on
// the values; X is returned in B.
template <typename R>
__host__ __device__ inline void solve4x2(R (&A)[4][4], R (&B)[4][2]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
#pragma unroll
    for (int r = c + 1; r < 4; ++r) {
      const bool sw = fabs(value(A[r][c])) > fabs(value(A[c][c]));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const R t = sw ? A[r][j] : A[c][j];
        A[r][j] = sw ? A[c][j] : A[r][j];
        A[c][j] = t;
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const R t = sw ? B[r][j] : B[c][j];
        B[r][j] = sw ? B[c][j] : B[r][j];
        B[c][j] = t;
      }
    }
#pragma unroll
    for (int r = c + 1; r < 4; ++r) {
      const R f = A[r][c] / A[c][c];
#pragma unroll
      for (int j = c + 1; j < 4; ++j) A[r][j] = A[r][j] - f * A[c][j];
#pragma unroll
      for (int j = 0; j < 2; ++j) B[r][j] = B[r][j] - f * B[c][j];
    }
  }
#pragma unroll
  for (int c = 3; c >= 0; --c) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      R acc = B[c][j];
#pragma unroll
      for (int m = c + 1; m < 4; ++m) acc = acc - A[c][m] * B[m][j];
      B[c][j] = acc / A[c][c];
    }
  }
}

// phi = k K(k) for the stack, where the thickness of layer j enters as X_j = s h_j
// (s = k for a plain evaluation, s = eps for the long-wave expansion).
template <typename R>
__host__ __device__ inline R stack_phi(const Stack& st, R s) {
  R S[4][2];
  if (st.rigid) {
    S[0][0] = cst<R>(0.0); S[0][1] = cst<R>(0.0);
    S[1][0] = cst<R>(0.0); S[1][1] = cst<R>(0.0);
    S[2][0] = cst<R>(1.0); S[2][1] = cst<R>(0.0);
    S[3][0] = cst<R>(0.0); S[3][1] = cst<R>(1.0);
  } else {
    const double q = st.qs, nu = st.nus;
    S[0][0] = cst<R>(-1.0); S[0][1] = cst<R>(3.0 - 4.0 * nu);
    S[1][0] = cst<R>(1.0);  S[1][1] = cst<R>(0.0);
    S[2][0] = cst<R>(q);    S[2][1] = cst<R>(-2.0 * (1.0 - nu) * q);
    S[3][0] = cst<R>(-q);   S[3][1] = cst<R>((1.0 - 2.0 * nu) * q);
  }
  for (int l = st.n - 1; l >= 0; --l) {
    const double q = st.L[l].q, nu = st.L[l].nu, ka = 3.0 - 4.0 * nu;
    const R X = s * cst<R>(st.L[l].h);
    const R e = expneg(X);
    // [B_g | -S] [G; w] = -B_d at the layer's bottom
    R A[4][4], Bm[4][2];
    A[0][0] = cst<R>(1.0); A[0][1] = cst<R>(ka);
    A[1][0] = cst<R>(1.0); A[1][1] = cst<R>(0.0);
    A[2][0] = cst<R>(q);   A[2][1] = cst<R>(2.0 * q * (1.0 - nu));
    A[3][0] = cst<R>(q);   A[3][1] = cst<R>(q * (1.0 - 2.0 * nu));
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      A[r][2] = -S[r][0];
      A[r][3] = -S[r][1];
    }
    Bm[0][0] = e;               Bm[0][1] = -(cst<R>(ka) - X) * e;
    Bm[1][0] = -e;              Bm[1][1] = -X * e;
    Bm[2][0] = -cst<R>(q) * e;  Bm[2][1] = -cst<R>(q) * (X - cst<R>(2.0 * (1.0 - nu))) * e;
    Bm[3][0] = cst<R>(q) * e;   Bm[3][1] = -cst<R>(q) * (cst<R>(1.0 - 2.0 * nu) - X) * e;
    solve4x2(A, Bm);
    // top state T_d + T_g G, columns for a and b
    const R g00 = Bm[0][0], g01 = Bm[0][1], g10 = Bm[1][0], g11 = Bm[1][1];
    R Tg[4][2];
    Tg[0][0] = e;              Tg[0][1] = (cst<R>(ka) - X) * e;
    Tg[1][0] = e;              Tg[1][1] = -X * e;
    Tg[2][0] = cst<R>(q) * e;  Tg[2][1] = cst<R>(q) * (cst<R>(2.0 * (1.0 - nu)) - X) * e;
    Tg[3][0] = cst<R>(q) * e;  Tg[3][1] = cst<R>(q) * (cst<R>(1.0 - 2.0 * nu) - X) * e;
    const double Td[4][2] = {{-1.0, ka}, {1.0, 0.0}, {q, -2.0 * q * (1.0 - nu)}, {-q, q * (1.0 - 2.0 * nu)}};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      S[r][0] = cst<R>(Td[r][0]) + Tg[r][0] * g00 + Tg[r][1] * g10;
      S[r][1] = cst<R>(Td[r][1]) + Tg[r][0] * g01 + Tg[r][1] * g11;
    }
  }
  // surface: tau = 0, sig = -1
  const R det = S[2][0] * S[3][1] - S[2][1] * S[3][0];
  const R w0 = S[2][1] / det, w1 = -S[2][0] / det;
  return (S[1][0] * w0 + S[1][1] * w1) / cst<R>(2.0 * st.mu_ref);
}

}  // namespace bem
