// Contact solves (Sec. 2): the inverse problem by Polonsky-Keer constrained
// conjugate gradients (non-adhesive, depth or force control) and the adhesive
// displacement-controlled procedure with the detachment criterion of Eq. (12).
//
// Every step runs on the device.  Scalars live in a device SolveState; reducing
// kernels finish their sums in the last block (reduce.cuh) and update the state
// there, so the host only launches work and reads the state once per chunk of
// iterations.  Every kernel returns at once when state.done is set.
//
// Gap tracking: the gap g = u + f - d is updated recursively (g -= tau K t) while
// the contact set is unchanged, which is exact in exact arithmetic and keeps the
// residual free of the cancellation in u + f - d; whenever a cell enters or leaves
// the set, u = K p is recomputed before the next step.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <unordered_set>
#include <vector>

#include "bem_internal.cuh"
#include "reduce.cuh"

namespace bem {

namespace {

constexpr int CHUNK = 8;   // iterations launched between host checks

template <typename T>
struct DV {
  T *p, *g, *t, *r, *u, *f, *x;
};

template <typename T>
DV<T> dv(const bem_kernel_s* k) {
  const size_t n = (size_t)k->N * k->N;
  T* base = (T*)k->ws.vec;
  return DV<T>{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n, base + 6 * n};
}

// Share of the contact set whose re-entry in one step restarts the conjugate
// directions.  Polonsky and Keer restart on any re-entry; on rough surfaces, where a
// few cells re-enter in most steps, that turns the iteration into steepest descent
// (at N = 1024, 193 of 218 steps restarted).  Keeping the recurrence through smaller
// re-entries reaches the same solution (the stopping test is unchanged) in 2-3 times
// fewer steps; a direction that is not a descent direction still restarts.
constexpr double kRestartShare = 0.1;   // 1 %: 27.5 ms, 10 %: 26.0 ms at N = 2048 (GB300)

// Blocks of a reduction sweep: per_sm blocks per SM (one wave at the kernel's register
// count; more resident threads keep more loads in flight), fewer for small n.
int red_blocks(size_t n, int per_sm) {
  size_t b = (n + NTHREADS * 16 - 1) / (NTHREADS * 16);
  if (b > (size_t)per_sm * 152) b = (size_t)per_sm * 152;
  b = std::max<size_t>(1, std::min<size_t>(b, RED_MAX_BLOCKS));
  return (int)b;
}

#define GRID_STRIDE(i, n) \
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// Four consecutive elements per access (16-byte loads for float, two for double).
#define VEC_LOOP(i4, n) \
  for (size_t i4 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i4 < (n) / 4; i4 += (size_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void ld4(const float* p, size_t i4, float (&o)[4]) {
  const float4 v = reinterpret_cast<const float4*>(p)[i4];
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, size_t i4, double (&o)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[2 * i4], b = reinterpret_cast<const double2*>(p)[2 * i4 + 1];
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, size_t i4, const float (&o)[4]) {
  reinterpret_cast<float4*>(p)[i4] = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void st4(double* p, size_t i4, const double (&o)[4]) {
  reinterpret_cast<double2*>(p)[2 * i4] = make_double2(o[0], o[1]);
  reinterpret_cast<double2*>(p)[2 * i4 + 1] = make_double2(o[2], o[3]);
}

__device__ __forceinline__ void finish(SolveState* st, int status) {
  st->done = 1;
  st->mv_p_on = 0;
  st->mv_t_on = 0;
  if (status != BEM_OK && st->status == BEM_OK) st->status = status;
}

// ---------------------------------------------------------------------------
// Polonsky-Keer CG kernels

// Initial guess for depth control: q = max(d - f, 0) scaled by the energy-optimal
// factor s = <q, d - f> / <q, K q>; the gap then follows from u = K q as s u + f - d.
// contact-set bytes of four consecutive cells: (p > 0) written by k_pk_begin, read
// by the sweeps that need only the set (p keeps its sign until k_pk_update)
template <typename T>
__device__ __forceinline__ void stm4(uint8_t* m, size_t i4, const T (&pv)[4]) {
  reinterpret_cast<uchar4*>(m)[i4] =
      make_uchar4(pv[0] > (T)0, pv[1] > (T)0, pv[2] > (T)0, pv[3] > (T)0);
}
__device__ __forceinline__ void ldm4(const uint8_t* m, size_t i4, bool (&o)[4]) {
  const uchar4 v = reinterpret_cast<const uchar4*>(m)[i4];
  o[0] = v.x != 0;
  o[1] = v.y != 0;
  o[2] = v.z != 0;
  o[3] = v.w != 0;
}

template <typename T>
__global__ void k_init_q(const T* __restrict__ f, T* __restrict__ q, double d, size_t n) {
  const T dT = (T)d;
  GRID_STRIDE(i, n) q[i] = (dT - f[i] > (T)0 ? dT - f[i] : (T)0);
}

template <typename T>
__global__ void k_init_scale(const T* __restrict__ f, const T* __restrict__ q, const T* __restrict__ u,
                             double* partials, unsigned int* ticket, SolveState* st, size_t n) {
  Acc<T> a0, a1;
  const T d = (T)st->d;
  GRID_STRIDE(i, n) {
    const T qi = q[i];
    a0.add(qi * (d - f[i]));
    a1.add(qi * u[i]);
  }
  Acc<T> v[2] = {a0, a1};
  double tot[2];
  if (grid_reduce<2>(v, partials, ticket, tot)) {
    if (tot[0] > 0.0 && !(tot[1] > 0.0)) {
      // q != 0 (q'(d - f) = |q|^2 > 0) with q'Kq <= 0: K is not positive definite on
      // the cells of q, and the problem has no unique solution
      st->scale = 0.0;
      finish(st, BEM_ENAN);
    } else {
      st->scale = (tot[1] > 0.0) ? tot[0] / tot[1] : 0.0;   // q = 0: no contact at this depth
    }
  }
}

template <typename T>
__global__ void k_init_apply(const T* __restrict__ f, T* __restrict__ q, const T* __restrict__ u,
                             T* __restrict__ p, T* __restrict__ g, const SolveState* st, size_t n) {
  const T s = (T)st->scale;
  const double d = st->d;
  const T dT = (T)d;
  GRID_STRIDE(i, n) {
    p[i] = s * q[i];
    g[i] = s * u[i] + (f[i] - dT);
    q[i] = (T)0;   // q's slot holds the pending pressure changes from here on
  }
}

// Start values for a warm or uniform start: g = f - d (the gap of p = 0) and dp = p,
// so that the first correction gives g = K p + f - d.
template <typename T>
__global__ void k_init_gap(const T* __restrict__ f, const T* __restrict__ p, T* __restrict__ g, T* __restrict__ dp,
                           const SolveState* st, size_t n) {
  const T dT = (T)st->d;
  VEC_LOOP(i4, n) {
    T fv[4], pv[4], gv[4];
    ld4(f, i4, fv);
    ld4(p, i4, pv);
#pragma unroll
    for (int e = 0; e < 4; ++e) gv[e] = fv[e] - dT;
    st4(g, i4, gv);
    st4(dp, i4, pv);
  }
}

// Start of an iteration.
// After a change of the contact set (refresh): the updates moved p by -tau t plus a
// sparse change dp (cells projected to 0 or re-activated since the last correction),
// accumulated in x; with u = K dp the gap becomes g + u, which keeps g a recursively
// updated residual; x counts as cleared (k_pk_update rewrites it from 0).  (When a replacement was scheduled, x holds the
// whole of p and g = f - d, so this recomputes g = K p + f - d from scratch.)
// Without a refresh only a pending load rescale is applied, with x scaled along.
// Either way with the scale s actually applied to p: g = s g' + (s - 1)(d - f), p *= s.
// Then sums over the contact set Ic = {p > 0}: sum g, count, sum g^2, sum u^2, sum p,
// and the set itself as bytes for the sweeps up to the update.
template <typename T>
__global__ void __launch_bounds__(NTHREADS, sizeof(T) == 4 ? 4 : 1) k_pk_begin(T* __restrict__ p, T* __restrict__ g, const T* __restrict__ f, T* __restrict__ dp,
                           const T* __restrict__ u, uint8_t* __restrict__ cm, double* partials,
                           unsigned int* ticket, SolveState* st, size_t n) {
  pdl_enter();
  if (st->done) return;
  const double s = st->scale, d = st->d;
  const T dT = (T)d;
  const bool refresh = st->refresh != 0;
  const bool apply = (!refresh) && (s != 1.0);
  // the gap moves with the scale actually applied to p (the float value of s)
  const T sT = (T)s, s1 = sT - (T)1;
  Acc<T> ag, agg, auu, ap, cnt;
  VEC_LOOP(i4, n) {
    T pv[4], gv[4], fv[4];
    ld4(p, i4, pv);
    ld4(g, i4, gv);
    ld4(f, i4, fv);
    if (refresh) {
      T uv[4];
      ld4(u, i4, uv);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        gv[e] = sT * (gv[e] + uv[e]) + s1 * (dT - fv[e]);
        pv[e] = sT * pv[e];
      }
      st4(p, i4, pv);
      st4(g, i4, gv);
    } else if (apply) {
      T xv[4];
      ld4(dp, i4, xv);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        pv[e] = sT * pv[e];
        gv[e] = sT * gv[e] + s1 * (dT - fv[e]);
        xv[e] = sT * xv[e];     // pending changes scale with p
      }
      st4(p, i4, pv);
      st4(g, i4, gv);
      st4(dp, i4, xv);
    }
    stm4(cm, i4, pv);
    T sg[4], suu[4], sp[4], sc[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool in = pv[e] > (T)0;
      const T ui = gv[e] - (fv[e] - dT);
      sg[e] = in ? gv[e] : (T)0;
      suu[e] = in ? ui * ui : (T)0;
      sp[e] = in ? pv[e] : (T)0;
      sc[e] = in ? (T)1 : (T)0;
    }
    // the gap sums element by element, with exact squares: under force control G is
    // their difference sum g^2 - 2 gbar sum g + n gbar^2, which cancels when the gaps
    // share a large common offset (a depth far off after a replacement, say)
    if (sc[0] + sc[1] + sc[2] + sc[3] > (T)0) {   // groups without a contact cell add nothing
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        ag.add(sg[e]);
        agg.add_sq(sg[e]);
      }
    }
    auu.add4(suu);
    ap.add4(sp);
    cnt.add4(sc);
  }
  Acc<T> v[5] = {ag, cnt, agg, auu, ap};
  double tot[5];
  if (grid_reduce<5>(v, partials, ticket, tot)) {
    st->scale = 1.0;
    st->x_clear = refresh ? 1 : 0;   // x was consumed by this iteration's correction
    st->refresh = 0;
    st->n_c = (int)tot[1];
    if (st->n_c == 0) {
      finish(st, st->control == BEM_CTRL_FORCE ? BEM_ENOCONV : BEM_OK);
      st->res = 0.0;
      return;
    }
    // the shift is applied to the stored gaps in the path precision; d moves by exactly that value
    const double gbar = (st->control == BEM_CTRL_FORCE) ? (double)(T)(tot[0] / tot[1]) : 0.0;
    st->uscale = sqrt(tot[3] / tot[1]);
    st->pscale = tot[4] / tot[1];
    // sum over Ic of (g - gbar)^2 with the shift actually applied (gbar in the path
    // precision), not the mean: written out, so that a rounded shift leaves no error
    double G = tot[2];
    if (st->control == BEM_CTRL_FORCE) {
      G = tot[2] - 2.0 * gbar * tot[0] + tot[1] * gbar * gbar;
      if (isfinite(G)) G = fmax(G, 0.0);
    }
    st->gbar = gbar;
    st->G = G;
    st->res = (tot[3] > 0.0) ? sqrt(G / tot[3]) : 0.0;
    if (!isfinite(G) || !isfinite(st->res)) {
      finish(st, BEM_ENAN);
      return;
    }
    st->replace = 0;
    if (st->res <= st->tol && st->n_neg == 0 && st->n_ol == 0) {
      finish(st, BEM_OK);
      return;
    }
    // Reliable updating: whenever the recursive residual has dropped 100-fold since
    // the gap was last recomputed, recompute it from u = K p (after this step), so the
    // recursion's drift stays at the rounding level of the residual at that point.
    // Not near the tolerance: the recomputed gap carries the product's rounding floor.
    if (st->res <= 1e-2 * st->res_replaced && st->res > 30.0 * st->tol) {
      st->replace = 1;
      st->res_replaced = st->res;
    }
    if (st->iter >= st->max_iter) {
      finish(st, BEM_ENOCONV);
      return;
    }
    // (a previous residual of zero, a level gap, leaves nothing to keep conjugate to)
    st->beta = st->Gold > 0.0 ? st->flag * G / st->Gold : 0.0;
    st->Gold = G;
    st->d += gbar;
  }
}

// Search direction: t = (g - gbar) + beta t on Ic, 0 elsewhere (gbar: force control).
// The shifted gap g - gbar is not stored: k_pk_rt and k_pk_update form the same
// float value from g when they read it, and k_pk_update stores the shifted step.
template <typename T>
__global__ void k_pk_dir(const uint8_t* __restrict__ cm, const T* __restrict__ g, T* __restrict__ t,
                         const SolveState* st, size_t n) {
  pdl_enter();
  if (st->done) return;
  const T gbar = (T)st->gbar, beta = (T)st->beta;
  VEC_LOOP(i4, n) {
    T gv[4], tv[4];
    bool in[4];
    ldm4(cm, i4, in);
    ld4(g, i4, gv);
    ld4(t, i4, tv);
#pragma unroll
    for (int e = 0; e < 4; ++e) tv[e] = in[e] ? (gv[e] - gbar) + beta * tv[e] : (T)0;
    st4(t, i4, tv);
  }
}

// Step length: tau = <g - gbar, t>_Ic / <r - rbar, t>_Ic with r = K t.
template <typename T>
__global__ void __launch_bounds__(NTHREADS, sizeof(T) == 4 ? 6 : 1) k_pk_rt(const uint8_t* __restrict__ cm, const T* __restrict__ g, const T* __restrict__ t,
                        const T* __restrict__ r, double* partials, unsigned int* ticket, SolveState* st, size_t n) {
  pdl_enter();
  if (st->done) return;
  const T gbar = (T)st->gbar;
  Acc<T> art, ar, at, agt, aab;
  VEC_LOOP(i4, n) {
    T gv[4], tv[4], rv[4];
    bool in[4];
    ldm4(cm, i4, in);
    ld4(g, i4, gv);
    ld4(t, i4, tv);
    ld4(r, i4, rv);
    T srt[4], sr[4], st_[4], sgt[4], sab[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      srt[e] = in[e] ? rv[e] * tv[e] : (T)0;
      sr[e] = in[e] ? rv[e] : (T)0;
      st_[e] = in[e] ? tv[e] : (T)0;
      sgt[e] = in[e] ? (gv[e] - gbar) * tv[e] : (T)0;
      sab[e] = in[e] ? fabs(rv[e] * tv[e]) : (T)0;
    }
    art.add4(srt);
    ar.add4(sr);
    at.add4(st_);
    agt.add4(sgt);
    aab.add4(sab);
  }
  Acc<T> v[5] = {art, ar, at, agt, aab};
  double tot[5];
  if (grid_reduce<5>(v, partials, ticket, tot)) {
    const double rbar = (st->control == BEM_CTRL_FORCE) ? tot[1] / (double)st->n_c : 0.0;
    const double den = tot[0] - rbar * tot[2];
    // rounding level of the curvature: the operator product's relative error (float
    // FFT ~1e-6, double ~1e-14) times the sizes of the terms it is formed from
    const double noise = (sizeof(T) == 4 ? 1e-5 : 1e-12) * (tot[4] + fabs(rbar * tot[2]));
    double tau = 0.0;
    if (den == 0.0 && tot[3] == 0.0) {
      // the gap is exactly level on the contact set (a symmetric set under force
      // control): the direction is zero and no step is taken, as in the oracle
    } else if (!isfinite(den) || !isfinite(tot[3]) || den < -noise) {
      finish(st, BEM_ENAN);   // non-finite, or a curvature clearly negative: K is indefinite on the set
      return;
    } else if (!(den > noise)) {
      // a curvature within the product's rounding: the direction is at the noise floor
      // of the path precision; no step is taken and the next direction restarts
      st->restart_next = 1;
    } else {
      tau = tot[3] / den;
      if (!isfinite(tau)) {
        finish(st, BEM_ENAN);
        return;
      }
    }
    // A direction kept conjugate across a small contact-set change may fail to be
    // a descent direction; then no step is taken and the next one restarts.
    if (!(tot[3] > 0.0)) {
      tau = 0.0;
      st->restart_next = 1;
    }
    st->rbar = rbar;
    st->tau = tau;
  }
}

// Update: p -= tau t on Ic with projection to p >= 0; cells outside Ic with a
// negative gap re-enter with p = -tau g; g -= tau K t (g here the shifted gap g - gbar).  When k_pk_begin scheduled a
// replacement of the recursive gap, the step instead leaves x = p and g = f - d, so
// that the next correction computes g = K p + f - d from scratch.
template <typename T>
__global__ void __launch_bounds__(NTHREADS, sizeof(T) == 4 ? 4 : 1) k_pk_update(T* __restrict__ p, T* __restrict__ g, const T* __restrict__ t, const T* __restrict__ r,
                            T* __restrict__ dp, const T* __restrict__ f, double* partials, unsigned int* ticket,
                            SolveState* st, size_t n) {
  pdl_enter();
  if (st->done) return;
  const T tau = (T)st->tau;
  const bool replace = st->replace != 0;
  const bool xz = st->x_clear != 0;   // x consumed this iteration: accumulate from 0
  const T dT = (T)st->d;
  const T gbar = (T)st->gbar;          // the shift of k_pk_dir, applied here to the stored gap
  // Rounding-noise thresholds (float path only): a re-activation needs a gap below
  // -noise * rms(u) and a projection counts as a change of the contact set only when
  // the pressure went below -noise * mean(p).  In double both thresholds are 0.
  const T noise = sizeof(T) == 4 ? (T)(16.0 * 1.1920929e-7) : (T)0;
  const T gthr = -noise * (T)st->uscale, pthr = -noise * (T)st->pscale;
  Acc<T> asum, nneg, nol;
  VEC_LOOP(i4, n) {
    T pv[4], gv[4], tv[4], rv[4], dv[4] = {(T)0, (T)0, (T)0, (T)0};
    ld4(p, i4, pv);
    ld4(g, i4, gv);
    ld4(t, i4, tv);
    ld4(r, i4, rv);
    if (!xz) ld4(dp, i4, dv);
    T cneg[4], col[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const T pi = pv[e], gi = gv[e] - gbar;
      T pn, dpn = dv[e];      // changes not yet applied to g accumulate until the next correction
      cneg[e] = (T)0;
      col[e] = (T)0;
      if (pi > (T)0) {
        pn = pi - tau * tv[e];
        if (pn < (T)0) {
          if (pn < pthr) cneg[e] = (T)1;
          dpn -= pn;          // the projection moves p from pn to 0
          pn = (T)0;
        }
      } else if (gi < gthr) {
        pn = -tau * gi;
        dpn += pn;            // re-activation: p moves from 0 to pn
        col[e] = (T)1;
      } else {
        pn = (T)0;
      }
      pv[e] = pn;
      dv[e] = dpn;
      gv[e] = gi - tau * rv[e];
    }
    asum.add4(pv);
    nneg.add4(cneg);
    nol.add4(col);
    if (replace) {
      T fv[4];
      ld4(f, i4, fv);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        dv[e] = pv[e];
        gv[e] = fv[e] - dT;
      }
    }
    st4(p, i4, pv);
    st4(g, i4, gv);
    st4(dp, i4, dv);
  }
  Acc<T> v[3] = {asum, nneg, nol};
  double tot[3];
  if (grid_reduce<3>(v, partials, ticket, tot)) {
    st->sum_p = tot[0];
    st->n_neg = (int)tot[1];
    st->n_ol = (int)tot[2];
    // Restart of the conjugate directions (steepest-descent step next): when more
    // than kRestartShare of the contact set re-entered in this step, after a step
    // that was not taken, and after a replacement of the gap (below).
    st->flag = (st->n_ol > kRestartShare * st->n_c || st->restart_next) ? 0.0 : 1.0;
    st->restart_next = 0;
    st->refresh = (st->n_neg + st->n_ol > 0 || st->replace) ? 1 : 0;
    st->mv_p_on = st->refresh;
    if (st->replace) st->flag = 0.0;   // the recomputed gap restarts the conjugate directions
    st->iter += 1;
    st->matvecs += 1 + (st->refresh ? 1 : 0);
    if (st->control == BEM_CTRL_FORCE) {
      if (!(tot[0] > 0.0)) {
        finish(st, BEM_ENOCONV);
        return;
      }
      st->scale = st->target / (st->delta2 * tot[0]);
    }
  }
}

// Final statistics from a fresh u = K p: sums over {p > 0} of g, g^2, u^2, count,
// and sum p over all cells.
template <typename T>
__global__ void k_final_stats(const T* __restrict__ p, const T* __restrict__ u, const T* __restrict__ f,
                              double* partials, unsigned int* ticket, double d, double* out, size_t n) {
  const T dT = (T)d;
  Acc<T> ag, agg, auu, ap, cnt;
  GRID_STRIDE(i, n) {
    const T pi = p[i];
    ap.add(pi);
    if (pi != (T)0) {
      const T ui = u[i];
      const T gi = ui + (f[i] - dT);
      ag.add(gi);
      agg.add_sq(gi);
      auu.add(ui * ui);
      cnt.add((T)1);
    }
  }
  Acc<T> v[5] = {ag, agg, auu, cnt, ap};
  double tot[5];
  if (grid_reduce<5>(v, partials, ticket, tot)) {
    for (int s = 0; s < 5; ++s) out[s] = tot[s];
  }
}

// ---------------------------------------------------------------------------
// Adhesive procedure kernels (fixed contact area C, p free in sign)

template <typename T>
__global__ void k_mask_restrict(T* __restrict__ x, const uint8_t* __restrict__ C, size_t n) {
  GRID_STRIDE(i, n) if (!C[i]) x[i] = (T)0;
}

// r = (d - f - K x) on C, s = r; sums |r|^2 and |d - f|^2 over C.
template <typename T>
__global__ void k_lin_init(const T* __restrict__ u, const T* __restrict__ f, const uint8_t* __restrict__ C,
                           T* __restrict__ r, T* __restrict__ s, double* partials, unsigned int* ticket,
                           SolveState* st, size_t n) {
  if (st->status != BEM_OK) return;   // the force-control set-up found no contact area
  const double d = st->d;
  const T dT = (T)d;
  Acc<T> arr, abb;
  GRID_STRIDE(i, n) {
    T ri = (T)0;
    if (C[i]) {
      const T bi = (dT - f[i]);
      ri = bi - u[i];
      arr.add(ri * ri);
      abb.add(bi * bi);
    }
    r[i] = ri;
    s[i] = ri;
  }
  Acc<T> v[2] = {arr, abb};
  double tot[2];
  if (grid_reduce<2>(v, partials, ticket, tot)) {
    st->rr = tot[0];
    st->b2 = tot[1];
    st->res = (tot[1] > 0.0) ? sqrt(tot[0] / tot[1]) : 0.0;
    st->done = 0;
    st->mv_t_on = 1;
    if (tot[1] == 0.0 || st->res <= st->tol) finish(st, BEM_OK);
  }
}

// alpha = <r, r> / <s, K s> on C; under force control also the means of K s and of r
// over C (r is zero-mean in exact arithmetic; its mean is the rounding drift that the
// update removes, so that the residual can fall below the drift's level)
template <typename T>
__global__ void k_lin_alpha(const T* __restrict__ s, const T* __restrict__ q, const T* __restrict__ r,
                            const uint8_t* __restrict__ C, double* partials, unsigned int* ticket, SolveState* st,
                            size_t n) {
  pdl_enter();
  if (st->done) return;
  const bool force = st->control == BEM_CTRL_FORCE;
  Acc<T> a, aq, ar;
  GRID_STRIDE(i, n) if (C[i]) {
    a.add(s[i] * q[i]);
    if (force) {
      aq.add(q[i]);
      ar.add(r[i]);
    }
  }
  Acc<T> v[3] = {a, aq, ar};
  double tot[3];
  if (grid_reduce<3>(v, partials, ticket, tot)) {
    const double alpha = st->rr / tot[0];
    if (!(tot[0] > 0.0) || !isfinite(alpha)) {
      finish(st, BEM_ENAN);
      return;
    }
    st->alpha = alpha;
    st->qbar = force ? (double)(T)(tot[1] / (double)st->n_c) : 0.0;
    st->lin_rbar = force ? (double)(T)(tot[2] / (double)st->n_c) : 0.0;
  }
}

template <typename T>
__global__ void k_lin_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ s, const T* __restrict__ q,
                             const uint8_t* __restrict__ C, double* partials, unsigned int* ticket, SolveState* st,
                             size_t n) {
  pdl_enter();
  if (st->done) return;
  const T alpha = (T)st->alpha;
  const T qbar = (T)st->qbar, rbar = (T)st->lin_rbar;   // 0 under depth control
  Acc<T> arr;
  GRID_STRIDE(i, n) {
    if (C[i]) {
      x[i] += alpha * s[i];
      const T ri = (r[i] - rbar) - alpha * (q[i] - qbar);
      r[i] = ri;
      arr.add(ri * ri);
    }
  }
  Acc<T> v[1] = {arr};
  double tot[1];
  if (grid_reduce<1>(v, partials, ticket, tot)) {
    // force control: the depth moves with the mean of the step's displacement, which
    // keeps the residual d - f - K x at zero mean over C
    if (st->control == BEM_CTRL_FORCE) st->d += st->alpha * st->qbar - st->lin_rbar;
    st->beta = tot[0] / st->rr;
    st->rr = tot[0];
    st->iter += 1;
    st->matvecs += 1;
    st->res = sqrt(tot[0] / st->b2);
    if (!isfinite(st->res)) {
      finish(st, BEM_ENAN);
    } else if (st->res <= st->tol) {
      finish(st, BEM_OK);
    } else if (st->iter >= st->max_iter) {
      finish(st, BEM_ENOCONV);
    }
  }
}

template <typename T>
__global__ void k_lin_dir(const T* __restrict__ r, T* __restrict__ s, const uint8_t* __restrict__ C,
                          const SolveState* st, size_t n) {
  pdl_enter();
  if (st->done) return;
  const T beta = (T)st->beta;
  GRID_STRIDE(i, n) s[i] = C[i] ? r[i] + beta * s[i] : (T)0;
}

// Adhesive force control (Sec. 2 procedure at a given total force F): the fixed-area
// CG runs on the pressures with delta^2 sum_C x = F, the depth d being the multiplier
// of that constraint.  Before each fixed-area solve, x is shifted uniformly on C to
// carry F (x loses pressure outside the area at every area update); after the first
// product, d = mean_C (f + K x), which makes the residual d - f - K x zero-mean on C.
template <typename T>
__global__ void k_lin_force_sum(const T* __restrict__ x, const uint8_t* __restrict__ C, double* partials,
                                unsigned int* ticket, SolveState* st, size_t n) {
  Acc<T> ax, ac;
  GRID_STRIDE(i, n) if (C[i]) {
    ax.add(x[i]);
    ac.add((T)1);
  }
  Acc<T> v[2] = {ax, ac};
  double tot[2];
  if (grid_reduce<2>(v, partials, ticket, tot)) {
    st->n_c = (int)tot[1];
    if (st->n_c == 0) {
      finish(st, BEM_EDETACHED);
      return;
    }
    st->lin_shift = (st->target / st->delta2 - tot[0]) / tot[1];
  }
}

template <typename T>
__global__ void k_lin_force_shift(T* __restrict__ x, const uint8_t* __restrict__ C, const SolveState* st, size_t n) {
  if (st->done) return;
  const T sh = (T)st->lin_shift;
  GRID_STRIDE(i, n) if (C[i]) x[i] += sh;
}

template <typename T>
__global__ void k_lin_force_depth(const T* __restrict__ u, const T* __restrict__ f, const uint8_t* __restrict__ C,
                                  double* partials, unsigned int* ticket, SolveState* st, size_t n) {
  if (st->done) return;
  Acc<T> a;
  GRID_STRIDE(i, n) if (C[i]) a.add(f[i] + u[i]);
  Acc<T> v[1] = {a};
  double tot[1];
  if (grid_reduce<1>(v, partials, ticket, tot)) st->d = (double)(T)(tot[0] / (double)st->n_c);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Contact-area update (Sec. 2): with g = K x + f - d, cells outside C with g < 0
// join; cells of C with a 4-neighbour outside C (window edge = outside) whose
// tension -x exceeds sigma_c (compared in double) leave.  Writes the new mask,
// zeroes x outside it, counts both moves and hashes the new set.
template <typename T>
__global__ void k_detach(T* __restrict__ x, const T* __restrict__ u, const T* __restrict__ f,
                         const uint8_t* __restrict__ C, uint8_t* __restrict__ Cn, int logN, double* partials,
                         unsigned int* ticket, SolveState* st) {
  const int N = 1 << logN;
  const size_t n = (size_t)N * N;
  const double d = st->d, sc = st->sig_c;
  const T dT = (T)d;
  Acc<T> nadd, ndet, ncon, ap, hq[4];
  GRID_STRIDE(i, n) {
    const int r = (int)(i >> logN), c = (int)(i & (N - 1));
    const bool in = C[i] != 0;
    bool out_in = in;
    if (!in) {
      const T gi = u[i] + (f[i] - dT);
      if (gi < (T)0) {
        out_in = true;
        nadd.add((T)1);
      }
    } else {
      const bool inner = (r > 0 && C[i - N]) && (r < N - 1 && C[i + N]) && (c > 0 && C[i - 1]) &&
                         (c < N - 1 && C[i + 1]);
      if (!inner && -(double)x[i] > sc) {
        out_in = false;
        ndet.add((T)1);
      }
    }
    Cn[i] = out_in ? 1 : 0;
    if (!out_in) x[i] = (T)0;
    if (out_in) {
      ncon.add((T)1);
      ap.add(x[i]);
      // order-free set hash: the sum of a 64-bit mix of the member indices, carried as
      // four exact sums of 16-bit digits
      const uint64_t h = mix64((uint64_t)i);
#pragma unroll
      for (int k = 0; k < 4; ++k) hq[k].add((T)(double)((h >> (16 * k)) & 0xffffu));
    }
  }
  Acc<T> v[8] = {nadd, ndet, ncon, ap, hq[0], hq[1], hq[2], hq[3]};
  double tot[8];
  if (grid_reduce<8>(v, partials, ticket, tot)) {
    st->n_add = (int)tot[0];
    st->n_detach = (int)tot[1];
    st->n_c = (int)tot[2];
    st->sum_p = tot[3];
    uint64_t hsh = 0;
    for (int k = 0; k < 4; ++k) hsh += ((uint64_t)tot[4 + k]) << (16 * k);
    st->mask_hash = hsh;
  }
}

// ---------------------------------------------------------------------------


template <typename T>
__global__ void k_fill(T* __restrict__ x, double value, size_t n) {
  GRID_STRIDE(i, n) x[i] = (T)value;
}

// Warm start: p = max(p, 0); under force control the pending rescale s = F/(delta^2 sum p)
// is left in the state for the first gap refresh to apply.
template <typename T>
__global__ void k_init_clamp(T* __restrict__ p, double* partials, unsigned int* ticket, SolveState* st, size_t n) {
  Acc<T> a;
  GRID_STRIDE(i, n) {
    const T v = p[i] > (T)0 ? p[i] : (T)0;
    p[i] = v;
    a.add(v);
  }
  Acc<T> v[1] = {a};
  double tot[1];
  if (grid_reduce<1>(v, partials, ticket, tot)) {
    if (st->control == BEM_CTRL_FORCE) {
      if (tot[0] > 0.0) st->scale = st->target / (st->delta2 * tot[0]);
      else finish(st, BEM_EINVAL);
    }
  }
}

template <typename T>
bem_status read_state(bem_kernel_s* k, cudaStream_t s) {
  BEM_CUDA_TRY(cudaMemcpyAsync(k->ws.state_host, k->ws.state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (k->timing.on) harvest_pass_timing(k);
  return BEM_OK;
}

struct Ctx {
  size_t n;
  int rb, rb6, eb;   // reduction blocks (4 and 6 per SM), element-wise blocks
};

template <typename T>
Ctx ctx_of(const bem_kernel_s* k) {
  Ctx c;
  c.n = (size_t)k->N * k->N;
  c.rb = red_blocks(c.n, 4);
  c.rb6 = red_blocks(c.n, 6);
  c.eb = (int)std::min<size_t>((c.n / 4 + NTHREADS - 1) / NTHREADS, 152 * 8);
  return c;
}

// Final statistics from a fresh u = K p, copied asynchronously to the handle's pinned
// aux_host[0..4]: sums over {p != 0} of g, g^2, u^2, their count, and sum p.
template <typename T>
bem_status final_stats_launch(bem_kernel_s* k, const T* p, double d, cudaStream_t s) {
  const Ctx c = ctx_of<T>(k);
  DV<T> v = dv<T>(k);
  launch_matvec<T>(k, p, v.u, s, nullptr);
  double* dout = k->ws.partials + 12 * RED_MAX_BLOCKS;
  k_final_stats<T><<<c.rb, NTHREADS, 0, s>>>(p, v.u, v.f, k->ws.partials, k->ws.ticket, d, dout, c.n);
  note_launches(1);
  BEM_CUDA_TRY(cudaGetLastError());
  BEM_CUDA_TRY(cudaMemcpyAsync(k->ws.aux_host, dout, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return BEM_OK;
}

// Fills the scalar outputs from aux_host (after the stream has been synchronised).
void fill_result(const bem_kernel_s* k, const bem_problem* prob, double d, bem_status st, bem_result* res) {
  const double* fs = k->ws.aux_host;
  const double delta2 = k->desc.delta * k->desc.delta;
  res->matvecs += 1;
  const double n_c = fs[3];
  double gbar = 0.0;
  if (prob->dgamma == 0.0 && prob->control == BEM_CTRL_FORCE && n_c > 0) gbar = fs[0] / n_c;
  const double G = fmax(fs[1] - n_c * gbar * gbar, 0.0);
  res->err_est = (fs[2] > 0.0) ? sqrt(G / fs[2]) : 0.0;
  res->force = delta2 * fs[4];
  res->depth = d;
  res->n_contact = (int)n_c;
  res->area = delta2 * n_c;
  res->a_eq = sqrt(res->area / M_PI);
  res->status = st;
}

// Initial state and first iterate of the Polonsky-Keer solve (asynchronous on s).
template <typename T>
bem_status pk_setup(bem_kernel_s* k, const bem_problem* prob, const T* pinit, cudaStream_t s) {
  const Ctx c = ctx_of<T>(k);
  DV<T> v = dv<T>(k);
  SolveState* st = k->ws.state;
  SolveState* hs = k->ws.state_host;
  double* part = k->ws.partials;
  unsigned int* tk = k->ws.ticket;
  const bool force = prob->control == BEM_CTRL_FORCE;
  const double delta2 = k->desc.delta * k->desc.delta;

  SolveState init{};
  init.d = force ? 0.0 : prob->target;
  init.Gold = 1.0;
  init.flag = 0.0;
  init.scale = 1.0;
  init.target = prob->target;
  init.delta2 = delta2;
  init.tol = prob->tol;
  init.control = prob->control;
  init.max_iter = prob->max_iter;
  init.n_neg = 1;  // no convergence test passes before one full iteration
  init.res_replaced = 1e300;
  init.loops = 0;
  init.max_loops = prob->max_iter / CHUNK + 2;
  init.status = BEM_OK;
  init.mv_t_on = 1;
  // products outside the iteration: one for the depth-control initial guess, or the
  // first refresh of a warm or uniform start (counted here, run by the first iteration)
  init.matvecs = 1;
  BEM_CUDA_TRY(cudaMemsetAsync(v.t, 0, c.n * sizeof(T), s));
  if (pinit != nullptr || force) {
    init.refresh = 1;
    init.mv_p_on = 1;
  }
  *hs = init;
  BEM_CUDA_TRY(cudaMemcpyAsync(st, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
  if (pinit != nullptr) {
    if (pinit != v.p) BEM_CUDA_TRY(cudaMemcpyAsync(v.p, pinit, c.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    k_init_clamp<T><<<c.rb, NTHREADS, 0, s>>>(v.p, part, tk, st, c.n);
    k_init_gap<T><<<c.eb, NTHREADS, 0, s>>>(v.f, v.p, v.g, v.x, st, c.n);
    note_launches(2);
  } else if (force) {
    k_fill<T><<<c.eb, NTHREADS, 0, s>>>(v.p, prob->target / (delta2 * (double)c.n), c.n);
    k_init_gap<T><<<c.eb, NTHREADS, 0, s>>>(v.f, v.p, v.g, v.x, st, c.n);
    note_launches(2);
  } else {
    k_init_q<T><<<c.eb, NTHREADS, 0, s>>>(v.f, v.x, prob->target, c.n);
    note_launches(1);
    launch_matvec<T>(k, v.x, v.u, s, nullptr);
    k_init_scale<T><<<c.rb, NTHREADS, 0, s>>>(v.f, v.x, v.u, part, tk, st, c.n);
    note_launches(1);
    k_init_apply<T><<<c.eb, NTHREADS, 0, s>>>(v.f, v.x, v.u, v.p, v.g, st, c.n);
    note_launches(1);
  }
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

// CHUNK iterations of the Polonsky-Keer CG as plain launches.  Every launch is
// gated by the device state, so iterations past convergence cost only their
// launch; pointers and problem scalars live in the handle's device memory, which
// makes the sequence independent of the problem and capturable once per handle.
template <typename T>
void pk_chunk_launches(bem_kernel_s* k, cudaStream_t s) {
  const Ctx c = ctx_of<T>(k);
  DV<T> v = dv<T>(k);
  SolveState* st = k->ws.state;
  double* part = k->ws.partials;
  unsigned int* tk = k->ws.ticket;
  uint8_t* cm = k->ws.mask;   // contact set of the iterations (the adhesive masks are not live here)
  for (int it = 0; it < CHUNK; ++it) {
    launch_matvec<T>(k, v.x, v.u, s, &st->mv_p_on);
    launch_pdl(k_pk_begin<T>, c.rb, NTHREADS, 0, s, v.p, v.g, (const T*)v.f, v.x, (const T*)v.u, cm, part, tk, st,
               c.n);
    launch_pdl(k_pk_dir<T>, c.eb, NTHREADS, 0, s, (const uint8_t*)cm, (const T*)v.g, v.t, (const SolveState*)st, c.n);
    launch_matvec<T>(k, v.t, v.r, s, &st->mv_t_on);
    launch_pdl(k_pk_rt<T>, sizeof(T) == 4 ? c.rb6 : c.rb, NTHREADS, 0, s, (const uint8_t*)cm, (const T*)v.g,
               (const T*)v.t, (const T*)v.r, part, tk, st, c.n);
    launch_pdl(k_pk_update<T>, c.rb, NTHREADS, 0, s, v.p, v.g, (const T*)v.t, (const T*)v.r, v.x, (const T*)v.f,
               part, tk, st, c.n);
    note_launches(4);
  }
}

// One chunk: replay of a captured graph of it when the stream allows capture and
// pass timing is off (timing needs events around individual passes); plain launches
// otherwise.  The first chunk of each kind on a handle always runs plainly, so
// one-time kernel attributes are set outside any capture.
template <typename F>
bem_status chunk_graph(const bem_kernel_s* k, cudaStream_t s, cudaGraphExec_t& exec, long long& nodes, int& warm,
                       F&& chunk_launches) {
  const bool capturable = s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
  if (!capturable || k->timing.on || !warm) {
    chunk_launches();
    warm = 1;
    BEM_CUDA_TRY(cudaGetLastError());
    return BEM_OK;
  }
  if (exec == nullptr) {
    cudaGraph_t g = nullptr;
    const long long before = launches();
    BEM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    chunk_launches();
    cudaError_t e = cudaStreamEndCapture(s, &g);
    nodes = launches() - before;
    note_launches(-nodes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  BEM_CUDA_TRY(cudaGraphLaunch(exec, s));
  note_launches(nodes);
  return BEM_OK;
}

template <typename T>
bem_status pk_chunk(bem_kernel_s* k, cudaStream_t s) {
  auto& gr = k->graphs;
  return chunk_graph(k, s, gr.pk_exec, gr.pk_nodes, gr.warm, [&] { pk_chunk_launches<T>(k, s); });
}

// Loop control of the device-side iteration, the condition of a conditional 'while'
// node of a CUDA graph: the next body runs while the solve is unfinished.  A solve
// still running after max_loops bodies stops with BEM_ENOCONV, which bounds the
// loop whatever the CG kernels do.
__global__ void k_loop_ctl(SolveState* st, cudaGraphConditionalHandle h) {
  st->loops += 1;
  if (!st->done && st->loops >= st->max_loops) finish(st, BEM_ENOCONV);
  cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

// Solves up to this iteration limit run the device-side loop; longer ones keep the
// host loop (a state read every chunk), as do traced and pass-timed solves.
constexpr int kDeviceLoopMaxIter = 200000;

bool device_loop(const bem_kernel_s* k, const bem_problem* prob, bool trace) {
  return !k->timing.on && !trace && prob->max_iter <= kDeviceLoopMaxIter;
}

// Adds to graph g a conditional 'while' node whose body is one chunk of k's
// constrained CG followed by the loop control; the body is captured on the library's
// capture stream (nothing runs).  *body_nodes: kernel nodes per body execution.
template <typename T>
bem_status add_loop_node(bem_kernel_s* k, cudaGraph_t g, long long* body_nodes) {
  cudaGraphConditionalHandle h;
  BEM_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  BEM_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs = capture_stream();
  prepare_passes<T>(k);
  const long long before = launches();
  BEM_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  pk_chunk_launches<T>(k, cs);
  k_loop_ctl<<<1, 1, 0, cs>>>(k->ws.state, h);
  note_launches(1);
  const cudaError_t e = cudaStreamEndCapture(cs, &body);
  *body_nodes = launches() - before;
  note_launches(-*body_nodes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture (iteration loop)");
  return BEM_OK;
}

// The handle's whole-solve loop graph, built once.
template <typename T>
bem_status loop_graph(bem_kernel_s* k) {
  auto& gr = k->graphs;
  if (gr.loop_exec != nullptr) return BEM_OK;
  cudaGraph_t g = nullptr;
  BEM_CUDA_TRY(cudaGraphCreate(&g, 0));
  long long nodes = 0;
  bem_status st = add_loop_node<T>(k, g, &nodes);
  if (st == BEM_OK) {
    const cudaError_t e = cudaGraphInstantiate(&gr.loop_exec, g, 0);
    if (e != cudaSuccess) {
      gr.loop_exec = nullptr;
      st = cuda_fail(e, "cudaGraphInstantiate (iteration loop)");
    }
  }
  cudaGraphDestroy(g);
  gr.loop_nodes = nodes;
  return st;
}

// Cache of batch graphs: one graph holds a loop node per instance (no edges between
// them, so the instances run concurrently) and is reused while the same handles, with
// the same captured kernels, come back in the same order.
struct BatchGraph {
  std::vector<uint64_t> key;
  std::vector<const bem_kernel_s*> ks;
  std::vector<long long> nodes;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch_cache;
constexpr size_t kBatchCacheSize = 4;

template <typename T>
bem_status batch_graph(bem_kernel_s* const* ks, const std::vector<int>& idx, cudaGraphExec_t* exec,
                       std::vector<long long>* nodes) {
  std::vector<uint64_t> key;
  for (int i : idx) key.push_back(ks[i]->serial);
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (auto& b : g_batch_cache) {
    if (b.key == key) {
      *exec = b.exec;
      *nodes = b.nodes;
      return BEM_OK;
    }
  }
  cudaGraph_t g = nullptr;
  BEM_CUDA_TRY(cudaGraphCreate(&g, 0));
  BatchGraph b;
  b.key = key;
  bem_status st = BEM_OK;
  for (int i : idx) {
    long long n = 0;
    if ((st = add_loop_node<T>(ks[i], g, &n)) != BEM_OK) break;
    b.ks.push_back(ks[i]);
    b.nodes.push_back(n);
  }
  if (st == BEM_OK) {
    const cudaError_t e = cudaGraphInstantiate(&b.exec, g, 0);
    if (e != cudaSuccess) {
      b.exec = nullptr;
      st = cuda_fail(e, "cudaGraphInstantiate (batch)");
    }
  }
  cudaGraphDestroy(g);
  if (st != BEM_OK) return st;
  if (g_batch_cache.size() >= kBatchCacheSize) {
    cudaGraphExecDestroy(g_batch_cache.front().exec);
    g_batch_cache.erase(g_batch_cache.begin());
  }
  g_batch_cache.push_back(b);
  *exec = b.exec;
  *nodes = b.nodes;
  return BEM_OK;
}

// CHUNK iterations of the fixed-area linear CG (adhesive inner solve), gated by the
// device state like the constrained CG's chunk.
template <typename T>
void lin_chunk_launches(bem_kernel_s* k, const uint8_t* C, cudaStream_t s) {
  const Ctx c = ctx_of<T>(k);
  DV<T> v = dv<T>(k);
  SolveState* st = k->ws.state;
  double* part = k->ws.partials;
  unsigned int* tk = k->ws.ticket;
  for (int it = 0; it < CHUNK; ++it) {
    launch_matvec<T>(k, v.t, v.g, s, &st->mv_t_on);
    launch_pdl(k_lin_alpha<T>, c.rb, NTHREADS, 0, s, (const T*)v.t, (const T*)v.g, (const T*)v.r, C, part, tk, st,
               c.n);
    launch_pdl(k_lin_update<T>, c.rb, NTHREADS, 0, s, v.x, v.r, (const T*)v.t, (const T*)v.g, C, part, tk, st, c.n);
    launch_pdl(k_lin_dir<T>, c.eb, NTHREADS, 0, s, (const T*)v.r, v.t, C, (const SolveState*)st, c.n);
    note_launches(3);
  }
}

template <typename T>
bem_status lin_chunk(bem_kernel_s* k, const uint8_t* C, cudaStream_t s) {
  auto& gr = k->graphs;
  if (gr.lin_exec != nullptr && gr.lin_mask != (const void*)C) {   // captured with another mask array
    BEM_CUDA_TRY(cudaGraphExecDestroy(gr.lin_exec));
    gr.lin_exec = nullptr;
  }
  gr.lin_mask = C;
  return chunk_graph(k, s, gr.lin_exec, gr.lin_nodes, gr.lin_warm, [&] { lin_chunk_launches<T>(k, C, s); });
}

template <typename T>
bem_status run_pk(bem_kernel_s* k, const bem_problem* prob, const T* pinit, cudaStream_t s) {
  bem_status e = pk_setup<T>(k, prob, pinit, s);
  if (e != BEM_OK) return e;
  static const bool trace = getenv("BEM_TRACE") != nullptr;   // diagnostic: residual per chunk on stderr
  if (device_loop(k, prob, trace)) {
    // the whole iteration in one graph launch; one state read at the end
    e = loop_graph<T>(k);
    if (e != BEM_OK) return e;
    BEM_CUDA_TRY(cudaGraphLaunch(k->graphs.loop_exec, s));
    e = read_state<T>(k, s);
    if (e != BEM_OK) return e;
    note_launches((long long)k->ws.state_host->loops * k->graphs.loop_nodes);
    return BEM_OK;
  }
  for (;;) {
    e = pk_chunk<T>(k, s);
    if (e != BEM_OK) return e;
    e = read_state<T>(k, s);
    if (e != BEM_OK) return e;
    const SolveState* hs = k->ws.state_host;
    if (trace)
      fprintf(stderr, "bem: iter %d res %.3e n_c %d neg %d ol %d refresh %d replaced_at %.3e\n", hs->iter, hs->res,
              hs->n_c, hs->n_neg, hs->n_ol, hs->refresh, hs->res_replaced);
    if (hs->done) break;
  }
  return BEM_OK;
}

template <typename T>
bem_status run_adhesive(bem_kernel_s* k, const bem_problem* prob, const T* pinit, uint8_t* mask_dev,
                        int* outer_out, int* iters_out, int* mv_out, double* res_out, double* d_out, cudaStream_t s) {
  const bool force = prob->control == BEM_CTRL_FORCE;
  *d_out = prob->target;
  const Ctx c = ctx_of<T>(k);
  DV<T> v = dv<T>(k);
  SolveState* st = k->ws.state;
  SolveState* hs = k->ws.state_host;
  double* part = k->ws.partials;
  unsigned int* tk = k->ws.ticket;
  uint8_t* C = mask_dev;
  uint8_t* Cn = k->ws.mask + c.n;
  const double delta = k->desc.delta;
  const double Es1 = k->desc.E1 / (1.0 - k->desc.nu1 * k->desc.nu1);
  // Eq. (12): sigma_c = sqrt(E1* dgamma / (0.473201 delta))
  const double sig_c = sqrt(Es1 * prob->dgamma / (0.473201 * delta));

  // x holds the pressure of the fixed-area solve
  if (pinit != nullptr) {
    if (pinit != v.x) BEM_CUDA_TRY(cudaMemcpyAsync(v.x, pinit, c.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  } else {
    BEM_CUDA_TRY(cudaMemsetAsync(v.x, 0, c.n * sizeof(T), s));
  }
  k_mask_restrict<T><<<c.eb, NTHREADS, 0, s>>>(v.x, C, c.n);
  note_launches(1);

  std::unordered_set<uint64_t> seen;
  int iters = 0, mv = 0, outer = 0;
  double res = 0.0;
  const int max_outer = 1000;
  for (outer = 1; outer <= max_outer; ++outer) {
    SolveState init{};
    init.d = force ? *d_out : prob->target;
    init.target = prob->target;
    init.control = prob->control;
    init.tol = prob->tol;
    init.max_iter = prob->max_iter;
    init.sig_c = sig_c;
    init.delta2 = delta * delta;
    init.status = BEM_OK;
    init.mv_t_on = 1;
    *hs = init;
    BEM_CUDA_TRY(cudaMemcpyAsync(st, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    if (force) {   // x carries F on C
      k_lin_force_sum<T><<<c.rb, NTHREADS, 0, s>>>(v.x, C, part, tk, st, c.n);
      k_lin_force_shift<T><<<c.eb, NTHREADS, 0, s>>>(v.x, C, st, c.n);
      note_launches(2);
    }
    // CG on K_CC x = (d - f)_C
    launch_matvec<T>(k, v.x, v.u, s, nullptr);
    if (force) {
      k_lin_force_depth<T><<<c.rb, NTHREADS, 0, s>>>(v.u, v.f, C, part, tk, st, c.n);
      note_launches(1);
    }
    k_lin_init<T><<<c.rb, NTHREADS, 0, s>>>(v.u, v.f, C, v.r, v.t, part, tk, st, c.n);
    note_launches(1);
    mv += 1;
    for (;;) {
      bem_status e = lin_chunk<T>(k, C, s);
      if (e != BEM_OK) return e;
      e = read_state<T>(k, s);
      if (e != BEM_OK) return e;
      if (hs->done) break;
    }
    iters += hs->iter;
    mv += hs->matvecs;
    res = hs->res;
    if (force) *d_out = hs->d;
    if (hs->status != BEM_OK) {
      *outer_out = outer; *iters_out = iters; *mv_out = mv; *res_out = res;
      if (hs->status == BEM_EDETACHED) {
        if (outer == 1) {   // the given starting area was empty
          set_error("force-controlled adhesive solve needs a non-empty starting contact area");
          return BEM_EINVAL;
        }
        set_error("the contact area vanished under the given force");
      }
      return (bem_status)hs->status;
    }
    // area update from the fresh gap
    launch_matvec<T>(k, v.x, v.u, s, nullptr);
    mv += 1;
    k_detach<T><<<c.rb, NTHREADS, 0, s>>>(v.x, v.u, v.f, C, Cn, k->logN, part, tk, st);
    note_launches(1);
    BEM_CUDA_TRY(cudaGetLastError());
    bem_status e = read_state<T>(k, s);
    if (e != BEM_OK) return e;
    if (hs->n_add == 0 && hs->n_detach == 0) break;
    if (!seen.insert(hs->mask_hash).second) {
      *outer_out = outer; *iters_out = iters; *mv_out = mv; *res_out = res;
      set_error("adhesive contact area revisited an earlier state");
      return BEM_ECYCLE;
    }
    BEM_CUDA_TRY(cudaMemcpyAsync(C, Cn, c.n, cudaMemcpyDeviceToDevice, s));
  }
  *outer_out = std::min(outer, max_outer);
  *iters_out = iters;
  *mv_out = mv;
  *res_out = res;
  if (outer > max_outer) {
    set_error("adhesive outer loop did not settle");
    return BEM_ENOCONV;
  }
  return BEM_OK;
}

template <typename T>
__global__ void k_nonfinite(const T* __restrict__ a, const T* __restrict__ b, double* partials, unsigned int* ticket,
                            double* out, size_t n) {
  Acc<T> cnt;
  GRID_STRIDE(i, n) {
    if (!isfinite(a[i])) cnt.add((T)1);
    if (b != nullptr && !isfinite(b[i])) cnt.add((T)1);
  }
  Acc<T> v[1] = {cnt};
  double tot[1];
  if (grid_reduce<1>(v, partials, ticket, tot)) out[0] = tot[0];
}

// Counts non-finite entries of the height map (and warm start) into aux_host[7].
template <typename T>
bem_status nonfinite_launch(bem_kernel_s* k, const T* pinit, cudaStream_t s) {
  const Ctx c = ctx_of<T>(k);
  DV<T> v = dv<T>(k);
  double* dout = k->ws.partials + 12 * RED_MAX_BLOCKS + 7;
  k_nonfinite<T><<<c.rb, NTHREADS, 0, s>>>(v.f, pinit, k->ws.partials, k->ws.ticket, dout, c.n);
  note_launches(1);
  BEM_CUDA_TRY(cudaGetLastError());
  BEM_CUDA_TRY(cudaMemcpyAsync(k->ws.aux_host + 7, dout, sizeof(double), cudaMemcpyDeviceToHost, s));
  return BEM_OK;
}

template <typename T>
bem_status solve_typed(bem_kernel_s* k, const bem_problem* prob, const T* f, const T* pinit, uint8_t* mask,
                       T* p_out, bem_result* res, cudaStream_t s) {
  DV<T> v = dv<T>(k);
  const size_t n = (size_t)k->N * k->N;
  if (f != v.f) BEM_CUDA_TRY(cudaMemcpyAsync(v.f, f, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  *res = bem_result{};
  {
    bem_status e0 = nonfinite_launch<T>(k, pinit, s);
    if (e0 != BEM_OK) return e0;
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (k->ws.aux_host[7] > 0.0) {
      set_error("non-finite value in the height map or the warm start");
      res->status = BEM_ENAN;
      return BEM_ENAN;
    }
  }
  bem_status st = BEM_OK;
  double d = prob->target;
  const T* psol = nullptr;
  if (prob->dgamma > 0.0) {
    int outer = 0, iters = 0, mv = 0;
    double r = 0.0;
    st = run_adhesive<T>(k, prob, pinit, mask, &outer, &iters, &mv, &r, &d, s);
    res->outer_iters = outer;
    res->iters = iters;
    res->matvecs = mv;
    res->residual = r;
    psol = v.x;
  } else {
    st = run_pk<T>(k, prob, pinit, s);
    const SolveState* hs = k->ws.state_host;
    res->iters = hs->iter;
    res->outer_iters = 1;
    res->matvecs = hs->matvecs;
    res->residual = hs->res;
    d = hs->d;
    if (st == BEM_OK) st = (bem_status)hs->status;
    psol = v.p;
  }
  bem_status e = final_stats_launch<T>(k, psol, d, s);
  if (e != BEM_OK) return e;
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  fill_result(k, prob, d, st, res);
  if (p_out != nullptr && p_out != psol)
    BEM_CUDA_TRY(cudaMemcpyAsync(p_out, psol, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  if (st == BEM_ENOCONV) set_error("iteration limit reached before the tolerance");
  if (st == BEM_ENAN) set_error("non-finite or non-positive curvature in CG");
  return st;
}

// Non-adhesive instances solved concurrently: instance i works on strm[i]; each
// round launches one chunk (a graph replay) per unfinished instance and then
// reads every instance's state; the height maps and warm starts are already in
// the handles' f and x slots.
template <typename T>
bem_status batch_typed(int n, bem_kernel_s* const* ks, const bem_problem* probs, const bool* has_pinit,
                       bem_result* res, cudaStream_t const* strm) {
  std::vector<int> active;
  for (int i = 0; i < n; ++i) {
    res[i] = bem_result{};
    bem_status e = nonfinite_launch<T>(ks[i], has_pinit[i] ? dv<T>(ks[i]).x : nullptr, strm[i]);
    if (e != BEM_OK) return e;
  }
  for (int i = 0; i < n; ++i) BEM_CUDA_TRY(cudaStreamSynchronize(strm[i]));
  for (int i = 0; i < n; ++i) {
    if (ks[i]->ws.aux_host[7] > 0.0) {
      res[i].status = BEM_ENAN;
      continue;
    }
    bem_status e = pk_setup<T>(ks[i], &probs[i], has_pinit[i] ? dv<T>(ks[i]).x : nullptr, strm[i]);
    if (e != BEM_OK) return e;
    active.push_back(i);
  }
  std::vector<int> next, finished;
  bool device = !active.empty();
  for (int i : active) device = device && device_loop(ks[i], &probs[i], false);
  if (device) {
    // one graph launch runs every instance's iteration loop on the device
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> nodes;
    bem_status e = batch_graph<T>(ks, active, &exec, &nodes);
    if (e != BEM_OK) return e;
    cudaStream_t s0 = strm[active[0]];
    for (int i : active) {
      BEM_CUDA_TRY(cudaEventRecord(ks[i]->ws.done_ev, strm[i]));
      BEM_CUDA_TRY(cudaStreamWaitEvent(s0, ks[i]->ws.done_ev, 0));
    }
    BEM_CUDA_TRY(cudaGraphLaunch(exec, s0));
    BEM_CUDA_TRY(cudaEventRecord(ks[active[0]]->ws.done_ev, s0));
    for (int i : active) {
      if (strm[i] != s0) BEM_CUDA_TRY(cudaStreamWaitEvent(strm[i], ks[active[0]]->ws.done_ev, 0));
      BEM_CUDA_TRY(cudaMemcpyAsync(ks[i]->ws.state_host, ks[i]->ws.state, sizeof(SolveState),
                                   cudaMemcpyDeviceToHost, strm[i]));
    }
    for (int i : active) BEM_CUDA_TRY(cudaStreamSynchronize(strm[i]));
    for (size_t a = 0; a < active.size(); ++a) {
      const int i = active[a];
      note_launches((long long)ks[i]->ws.state_host->loops * nodes[a]);
      finished.push_back(i);
    }
    active.clear();
  }
  while (!active.empty()) {
    for (int i : active) {
      bem_kernel_s* k = ks[i];
      bem_status e = pk_chunk<T>(k, strm[i]);
      if (e != BEM_OK) return e;
      BEM_CUDA_TRY(cudaMemcpyAsync(k->ws.state_host, k->ws.state, sizeof(SolveState), cudaMemcpyDeviceToHost,
                                   strm[i]));
      BEM_CUDA_TRY(cudaEventRecord(k->ws.done_ev, strm[i]));
    }
    next.clear();
    for (int i : active) {
      BEM_CUDA_TRY(cudaEventSynchronize(ks[i]->ws.done_ev));
      if (ks[i]->timing.on) harvest_pass_timing(ks[i]);
      if (ks[i]->ws.state_host->done) finished.push_back(i);
      else next.push_back(i);
    }
    active.swap(next);
  }
  for (int i : finished) {
    const SolveState* hs = ks[i]->ws.state_host;
    res[i].iters = hs->iter;
    res[i].outer_iters = 1;
    res[i].matvecs = hs->matvecs;
    res[i].residual = hs->res;
    res[i].status = hs->status;
    bem_status e = final_stats_launch<T>(ks[i], dv<T>(ks[i]).p, hs->d, strm[i]);
    if (e != BEM_OK) return e;
  }
  for (int i : finished) BEM_CUDA_TRY(cudaStreamSynchronize(strm[i]));
  for (int i : finished) {
    const SolveState* hs = ks[i]->ws.state_host;
    fill_result(ks[i], &probs[i], hs->d, (bem_status)hs->status, &res[i]);
  }
  return BEM_OK;
}

}  // namespace

void release_batch_graph(const bem_kernel_s* k) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (size_t b = 0; b < g_batch_cache.size();) {
    auto& ks = g_batch_cache[b].ks;
    if (std::find(ks.begin(), ks.end(), k) != ks.end()) {
      cudaGraphExecDestroy(g_batch_cache[b].exec);
      g_batch_cache.erase(g_batch_cache.begin() + b);
    } else {
      ++b;
    }
  }
}

bem_status solve_batch_device(int n, bem_kernel_s* const* ks, const bem_problem* probs, const bool* has_pinit,
                              bem_result* res, cudaStream_t const* strm) {
  if (n == 0) return BEM_OK;
  if (ks[0]->prec == BEM_FP64) return batch_typed<double>(n, ks, probs, has_pinit, res, strm);
  return batch_typed<float>(n, ks, probs, has_pinit, res, strm);
}

bem_status solve_contact_device(bem_kernel_s* k, const bem_problem* prob, const void* f, const void* pinit,
                                uint8_t* mask, void* p_out, bem_result* res, cudaStream_t s) {
  if (k->prec == BEM_FP64)
    return solve_typed<double>(k, prob, (const double*)f, (const double*)pinit, mask, (double*)p_out, res, s);
  return solve_typed<float>(k, prob, (const float*)f, (const float*)pinit, mask, (float*)p_out, res, s);
}

}  // namespace bem
