// One-CTA pivoted QR of a small row-major matrix held in global memory and
// the solve for the interpolation matrix P (Algorithm 4 steps 4-8,
// transposed).  Used by the pivoted-QR kernels and by the batched sketch
// kernel, which finishes each matrix of a batch in the CTA that completes its
// last work item.
#pragma once

#include <float.h>

#include "idsk_internal.h"

namespace idsk {
namespace qr {

constexpr int kQrCols = 32;   // columns per thread at most (pivot bit mask)

struct ArgMax {
  double v;
  int i;
};

__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

__device__ __forceinline__ ArgMax warp_argmax(ArgMax a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax b;
    b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
    b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
    a = better(a, b);
  }
  return a;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared scratch of cta_pivoted_qr (up to 1024 threads).
struct QrShared {
  ArgMax red[32];
  double vs[kLMaxW];
  double fro_part[32];
  double tau, beta, tol;
  int p, stop;
};

// Column-pivoted Householder QR of M (rows x n, leading dimension ld, rows
// <= 96) by the NT threads of one CTA, in place: thread t owns columns t,
// t + NT, ... (n <= 32 NT).  k pivots at most; stops early below the rank
// tolerance tol_factor * eps * ||M||_F.  Writes R (k x n), J (k, -1 past
// k_out), colpos (n: pivot position or -1) and *kout.
template <int NT>
__device__ __forceinline__ void cta_pivoted_qr(double* __restrict__ M, int rows, int n, int ld,
                                               int k, double tol_factor, double* __restrict__ R,
                                               int* __restrict__ J, int* __restrict__ colpos,
                                               int* __restrict__ kout, QrShared& sh) {
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps, at most 32");
  ArgMax* red = sh.red;
  double* vs = sh.vs;
  double* fro_part = sh.fro_part;
  double& sh_tau = sh.tau;
  double& sh_beta = sh.beta;
  double& sh_tol = sh.tol;
  int& sh_p = sh.p;
  int& sh_stop = sh.stop;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int kmax = min(k, min(rows, n));
  uint32_t pivoted = 0u;   // bit q: column t + q*NT was pivoted

  // ||M||_F for the rank tolerance
  {
    double ss = 0.0;
    for (int q = 0; q < kQrCols; ++q) {
      const int j = t + q * NT;
      if (j >= n) break;
      for (int i = 0; i < rows; ++i) {
        const double x = M[(int64_t)i * ld + j];
        ss += x * x;
      }
      colpos[j] = -1;
    }
    ss = warp_sum(ss);
    if (lane == 0) fro_part[warp] = ss;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += fro_part[w];
      sh_tol = tol_factor * DBL_EPSILON * sqrt(s);
    }
    __syncthreads();
  }

  int s = 0;
  for (; s < kmax; ++s) {
    // residual norms of the non-pivoted columns
    ArgMax best{-1.0, 0x7fffffff};
    for (int q = 0; q < kQrCols; ++q) {
      const int j = t + q * NT;
      if (j >= n) break;
      if (pivoted & (1u << q)) continue;
      double ss = 0.0;
      for (int i = s; i < rows; ++i) {
        const double x = M[(int64_t)i * ld + j];
        ss += x * x;
      }
      best = better(best, ArgMax{ss, j});
    }
    best = warp_argmax(best);
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (warp == 0) {
      ArgMax b = lane < NT / 32 ? red[lane] : ArgMax{-1.0, 0x7fffffff};
      b = warp_argmax(b);
      if (lane == 0) {
        sh_p = b.i;
        sh_stop = !(b.v > sh_tol * sh_tol);
      }
    }
    __syncthreads();
    if (sh_stop) break;
    const int p = sh_p;
    // Householder reflector of the pivot column, rows s..rows-1 (one warp;
    // lane holds rows s + lane, s + lane + 32, s + lane + 64)
    if (warp == 0) {
      const int len = rows - s;
      double x0 = (lane < len) ? M[(int64_t)(s + lane) * ld + p] : 0.0;
      double x1 = (lane + 32 < len) ? M[(int64_t)(s + lane + 32) * ld + p] : 0.0;
      double x2 = (lane + 64 < len) ? M[(int64_t)(s + lane + 64) * ld + p] : 0.0;
      const double alpha = __shfl_sync(0xffffffffu, x0, 0);
      const double sigma = warp_sum((lane == 0 ? 0.0 : x0 * x0) + x1 * x1 + x2 * x2);
      double tau = 0.0, beta = alpha, scale = 0.0;
      if (sigma != 0.0) {
        const double nrm = sqrt(alpha * alpha + sigma);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = alpha - beta;
      }
      if (lane < len) vs[lane] = lane == 0 ? 1.0 : (sigma != 0.0 ? x0 / scale : 0.0);
      if (lane + 32 < len) vs[lane + 32] = sigma != 0.0 ? x1 / scale : 0.0;
      if (lane + 64 < len) vs[lane + 64] = sigma != 0.0 ? x2 / scale : 0.0;
      if (lane == 0) {
        sh_tau = tau;
        sh_beta = beta;
        J[s] = p;
        colpos[p] = s;
      }
    }
    __syncthreads();
    const double tau = sh_tau;
    // apply H = I - tau v v^T to the other non-pivoted columns; emit row s of R
    for (int q = 0; q < kQrCols; ++q) {
      const int j = t + q * NT;
      if (j >= n) break;
      double rsj;
      if (j == p) {
        pivoted |= (1u << q);
        rsj = sh_beta;
      } else if (pivoted & (1u << q)) {
        rsj = 0.0;
      } else {
        if (tau != 0.0) {
          double d = 0.0;
          for (int i = s; i < rows; ++i) d += vs[i - s] * M[(int64_t)i * ld + j];
          const double td = tau * d;
          for (int i = s; i < rows; ++i) M[(int64_t)i * ld + j] -= td * vs[i - s];
        }
        rsj = M[(int64_t)s * ld + j];
      }
      R[(int64_t)s * n + j] = rsj;
    }
    __syncthreads();
  }
  if (t == 0) *kout = s;
  for (int q = s + t; q < k; q += NT) J[q] = -1;
}

// P's solve, shared part: J, R11 = R(:, J) (row-major k_out x k_out) and the
// reciprocals of its diagonal into shared memory (the whole CTA).
__device__ __forceinline__ int solve_setup(const double* __restrict__ R, const int* __restrict__ J,
                                           const int* __restrict__ kout, int n, double* r11,
                                           int* Js, double* rdiag) {
  const int kk = *kout;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) Js[e] = J[e];
  __syncthreads();
  for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) {
    const int tt = e / kk, u = e % kk;
    r11[e] = R[(int64_t)tt * n + Js[u]];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk; e += blockDim.x) rdiag[e] = 1.0 / r11[e * kk + e];
  __syncthreads();
  return kk;
}

// Column j of P by one warp: e_u when j = J[u]; otherwise the solution of
// R11 x = R(:, j) by back-substitution, column-oriented: x_t = b_t / R11(t, t)
// (by the diagonal's reciprocal), then b_u -= R11(u, t) x_t for u < t, lane
// u holding b_u, b_{u+32}, b_{u+64} (k_out <= 96).  Rows past k_out are 0.
__device__ __forceinline__ void solve_column(int j, const double* __restrict__ R,
                                             const int* __restrict__ colpos, int k, int kk, int n,
                                             double* __restrict__ P, const double* r11,
                                             const double* rdiag) {
  const int lane = threadIdx.x & 31;
  const int cp = colpos[j];
  if (cp >= 0) {
    for (int tt = lane; tt < k; tt += 32) P[(int64_t)tt * n + j] = (tt == cp) ? 1.0 : 0.0;
    return;
  }
  double b0 = lane < kk ? R[(int64_t)lane * n + j] : 0.0;
  double b1 = lane + 32 < kk ? R[(int64_t)(lane + 32) * n + j] : 0.0;
  double b2 = lane + 64 < kk ? R[(int64_t)(lane + 64) * n + j] : 0.0;
  for (int tt = kk - 1; tt >= 0; --tt) {
    const double bt = __shfl_sync(0xffffffffu, tt < 32 ? b0 : (tt < 64 ? b1 : b2), tt & 31);
    const double xt = bt * rdiag[tt];
    if (lane == (tt & 31)) {
      if (tt < 32)
        b0 = xt;
      else if (tt < 64)
        b1 = xt;
      else
        b2 = xt;
    }
    if (lane < tt) b0 -= r11[lane * kk + tt] * xt;
    if (lane + 32 < tt) b1 -= r11[(lane + 32) * kk + tt] * xt;
    if (lane + 64 < tt) b2 -= r11[(lane + 64) * kk + tt] * xt;
  }
  for (int tt = lane; tt < k; tt += 32)
    P[(int64_t)tt * n + j] = tt < kk ? (tt < 32 ? b0 : (tt < 64 ? b1 : b2)) : 0.0;
}

}  // namespace qr
}  // namespace idsk
