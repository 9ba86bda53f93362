// Column-pivoted Householder QR of the small sketch W (l x n, FP64) and the
// solve for the interpolation matrix P.
//
// Algorithm 4 steps 4-8 (transposed): k pivots of a column-pivoted QR of W
// select the skeleton J; C = R11^{-1} R12 by back-substitution; P(:,J) = I,
// P(:,Jc) = C.  The paper's QR is pivoted modified Gram-Schmidt (mgsqr,
// Sec. 2.4); Householder reflections with the same pivot rule give the same
// pivots and R in exact arithmetic and are the stabler choice.
//
// Pivot rule: the largest residual column norm ||W^(s)(s:, j)||, recomputed
// from the updated matrix at every step (no downdating) and compared as its
// square, ties to the lowest column index.
//
// n <= 1024 (cpqr_cluster_kernel): a cluster of 8 CTAs x 128 threads, one
// column per thread held in registers for the whole factorization.  Per
// step, each CTA's best candidate and then the pivot column are published in
// its shared memory and read by the other CTAs through distributed shared
// memory (two cluster barriers per step, double-buffered slots).
// Larger n, or l > 64 rows (cpqr_small_kernel, up to 96 rows): one CTA of 1024
// threads works in place on a copy of W held row-major in global memory
// (L2-resident); thread t owns columns t, t + 1024, ...
// In both, norms and the argmax use warp shuffles and fixed-order sums, and
// the reflector of the pivot column is formed by one warp.
#include <cooperative_groups.h>
#include <float.h>

#include "cta_qr.cuh"
#include "idsk_internal.h"

namespace cg = cooperative_groups;

namespace idsk {
namespace {

using qr::ArgMax;
using qr::better;
using qr::warp_argmax;
using qr::warp_sum;

constexpr int NT = 1024;
constexpr int QMAX = 32;   // columns per thread -> n <= 32768

__global__ void __launch_bounds__(NT, 1)
cpqr_small_kernel(double* __restrict__ M, int rows, int n, int ld, int k, double tol_factor,
                  double* __restrict__ R, int* __restrict__ J, int* __restrict__ colpos,
                  int* __restrict__ kout) {
  __shared__ qr::QrShared sh;
  qr::cta_pivoted_qr<NT>(M, rows, n, ld, k, tol_factor, R, J, colpos, kout, sh);
}


constexpr int CL_CTAS = 8, CL_THREADS = 128;   // cluster kernel: n <= 1024

__device__ __forceinline__ void cpqr_cluster_body(const double* __restrict__ M, int rows, int n,
                                                  int ld, int k, double tol_factor,
                                                  double* __restrict__ R, int* __restrict__ J,
                                                  int* __restrict__ colpos,
                                                  int* __restrict__ kout) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ ArgMax cand[2];              // this CTA's best candidate (by step parity)
  __shared__ double pcol[2][kLMax];       // pivot column, published by its owner CTA
  __shared__ double fro_cta;
  __shared__ ArgMax wred[CL_THREADS / 32];
  __shared__ double fred[CL_THREADS / 32];
  __shared__ double vs[kLMax];
  __shared__ double sh_tau, sh_beta;
  const int rank = (int)cl.block_rank();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int j = rank * CL_THREADS + t;
  const bool have = j < n;
  const int kmax = min(k, min(rows, n));
  double c[kLMax];
#pragma unroll
  for (int i = 0; i < kLMax; ++i) c[i] = (have && i < rows) ? M[(int64_t)i * ld + j] : 0.0;
  if (have) colpos[j] = -1;
  bool piv = false;

  // ||W||_F: rows in order per column, then warps, then CTAs in rank order
  {
    double ss = 0.0;
#pragma unroll
    for (int i = 0; i < kLMax; ++i) ss += c[i] * c[i];
    ss = warp_sum(ss);
    if (lane == 0) fred[warp] = ss;
    __syncthreads();
    if (t == 0) {
      double a = 0.0;
      for (int w = 0; w < CL_THREADS / 32; ++w) a += fred[w];
      fro_cta = a;
    }
  }
  cl.sync();
  double fro2 = 0.0;
  for (int r = 0; r < CL_CTAS; ++r) fro2 += *cl.map_shared_rank(&fro_cta, r);
  const double tol = tol_factor * DBL_EPSILON * sqrt(fro2);

  int s = 0;
  for (; s < kmax; ++s) {
    const int b = s & 1;
    // residual norm of this thread's column, rows s.. in order
    ArgMax best{-1.0, 0x7fffffff};
    if (have && !piv) {
      double ss = 0.0;
#pragma unroll
      for (int i = 0; i < kLMax; ++i)
        if (i >= s && i < rows) ss += c[i] * c[i];
      best = ArgMax{ss, j};
    }
    best = warp_argmax(best);
    if (lane == 0) wred[warp] = best;
    __syncthreads();
    if (t == 0) {
      ArgMax a = wred[0];
      for (int w = 1; w < CL_THREADS / 32; ++w) a = better(a, wred[w]);
      cand[b] = a;
    }
    cl.sync();   // candidates published
    ArgMax g = *cl.map_shared_rank(&cand[b], 0);
    for (int r = 1; r < CL_CTAS; ++r) g = better(g, *cl.map_shared_rank(&cand[b], r));
    if (!(g.v > tol * tol)) break;   // uniform over the cluster
    const int p = g.i;
    if (j == p) {
#pragma unroll
      for (int i = 0; i < kLMax; ++i) pcol[b][i] = c[i];
    }
    cl.sync();   // pivot column published
    if (warp == 0) {   // Householder reflector of the pivot column, rows s..rows-1
      const double* pc = cl.map_shared_rank(&pcol[b][0], p / CL_THREADS);
      const int len = rows - s;
      const double x0 = (lane < len) ? pc[s + lane] : 0.0;
      const double x1 = (lane + 32 < len) ? pc[s + lane + 32] : 0.0;
      const double alpha = __shfl_sync(0xffffffffu, x0, 0);
      const double sigma = warp_sum((lane == 0 ? 0.0 : x0 * x0) + x1 * x1);
      double tau = 0.0, beta = alpha, scale = 0.0;
      if (sigma != 0.0) {
        const double nrm = sqrt(alpha * alpha + sigma);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = alpha - beta;
      }
      if (lane < len) vs[lane] = lane == 0 ? 1.0 : (sigma != 0.0 ? x0 / scale : 0.0);
      if (lane + 32 < len) vs[lane + 32] = sigma != 0.0 ? x1 / scale : 0.0;
      if (lane == 0) {
        sh_tau = tau;
        sh_beta = beta;
        if (rank == 0) {
          J[s] = p;
          colpos[p] = s;
        }
      }
    }
    __syncthreads();
    if (have) {
      double rsj;
      if (j == p) {
        piv = true;
        rsj = sh_beta;
      } else if (piv) {
        rsj = 0.0;
      } else {
        const double tau = sh_tau;
        if (tau != 0.0) {
          double d = 0.0;
#pragma unroll
          for (int i = 0; i < kLMax; ++i)
            if (i >= s && i < rows) d += vs[i - s] * c[i];
          const double td = tau * d;
#pragma unroll
          for (int i = 0; i < kLMax; ++i)
            if (i >= s && i < rows) c[i] -= td * vs[i - s];
        }
#pragma unroll
        for (int i = 0; i < kLMax; ++i)
          if (i == s) rsj = c[i];
      }
      R[(int64_t)s * n + j] = rsj;
    }
  }
  if (rank == 0) {
    if (t == 0) *kout = s;
    for (int q = s + t; q < k; q += CL_THREADS) J[q] = -1;
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

__global__ void __cluster_dims__(CL_CTAS, 1, 1) __launch_bounds__(CL_THREADS, 1)
    cpqr_cluster_kernel(const double* __restrict__ M, int rows, int n, int ld, int k,
                        double tol_factor, double* __restrict__ R, int* __restrict__ J,
                        int* __restrict__ colpos, int* __restrict__ kout) {
  cpqr_cluster_body(M, rows, n, ld, k, tol_factor, R, J, colpos, kout);
}


// P(:, j) for every column j: e_u when j = J[u]; otherwise the solution of
// R11 x = R(:, j) by back-substitution, R11(t, u) = R(t, J[u]).  One warp per
// column, column-oriented: x_t = b_t / R11(t, t) (by the diagonal's
// reciprocal, formed once per block), then b_u -= R11(u, t) x_t
// for u < t, lane u holding b_u and b_{u+32}.  R11 lives in shared memory.
constexpr int SP_WARPS = 8;
__device__ __forceinline__ void solve_p_body(const double* __restrict__ R,
                                             const int* __restrict__ J,
                                             const int* __restrict__ colpos,
                                             const int* __restrict__ kout, int k, int n,
                                             double* __restrict__ P, int cblock) {
  extern __shared__ double r11[];   // kk x kk, row-major
  __shared__ int Js[kLMaxW];
  __shared__ double rdiag[kLMaxW];   // 1 / R11(t, t)
  const int kk = qr::solve_setup(R, J, kout, n, r11, Js, rdiag);
  const int j = cblock * SP_WARPS + (threadIdx.x >> 5);
  if (j < n) qr::solve_column(j, R, colpos, k, kk, n, P, r11, rdiag);
}

__global__ void __launch_bounds__(SP_WARPS * 32) solve_p_kernel(
    const double* __restrict__ R, const int* __restrict__ J, const int* __restrict__ colpos,
    const int* __restrict__ kout, int k, int n, double* __restrict__ P) {
  solve_p_body(R, J, colpos, kout, k, n, P, blockIdx.x);
}


}  // namespace

// one_cta: the one-CTA kernel whatever the size (the QR then occupies a
// single SM, beside the coarse QR that id_factor starts on a side stream).
cudaError_t launch_cpqr_small(double* M, int rows, int n, int ld, int k, double tol_factor,
                              double* R, int* J, int* colpos, int* kout, cudaStream_t st,
                              bool one_cta) {
  if (n > NT * QMAX || rows > kLMaxW || k > kLMaxW) return cudaErrorInvalidValue;
  if (!one_cta && n <= CL_CTAS * CL_THREADS && rows <= kLMax)   // cluster: a column in registers
    cpqr_cluster_kernel<<<CL_CTAS, CL_THREADS, 0, st>>>(M, rows, n, ld, k, tol_factor, R, J,
                                                        colpos, kout);
  else
    cpqr_small_kernel<<<1, NT, 0, st>>>(M, rows, n, ld, k, tol_factor, R, J, colpos, kout);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_solve_p(const double* R, const int* J, const int* colpos, const int* kout,
                           int k, int n, double* P, cudaStream_t st) {
  const size_t sm = sizeof(double) * (size_t)k * k;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(solve_p_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  solve_p_kernel<<<(n + SP_WARPS - 1) / SP_WARPS, SP_WARPS * 32, sm, st>>>(R, J, colpos, kout, k,
                                                                         n, P);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace idsk
