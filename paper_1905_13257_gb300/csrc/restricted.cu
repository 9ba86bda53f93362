// ID of the sketch W (l x n) whose skeleton is chosen among candidate
// columns (the learned proposal's candidates): the pivoted QR of W(:, cand)
// gives J (cpqr.cu), and P over all n columns is the least-squares fit of W
// on W(:, J), which for a pivoted QR equals R11^-1 R12 (Sec. 2.4), with
// P(:, J) = I exactly.
//
//   gather_cols_kernel   Wc = W(:, cand), row-major l x ncand
//   map_pivots_kernel    J[u] = cand[Jc[u]] for the k_out pivots, -1 after
//   fixed_qr_kernel      one CTA: Householder QR of W(:, J) without pivoting
//                        (LAPACK dlarfg convention), reflectors V, tau, R
//   fixed_apply_kernel   one thread per column: apply the reflectors, solve
//                        with R; the columns of J get unit columns of P
// FP64 throughout; every sum runs in a fixed order.
#include <math.h>

#include "idsk_internal.h"

namespace idsk {
namespace {

constexpr int FQ_ROWS = 64;   // l <= kLMax

__global__ void gather_cols_kernel(const double* __restrict__ W, int64_t ldw, int l,
                                   const int* __restrict__ cand, int ncand,
                                   double* __restrict__ Wc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)l * ncand) return;
  const int i = (int)(e / ncand), q = (int)(e - (int64_t)i * ncand);
  Wc[e] = W[(int64_t)i * ldw + cand[q]];
}

__global__ void map_pivots_kernel(const int* __restrict__ Jc, const int* __restrict__ cand,
                                  const int* __restrict__ kout, int k, int* __restrict__ J) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= k) return;
  J[u] = u < *kout ? cand[Jc[u]] : -1;
}

// blockDim.x == FQ_ROWS: thread i owns row i.  V: l x k, column t at V + t l;
// R: k x k row-major.
__global__ void __launch_bounds__(FQ_ROWS) fixed_qr_kernel(const double* __restrict__ W,
                                                           int64_t ldw, int l,
                                                           const int* __restrict__ J,
                                                           const int* __restrict__ kout, int k,
                                                           double* __restrict__ V,
                                                           double* __restrict__ tau,
                                                           double* __restrict__ R) {
  __shared__ double a[FQ_ROWS][FQ_ROWS + 1];
  __shared__ double red[FQ_ROWS];
  __shared__ double sc[3];
  __shared__ double wsh;
  const int i = threadIdx.x;
  const int kk = *kout;
  for (int c = 0; c < kk; ++c) a[i][c] = i < l ? W[(int64_t)i * ldw + J[c]] : 0.0;
  __syncthreads();
  for (int t = 0; t < kk; ++t) {
    red[i] = (i > t && i < l) ? a[i][t] * a[i][t] : 0.0;
    __syncthreads();
    if (i == 0) {
      double sigma = 0.0;
      for (int r = 0; r < FQ_ROWS; ++r) sigma += red[r];
      const double alpha = a[t][t];
      double tv = 0.0, beta = alpha, scale = 0.0;
      if (sigma != 0.0) {
        const double nrm = sqrt(alpha * alpha + sigma);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tv = (beta - alpha) / beta;
        scale = alpha - beta;
      }
      sc[0] = tv;
      sc[1] = beta;
      sc[2] = scale;
    }
    __syncthreads();
    const double tv = sc[0], scale = sc[2];
    double vi = 0.0;
    if (i == t)
      vi = 1.0;
    else if (i > t && i < l && scale != 0.0)
      vi = a[i][t] / scale;
    if (i < l) V[(int64_t)t * l + i] = vi;
    if (i == 0) {
      tau[t] = tv;
      R[(int64_t)t * k + t] = sc[1];
    }
    for (int c = t + 1; c < kk; ++c) {
      red[i] = vi * a[i][c];
      __syncthreads();
      if (i == 0) {
        double w = 0.0;
        for (int r = 0; r < FQ_ROWS; ++r) w += red[r];
        wsh = w;
      }
      __syncthreads();
      a[i][c] -= tv * wsh * vi;
      if (i == t) R[(int64_t)t * k + c] = a[i][c];
      __syncthreads();
    }
  }
}

// Shared memory: V (kk x l), tau (kk), R (kk rows of k).
__global__ void fixed_apply_kernel(const double* __restrict__ W, int64_t ldw, int l, int n,
                                   const double* __restrict__ V, const double* __restrict__ tau,
                                   const double* __restrict__ R, const int* __restrict__ J,
                                   const int* __restrict__ kout, int k, double* __restrict__ P) {
  extern __shared__ double fsm[];
  const int kk = *kout;
  double* Vs = fsm;
  double* ts = Vs + (size_t)k * l;
  double* Rs = ts + k;
  for (int e = threadIdx.x; e < kk * l; e += blockDim.x) Vs[e] = V[e];
  for (int e = threadIdx.x; e < kk; e += blockDim.x) ts[e] = tau[e];
  for (int e = threadIdx.x; e < kk * k; e += blockDim.x) Rs[e] = R[e];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double x[FQ_ROWS];
  for (int i = 0; i < FQ_ROWS; ++i) x[i] = i < l ? W[(int64_t)i * ldw + j] : 0.0;
  for (int t = 0; t < kk; ++t) {   // x = H_t x, rows t..l-1
    const double* v = Vs + (size_t)t * l;
    double d = 0.0;
    for (int i = t; i < l; ++i) d += v[i] * x[i];
    const double td = ts[t] * d;
    for (int i = t; i < l; ++i) x[i] -= td * v[i];
  }
  for (int t = kk - 1; t >= 0; --t) {   // R11 y = (Q^T w)(0:kk)
    double s = x[t];
    for (int c = t + 1; c < kk; ++c) s -= Rs[(size_t)t * k + c] * x[c];
    x[t] = s / Rs[(size_t)t * k + t];
  }
  int pos = -1;
  for (int u = 0; u < kk; ++u)
    if (J[u] == j) pos = u;
  for (int t = 0; t < k; ++t) {
    double v = 0.0;
    if (t < kk) v = pos >= 0 ? (t == pos ? 1.0 : 0.0) : x[t];
    P[(int64_t)t * n + j] = v;
  }
}

}  // namespace

cudaError_t launch_gather_cols(const double* W, int64_t ldw, int l, const int* cand, int ncand,
                               double* Wc, cudaStream_t st) {
  const int64_t tot = (int64_t)l * ncand;
  gather_cols_kernel<<<(int)((tot + 255) / 256), 256, 0, st>>>(W, ldw, l, cand, ncand, Wc);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_map_pivots(const int* Jc, const int* cand, const int* kout, int k, int* J,
                              cudaStream_t st) {
  map_pivots_kernel<<<1, 64, 0, st>>>(Jc, cand, kout, k, J);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fixed_solve(const double* W, int64_t ldw, int l, int n, const int* J,
                               const int* kout, int k, double* fq, double* P, cudaStream_t st) {
  if (l > FQ_ROWS || k > FQ_ROWS || k < 1 || n < 1) return cudaErrorInvalidValue;
  double* V = fq;
  double* tau = V + (size_t)k * l;
  double* R = tau + k;
  fixed_qr_kernel<<<1, FQ_ROWS, 0, st>>>(W, ldw, l, J, kout, k, V, tau, R);
  const size_t sm = sizeof(double) * ((size_t)k * l + k + (size_t)k * k);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fixed_apply_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  fixed_apply_kernel<<<(n + 127) / 128, 128, sm, st>>>(W, ldw, l, n, V, tau, R, J, kout, k, P);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace idsk
