// Deterministic k-step column-pivoted QR of the coarse matrix A_c (m_c x n),
// the core of the sub-sampled ID (Algorithm 5 steps 3-7, transposed).
//
// A_c is tall (e.g. 73,728 x 1000), so the QR is LEFT-looking: the
// reflectors are kept as V (m_c x s) and the trailing matrix is never formed.
// With F = A^T V T accumulated one column per step (the compact form used by
// blocked pivoted QR),
//   A^(s)          = A - V_s F_s^T                      (after s reflectors)
//   pivot column   u = A(:, p) - V_s F(p, :)^T          (rows >= s)
//   F(:, s)        = tau_s (A^T v_s - F_s (V_s^T v_s))  (one pass over A_c)
//   R(s, j)        = A(s, j) - V(s, 0:s+1) F(j, 0:s+1)^T
//   nu_j^2        -= R(s, j)^2                          (norm downdate)
// A downdated norm that lost more than 20 bits to cancellation is recomputed
// from its definition ||A^(s+1)(s+1:, j)||^2.  The pivot rule is the largest
// residual norm, ties to the lowest index; pivoting stops below the rank
// tolerance.  Reductions run in a fixed order.
//
// Precision: FP64 throughout, except the one O(m_c n) product per step,
// A_c^T v_s.  For FP32 data it runs on the FP32 units as exact FP32
// products of A_c with v_s split into an FP32 pair, summed as FP32 pairs
// (about 48 significant bits): FP64 arithmetic on this GPU is too slow for a
// pass over A_c at memory speed, while the FP32 units are not.  Each CTA owns
// whole columns, so no cross-CTA partial sums are needed.
#include <float.h>

#include <algorithm>

#include "idsk_internal.h"

namespace idsk {
namespace {

constexpr double kRecomputeFrac = 1.0 / (1 << 20);
// cint layout
constexpr int CI_P = 0, CI_STOP = 1, CI_NREC = 2, CI_KOUT = 3;
// cscal layout
constexpr int CS_ALPHA = 0, CS_SIGMA = 1, CS_BETA = 2, CS_TAU = 3, CS_DEN = 4, CS_TOL = 5;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// fixed-order block reduction (blockDim multiple of 32, <= 1024)
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < nw; ++w) s += sh[w];
    sh[32] = s;
  }
  __syncthreads();
  return sh[32];
}

template <typename T>
__global__ void init_norms_kernel(const T* __restrict__ Ac, int64_t mc, int n,
                                  double* __restrict__ nu2, double* __restrict__ nu20,
                                  int* __restrict__ colpos) {
  __shared__ double sh[33];
  const int j = blockIdx.x;
  double ss = 0.0;
  for (int64_t i = threadIdx.x; i < mc; i += blockDim.x) {
    const double x = (double)Ac[i + (int64_t)j * mc];
    ss += x * x;
  }
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) {
    nu2[j] = ss;
    nu20[j] = ss;
    colpos[j] = -1;
  }
}

__global__ void init_tol_kernel(const double* __restrict__ nu20, int n, double tol_factor,
                                double* __restrict__ cscal, int* __restrict__ cint) {
  __shared__ double sh[33];
  double ss = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) ss += nu20[j];
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) {
    cscal[CS_TOL] = tol_factor * DBL_EPSILON * sqrt(ss);
    cint[CI_P] = -1;
    cint[CI_STOP] = 0;
    cint[CI_NREC] = 0;
    cint[CI_KOUT] = 0;
  }
}

__global__ void __launch_bounds__(1024) pick_kernel(const double* __restrict__ nu2, int n, int s,
                                                    int* __restrict__ colpos,
                                                    int* __restrict__ Jc,
                                                    const double* __restrict__ cscal,
                                                    int* __restrict__ cint) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  if (cint[CI_STOP]) return;
  double v = -1.0;
  int idx = 0x7fffffff;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    if (colpos[j] >= 0) continue;
    const double nu = sqrt(fmax(nu2[j], 0.0));
    if (nu > v) {   // j increases within a thread: strict > keeps the lowest index
      v = nu;
      idx = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    bv[warp] = v;
    bi[warp] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = bv[0];
    int p = bi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      if (bv[w] > b || (bv[w] == b && bi[w] < p)) {
        b = bv[w];
        p = bi[w];
      }
    }
    cint[CI_NREC] = 0;
    if (!(b > cscal[CS_TOL])) {
      cint[CI_STOP] = 1;
      cint[CI_KOUT] = s;
    } else {
      cint[CI_P] = p;
      Jc[s] = p;
      colpos[p] = s;
    }
  }
}

// u = A(:, p) - V_s F(p, 0:s)^T on rows >= s -> V(:, s); partial sums of u_i^2, i > s
template <typename T>
__global__ void pivcol_kernel(const T* __restrict__ Ac, int64_t mc, int s,
                              double* __restrict__ V, const double* __restrict__ F, int64_t ldf,
                              double* __restrict__ upart, int rows_per_block,
                              const int* __restrict__ cint) {
  __shared__ double fp[kLMax];
  __shared__ double sh[33];
  if (cint[CI_STOP]) return;
  const int p = cint[CI_P];
  for (int t = threadIdx.x; t < s; t += blockDim.x) fp[t] = F[(int64_t)t * ldf + p];
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = (mc < r0 + rows_per_block) ? mc : r0 + rows_per_block;
  double ss = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double u = 0.0;
    if (i >= s) {
      u = (double)Ac[i + (int64_t)p * mc];
      for (int t = 0; t < s; ++t) u -= V[(int64_t)t * mc + i] * fp[t];
      if (i > s) ss += u * u;
    }
    V[(int64_t)s * mc + i] = u;
  }
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) upart[blockIdx.x] = ss;
}

__global__ void house_kernel(int s, int nblk, double* __restrict__ V, int64_t mc,
                             const double* __restrict__ upart, double* __restrict__ Rc, int n,
                             double* __restrict__ cscal, const int* __restrict__ cint) {
  if (cint[CI_STOP]) return;
  double part = 0.0;   // fixed order: lane-strided partial sums, then shuffles
  for (int b = threadIdx.x; b < nblk; b += 32) part += upart[b];
  const double sigma = warp_sum(part);
  if (threadIdx.x != 0) return;
  const int p = cint[CI_P];
  const double alpha = V[(int64_t)s * mc + s];
  double beta = alpha, tau = 0.0, den = 0.0;
  if (sigma != 0.0) {
    const double nrm = sqrt(alpha * alpha + sigma);
    beta = alpha >= 0.0 ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    den = alpha - beta;
  }
  cscal[CS_ALPHA] = alpha;
  cscal[CS_SIGMA] = sigma;
  cscal[CS_BETA] = beta;
  cscal[CS_TAU] = tau;
  cscal[CS_DEN] = den;
  V[(int64_t)s * mc + s] = 1.0;
  Rc[(int64_t)s * n + p] = beta;
}

// v_s = u / (alpha - beta) on rows > s (written back into V), v_s[s] = 1, and
// its FP32 pair (hi, lo) for the double-float GEMV below.
__global__ void scale_kernel(int64_t mc, int s, double* __restrict__ V, float* __restrict__ vh,
                             float* __restrict__ vl, const double* __restrict__ cscal,
                             const int* __restrict__ cint) {
  if (cint[CI_STOP]) return;
  const double den = cscal[CS_DEN];
  const double sigma = cscal[CS_SIGMA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mc;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i == s) {
      v = 1.0;
    } else if (i > s) {
      v = sigma != 0.0 ? V[(int64_t)s * mc + i] / den : 0.0;
      V[(int64_t)s * mc + i] = v;
    }
    const float hi = (float)v;
    vh[i] = hi;
    vl[i] = (float)(v - (double)hi);
  }
}

// a * (bh + bl) added to the FP32 pair (hi, lo): exact product error by FMA,
// TwoSum for the running sum, small terms gathered in lo (about 48 bits).
__device__ __forceinline__ void df_acc(float& hi, float& lo, float a, float bh, float bl) {
  const float p = a * bh;
  const float pe = fmaf(a, bh, -p);
  const float q = fmaf(a, bl, pe);
  const float t = hi + p;
  const float bp = t - hi;
  const float err = (hi - (t - bp)) + (p - bp);
  hi = t;
  lo += err + q;
}

// Partial g_j = A(rows, j)^T v_s for groups of 8 columns and one of RS row
// ranges per CTA (partials gpart[rs][j], summed in a fixed order by
// finalize), and partial h_t = V(rows, t)^T v_s for t < s in the CTAs after
// the column groups.  FP32 data: FP32 products summed as FP32 pairs; FP64
// data and the h terms: FP64.  The row loop is unrolled by 4 so that 32
// loads are in flight per thread.
constexpr int GCOLS = 8;
constexpr int RS = 8;
template <typename T>
__global__ void __launch_bounds__(256) gemv_cols_kernel(
    const T* __restrict__ Ac, int64_t mc, int n, int s, const double* __restrict__ V,
    const float* __restrict__ vh, const float* __restrict__ vl, int ngroups,
    double* __restrict__ gpart, double* __restrict__ hpart, const int* __restrict__ cint) {
  __shared__ double sh[GCOLS][8];
  if (cint[CI_STOP]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t span = mc - s;
  const int64_t chunk = (span + RS - 1) / RS;
  if ((int)blockIdx.x >= ngroups * RS) {   // partial h_t
    const int b = blockIdx.x - ngroups * RS;
    const int t = b / RS, rs = b - t * RS;
    const int64_t i0 = s + rs * chunk, i1 = min(mc, i0 + chunk);
    double acc = 0.0;
    const double* col = V + (int64_t)t * mc;
    for (int64_t i = i0 + tid; i < i1; i += 256) acc += col[i] * ((double)vh[i] + (double)vl[i]);
    acc = warp_sum(acc);
    if (lane == 0) sh[0][warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double r = 0.0;
      for (int w = 0; w < 8; ++w) r += sh[0][w];
      hpart[rs * kLMax + t] = r;
    }
    return;
  }
  const int grp = blockIdx.x / RS, rs = blockIdx.x - grp * RS;
  const int64_t i0 = s + rs * chunk, i1 = min(mc, i0 + chunk);
  const int j0 = grp * GCOLS;
  const T* cols[GCOLS];
#pragma unroll
  for (int q = 0; q < GCOLS; ++q) cols[q] = Ac + (int64_t)min(j0 + q, n - 1) * mc;
  double r[GCOLS];
  if (sizeof(T) == 4) {
    float hi[GCOLS], lo[GCOLS];
#pragma unroll
    for (int q = 0; q < GCOLS; ++q) hi[q] = lo[q] = 0.f;
    int64_t i = i0 + tid;
    for (; i + 3 * 256 < i1; i += 4 * 256) {
      float a[4][GCOLS], bh[4], bl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        bh[u] = vh[i + u * 256];
        bl[u] = vl[i + u * 256];
#pragma unroll
        for (int q = 0; q < GCOLS; ++q) a[u][q] = (float)cols[q][i + u * 256];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < GCOLS; ++q) df_acc(hi[q], lo[q], a[u][q], bh[u], bl[u]);
    }
    for (; i < i1; i += 256) {
      const float bh = vh[i], bl = vl[i];
#pragma unroll
      for (int q = 0; q < GCOLS; ++q) df_acc(hi[q], lo[q], (float)cols[q][i], bh, bl);
    }
#pragma unroll
    for (int q = 0; q < GCOLS; ++q) r[q] = (double)hi[q] + (double)lo[q];
  } else {
#pragma unroll
    for (int q = 0; q < GCOLS; ++q) r[q] = 0.0;
    for (int64_t i = i0 + tid; i < i1; i += 256) {
      const double b = (double)vh[i] + (double)vl[i];
#pragma unroll
      for (int q = 0; q < GCOLS; ++q) r[q] += (double)cols[q][i] * b;
    }
  }
#pragma unroll
  for (int q = 0; q < GCOLS; ++q) {
    const double v = warp_sum(r[q]);
    if (lane == 0) sh[q][warp] = v;
  }
  __syncthreads();
  if (tid < GCOLS && j0 + tid < n) {
    double acc = 0.0;
    for (int w = 0; w < 8; ++w) acc += sh[tid][w];
    gpart[(int64_t)rs * n + j0 + tid] = acc;
  }
}

template <typename T>
__global__ void finalize_kernel(const T* __restrict__ Ac, int64_t mc, int n, int s,
                                const double* __restrict__ V, double* __restrict__ F, int64_t ldf,
                                const double* __restrict__ gpart, const double* __restrict__ hpart,
                                const int* __restrict__ colpos, double* __restrict__ Rc,
                                double* __restrict__ nu2, const double* __restrict__ nu20,
                                int* __restrict__ rlist, const double* __restrict__ cscal,
                                int* __restrict__ cint) {
  __shared__ double h[kLMax];
  __shared__ double vrow[kLMax + 1];
  if (cint[CI_STOP]) return;
  for (int t = threadIdx.x; t < s; t += blockDim.x) {
    double acc = 0.0;
    for (int rs = 0; rs < RS; ++rs) acc += hpart[rs * kLMax + t];
    h[t] = acc;
  }
  for (int t = threadIdx.x; t <= s; t += blockDim.x) vrow[t] = V[(int64_t)t * mc + s];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int cp = colpos[j];
  if (cp >= 0) {
    if (cp < s) Rc[(int64_t)s * n + j] = 0.0;   // R(s, p) itself was set with beta
    return;
  }
  const double tau = cscal[CS_TAU];
  double fh = 0.0;
  for (int t = 0; t < s; ++t) fh += F[(int64_t)t * ldf + j] * h[t];
  double gj = 0.0;
  for (int rs = 0; rs < RS; ++rs) gj += gpart[(int64_t)rs * n + j];
  const double fjs = tau * (gj - fh);
  F[(int64_t)s * ldf + j] = fjs;
  double r = (double)Ac[s + (int64_t)j * mc];
  for (int t = 0; t < s; ++t) r -= vrow[t] * F[(int64_t)t * ldf + j];
  r -= vrow[s] * fjs;
  Rc[(int64_t)s * n + j] = r;
  const double nn = nu2[j] - r * r;
  nu2[j] = nn;
  if (nn <= kRecomputeFrac * nu20[j]) {
    const int slot = atomicAdd(&cint[CI_NREC], 1);
    rlist[slot] = j;
  }
}

// nu_j^2 = ||A^(s+1)(s+1:, j)||^2 from the definition, for the flagged columns
template <typename T>
__global__ void recompute_kernel(const T* __restrict__ Ac, int64_t mc, int s,
                                 const double* __restrict__ V, const double* __restrict__ F,
                                 int64_t ldf, const int* __restrict__ rlist,
                                 double* __restrict__ nu2, double* __restrict__ nu20,
                                 const int* __restrict__ cint) {
  __shared__ double fj[kLMax + 1];
  __shared__ double sh[33];
  if (cint[CI_STOP]) return;
  const int nrec = cint[CI_NREC];
  for (int idx = blockIdx.x; idx < nrec; idx += gridDim.x) {
    const int j = rlist[idx];
    __syncthreads();
    for (int t = threadIdx.x; t <= s; t += blockDim.x) fj[t] = F[(int64_t)t * ldf + j];
    __syncthreads();
    double ss = 0.0;
    for (int64_t i = s + 1 + threadIdx.x; i < mc; i += blockDim.x) {
      double a = (double)Ac[i + (int64_t)j * mc];
      for (int t = 0; t <= s; ++t) a -= V[(int64_t)t * mc + i] * fj[t];
      ss += a * a;
    }
    ss = block_sum(ss, sh);
    if (threadIdx.x == 0) {
      nu2[j] = ss;
      nu20[j] = ss;
    }
  }
}

__global__ void coarse_done_kernel(int kmax, int k, int* __restrict__ Jc, int* __restrict__ cint) {
  if (threadIdx.x == 0 && !cint[CI_STOP]) cint[CI_KOUT] = kmax;
  __syncthreads();
  for (int q = cint[CI_KOUT] + threadIdx.x; q < k; q += blockDim.x) Jc[q] = -1;
}

template <typename T>
cudaError_t run(id_sketch* h, int64_t n64, cudaStream_t st) {
  const T* Ac = reinterpret_cast<const T*>(h->d_Ac);
  const int64_t mc = h->mc;
  const int n = (int)n64;
  const int k = h->k;
  const int kmax = (int)std::min<int64_t>(k, std::min<int64_t>(mc, n64));
  const int64_t ldf = h->n_max;
  const int ngroups = (n + GCOLS - 1) / GCOLS;
  int rpb = (int)((mc + 2 * h->nsm - 1) / (2 * h->nsm));
  rpb = std::max(32, ((rpb + 31) / 32) * 32);
  rpb = std::min(rpb, 4096);
  const int nblk = (int)((mc + rpb - 1) / rpb);
  if (nblk > h->coarse_blocks) return cudaErrorInvalidValue;

  init_norms_kernel<T><<<n, 256, 0, st>>>(Ac, mc, n, h->d_nu2, h->d_nu20, h->d_colposc);
  init_tol_kernel<<<1, 1024, 0, st>>>(h->d_nu20, n, ID_RANK_TOL_FACTOR, h->d_cscal, h->d_cint);
  count_launches(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int s = 0; s < kmax; ++s) {
    pick_kernel<<<1, 1024, 0, st>>>(h->d_nu2, n, s, h->d_colposc, h->d_Jc, h->d_cscal, h->d_cint);
    pivcol_kernel<T><<<nblk, 256, 0, st>>>(Ac, mc, s, h->d_V, h->d_F, ldf, h->d_upart, rpb,
                                           h->d_cint);
    house_kernel<<<1, 32, 0, st>>>(s, nblk, h->d_V, mc, h->d_upart, h->d_Rc, n, h->d_cscal,
                                   h->d_cint);
    scale_kernel<<<2 * h->nsm, 256, 0, st>>>(mc, s, h->d_V, h->d_vh, h->d_vl, h->d_cscal,
                                             h->d_cint);
    gemv_cols_kernel<T><<<(ngroups + s) * RS, 256, 0, st>>>(Ac, mc, n, s, h->d_V, h->d_vh,
                                                            h->d_vl, ngroups, h->d_gvec,
                                                            h->d_hvec, h->d_cint);
    finalize_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(
        Ac, mc, n, s, h->d_V, h->d_F, ldf, h->d_gvec, h->d_hvec, h->d_colposc, h->d_Rc,
        h->d_nu2, h->d_nu20, h->d_rlist, h->d_cscal, h->d_cint);
    recompute_kernel<T><<<64, 256, 0, st>>>(Ac, mc, s, h->d_V, h->d_F, ldf, h->d_rlist, h->d_nu2,
                                            h->d_nu20, h->d_cint);
    count_launches(7);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  coarse_done_kernel<<<1, 256, 0, st>>>(kmax, k, h->d_Jc, h->d_cint);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_solve_p(h->d_Rc, h->d_Jc, h->d_colposc, h->d_cint + CI_KOUT, k, n, h->d_Pc, st);
}

}  // namespace

cudaError_t launch_coarse_cpqr(id_sketch* h, int64_t n, cudaStream_t st) {
  if (h->cfg.dtype == ID_F64) return run<double>(h, n, st);
  return run<float>(h, n, st);
}

int coarse_blocks_needed(int64_t mc, int nsm) {
  int rpb = (int)((mc + 2 * nsm - 1) / (2 * nsm));
  rpb = std::max(32, ((rpb + 31) / 32) * 32);
  rpb = std::min(rpb, 4096);
  return (int)((mc + rpb - 1) / rpb);
}

}  // namespace idsk
