// Deterministic k-step column-pivoted QR of the coarse matrix A_c (m_c x n),
// the core of the sub-sampled ID (Algorithm 5 steps 3-7, transposed).
//
// A_c is tall (e.g. 73,728 x 1000), so the QR is LEFT-looking: the
// reflectors are kept as V (m_c x s) and the trailing matrix is never formed.
// With F = A^T V T accumulated one column per step (the compact form used by
// blocked pivoted QR), step s with pivot column p computes
//   u              = A(:, p) - V_s F(p, :)^T          (rows >= s)
//   v_s            = u / (u_s - beta) below row s, v_s[s] = 1
//   F(:, s)        = tau_s (A^T v_s - F_s (V_s^T v_s))
//   R(s, j)        = A(s, j) - V(s, 0:s+1) F(j, 0:s+1)^T
//   nu_j^2        -= R(s, j)^2                        (norm downdate)
// A downdated norm that lost more than 20 bits to cancellation is recomputed
// from its definition ||A^(s+1)(s+1:, j)||^2.  The pivot rule is the largest
// residual norm, ties to the lowest index; pivoting stops below the rank
// tolerance.
//
// Pass structure (four launches per step).  A^T v_s = A(s, :)^T +
// (A^T u below row s) / (u_s - beta), so the one O(m_c n) product per step
// needs u only, not the Householder scalars:
//   step_kernel        every CTA finds the step's pivot from the norms, forms
//                      u for its rows and the partials of V^T u and ||u||^2;
//                      the last CTA to finish sums them into the scalars;
//   stream_gemv_kernel A_c^T u (or gemv_kernel when A_c cannot be streamed);
//   finalize_kernel    sums the A_c^T u partials per column, updates F, R and
//                      the norms, flags norms that lost too many bits;
//   recompute_kernel   recomputes the flagged norms (usually none).
// Every sum runs in a fixed order (CTA-ordered partials), so results do not
// depend on scheduling.
//
// Precision: the O(m_c n) product A_c^T u and the O(m_c s) work of each
// step (u, V_s^T u, ||u||^2, the reflectors V themselves) run on the FP32
// units in FP32-pair arithmetic (value = hi + lo, exact products by FMA,
// TwoSum accumulation: about 48 significant bits); the Householder scalars,
// F, R and the norms are FP64.  FP64 arithmetic on this GPU (1.25 TFLOP/s)
// is too slow for these passes at memory speed, its FP32 units are not.
#include <float.h>
#include <stdlib.h>

#include <algorithm>

#include "df.cuh"
#include "idsk_internal.h"
#include "tc_common.cuh"

namespace idsk {
namespace {

constexpr double kRecomputeFrac = 1.0 / (1 << 20);
// cint layout
constexpr int CI_P = 0, CI_STOP = 1, CI_NREC = 2, CI_KOUT = 3, CI_CNT_STEP = 4;
// cscal layout
constexpr int CS_ALPHA = 0, CS_SIGMA = 1, CS_BETA = 2, CS_TAU = 3, CS_DEN = 4, CS_TOL = 5;

constexpr int ST_THREADS = 256;            // step_kernel block = rows per sub-chunk
constexpr int HP = kLMax + 1;              // per-CTA partials: V^T u (kLMax), ||u||^2

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

// Pivot of step s over the columns not pivoted at steps 0..s-1: largest
// residual norm (compared as squared norms, which orders the same way), ties
// to the lowest index.  A non-negative double orders like its IEEE bit pattern
// read as an unsigned integer, so the comparisons run on the integer units
// (negative downdated values count as zero).  Whole block; every block of a
// grid may run it on the same norms and gets the same pivot (-1: stop below
// the rank tolerance); the writer block records it.
__device__ __forceinline__ unsigned long long norm_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? 0ull : b;
}

__device__ int pick_pivot(const double* __restrict__ nu2, int n, int s, int* __restrict__ colpos,
                          int* __restrict__ Jc, const double* __restrict__ cscal,
                          int* __restrict__ cint, bool writer) {
  __shared__ unsigned long long bv[32];
  __shared__ int bi[32];
  __shared__ int chosen;
  unsigned long long v = 0ull;
  int idx = 0x7fffffff;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int cp = colpos[j];
    if (cp >= 0 && cp < s) continue;   // pivoted at an earlier step
    const unsigned long long key = norm_key(nu2[j]);
    if (idx == 0x7fffffff || key > v) {   // j increases within a thread: strict >
      v = key;
      idx = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (oi != 0x7fffffff && (idx == 0x7fffffff || ov > v || (ov == v && oi < idx))) {
      v = ov;
      idx = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    bv[warp] = v;
    bi[warp] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = bv[0];
    int p = bi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      if (bi[w] != 0x7fffffff && (p == 0x7fffffff || bv[w] > b || (bv[w] == b && bi[w] < p))) {
        b = bv[w];
        p = bi[w];
      }
    }
    const double tol = cscal[CS_TOL];
    const bool stop = p == 0x7fffffff || !(b > norm_key(tol * tol));
    chosen = stop ? -1 : p;
    if (writer) {
      if (stop) {
        cint[CI_STOP] = 1;
        cint[CI_KOUT] = s;
      } else {
        cint[CI_P] = p;
        Jc[s] = p;
        colpos[p] = s;
      }
    }
  }
  __syncthreads();
  return chosen;
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

// Rank tolerance and counters.
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
    cint[CI_CNT_STEP] = 0;

  }
}

// True in every thread of the one CTA that finished last (release/acquire
// through a device-scope counter, which that CTA resets for the next launch).
__device__ bool last_cta(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
    if (last) *counter = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Step s over the CTA's row range [r0, r1) of A_c:
//   * scales column s-1 of V into v_{s-1} (its scalars are final now),
//   * u = A(:, p) - V_s F(p, :)^T on rows >= s, stored as column s of V and,
//     below row s, as an FP32 pair (uh, ul) for gemv_kernel (zero elsewhere),
//   * partials of V_s^T u and ||u||^2 over rows > s.
// The last CTA sums the partials (fixed CTA order) and forms the Householder
// scalars alpha = u_s, beta, tau, den = alpha - beta and h = V_s^T v_s.
template <typename T>
__global__ void __launch_bounds__(ST_THREADS) step_kernel(
    const T* __restrict__ Ac, int64_t mc, int n, int s, int64_t rpc,
    float2* __restrict__ V, const double* __restrict__ F, int64_t ldf,
    float* __restrict__ uh, float* __restrict__ ul, double* __restrict__ hpart,
    double* __restrict__ hvec, double* __restrict__ Rc, double* __restrict__ cscal,
    const double* __restrict__ nu2, int* __restrict__ colpos, int* __restrict__ Jc,
    int* __restrict__ cint) {
  __shared__ float2 fp[kLMax];
  __shared__ float2 ud[ST_THREADS];
  if (cint[CI_STOP]) return;
  // pivot of this step, found by every CTA from the final norms of step s-1
  const int p = pick_pivot(nu2, n, s, colpos, Jc, cscal, cint, blockIdx.x == 0);
  if (p < 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (blockIdx.x == 0 && tid == 0) cint[CI_NREC] = 0;   // appended to by this step's finalize
  for (int t = tid; t < s; t += ST_THREADS) fp[t] = df_of(F[(int64_t)t * ldf + p]);
  const double psig = s > 0 ? cscal[CS_SIGMA] : 0.0;
  const float2 prcp = df_of((s > 0 && psig != 0.0) ? 1.0 / cscal[CS_DEN] : 0.0);   // v = u / den
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = (mc < r0 + rpc) ? mc : r0 + rpc;
  float2 sig = make_float2(0.f, 0.f);
  float2 hacc[kLMax / 8];
#pragma unroll
  for (int q = 0; q < kLMax / 8; ++q) hacc[q] = make_float2(0.f, 0.f);
  for (int64_t c0 = r0; c0 < r1; c0 += ST_THREADS) {
    const int nrow = (int)((r1 - c0) < ST_THREADS ? (r1 - c0) : ST_THREADS);
    const int64_t i = c0 + tid;
    float2 uu = make_float2(0.f, 0.f);
    if (tid < nrow) {
      if (s > 0) {   // v_{s-1}: zero above row s-1, one at it, u / den below
        float2* vp = V + (int64_t)(s - 1) * mc + i;
        if (i == s - 1)
          *vp = make_float2(1.f, 0.f);
        else if (i > s - 1)
          *vp = df_mul(*vp, prcp);
      }
      float2 u = make_float2(0.f, 0.f);
      if (i >= s) {
        u = df_of((double)Ac[i + (int64_t)p * mc]);
        for (int t0 = 0; t0 < s; t0 += 16) {   // 16 loads of V in flight, then the sums
          float2 vv[16];
#pragma unroll
          for (int q = 0; q < 16; ++q)
            vv[q] = t0 + q < s ? V[(int64_t)(t0 + q) * mc + i] : make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            if (t0 + q < s) {
              const float2 pr = df_mul(vv[q], fp[t0 + q]);
              df_add(u.x, u.y, -pr.x, -pr.y);
            }
          }
        }
        u = df_norm(u.x, u.y);
      }
      V[(int64_t)s * mc + i] = u;
      if (i > s) uu = u;
      uh[i] = uu.x;
      ul[i] = uu.y;
    }
    ud[tid] = uu;
    const float2 u2 = df_mul(uu, uu);
    df_add(sig.x, sig.y, u2.x, u2.y);
    __syncthreads();
    // V_s^T u: warp w takes t = w + 8q, each lane keeps partials over its rows.
    // The loads of four quantities x 4 rows per lane are in flight together;
    // every partial still adds its rows in the same order.
#pragma unroll
    for (int qg = 0; qg < kLMax / 8; qg += 4) {
      if (warp + 8 * qg >= s) continue;
      for (int k0 = 0; k0 < nrow; k0 += 128) {
        float2 vv[4][4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const int t = warp + 8 * (qg + qq);
          const float2* vc = V + (int64_t)t * mc + c0;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = k0 + 32 * e + lane;
            vv[qq][e] = (t < s && k < nrow) ? vc[k] : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const int q = qg + qq;
          if (warp + 8 * q < s) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int k = k0 + 32 * e + lane;
              if (k < nrow) {
                const float2 pr = df_mul(vv[qq][e], ud[k]);
                df_add(hacc[q].x, hacc[q].y, pr.x, pr.y);
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  // warp sums of the pair partials (fixed shuffle tree)
#pragma unroll
  for (int q = 0; q < kLMax / 8; ++q) {
    if (warp + 8 * q < s) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hacc[q].x, o);
        const float ol = __shfl_xor_sync(0xffffffffu, hacc[q].y, o);
        df_add(hacc[q].x, hacc[q].y, oh, ol);
      }
      hacc[q] = df_norm(hacc[q].x, hacc[q].y);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, sig.x, o);
    const float ol = __shfl_xor_sync(0xffffffffu, sig.y, o);
    df_add(sig.x, sig.y, oh, ol);
  }
  __shared__ float2 sig_w[ST_THREADS / 32];
  if (lane == 0) sig_w[warp] = sig;
  __syncthreads();
  // partials stored as FP32 pairs, summed by the last CTA on the FP32 units
  float2* hp = reinterpret_cast<float2*>(hpart) + (int64_t)blockIdx.x * HP;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < kLMax / 8; ++q)
      if (warp + 8 * q < s) hp[warp + 8 * q] = hacc[q];
  }
  if (tid == 0) {
    float2 a = sig_w[0];
    for (int w = 1; w < ST_THREADS / 32; ++w) df_add(a.x, a.y, sig_w[w].x, sig_w[w].y);
    hp[kLMax] = df_norm(a.x, a.y);
  }
  if (!last_cta(reinterpret_cast<unsigned*>(cint + CI_CNT_STEP))) return;

  // ---- last CTA: Householder scalars and h = V_s^T v_s.  Warp w sums the
  // CTA partials of quantities w, w + 8, ... (t < s, and ||u||^2 as quantity
  // kLMax), lane-strided over the CTAs and then by a fixed shuffle tree.
  const int G = gridDim.x;
  __shared__ double hs[kLMax + 1];
  // The partials are summed as FP32 pairs (TwoSum accumulation, about 48
  // bits): FP64 adds on this GPU are too slow for a G x (s + 1) reduction on
  // one SM.
  constexpr int NQ = kLMax / 8 + 1;   // quantities warp + 8q, q < NQ
  float ah[NQ], al[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) ah[q] = al[q] = 0.f;
  for (int b = lane; b < G; b += 64) {   // two CTA strides of loads in flight
    float2 x0[NQ], x1[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int qn = warp + 8 * q;
      const bool use = qn < s || qn == kLMax;
      const float2* hp2 = reinterpret_cast<const float2*>(hpart);
      x0[q] = use ? hp2[(int64_t)b * HP + qn] : make_float2(0.f, 0.f);
      x1[q] = (use && b + 32 < G) ? hp2[(int64_t)(b + 32) * HP + qn] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int qn = warp + 8 * q;
      if (qn < s || qn == kLMax) {
        df_add(ah[q], al[q], x0[q].x, x0[q].y);
        if (b + 32 < G) df_add(ah[q], al[q], x1[q].x, x1[q].y);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int qn = warp + 8 * q;
    if (qn < s || qn == kLMax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, ah[q], o);
        const float ol = __shfl_xor_sync(0xffffffffu, al[q], o);
        df_add(ah[q], al[q], oh, ol);
      }
      if (lane == 0) hs[qn] = (double)ah[q] + (double)al[q];
    }
  }
  __syncthreads();
  const double sigma = hs[kLMax];
  const double alpha = df_val(V[(int64_t)s * mc + s]);
  double beta = alpha, tau = 0.0, den = 0.0;
  if (sigma != 0.0) {
    const double nrm = sqrt(alpha * alpha + sigma);
    beta = alpha >= 0.0 ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    den = alpha - beta;
  }
  const double rden = sigma != 0.0 ? 1.0 / den : 0.0;
  for (int t = tid; t < s; t += ST_THREADS) {
    const double vst = df_val(V[(int64_t)t * mc + s]);   // v_t[s]
    hvec[t] = vst + hs[t] * rden;
  }
  if (tid == 0) {
    cscal[CS_ALPHA] = alpha;
    cscal[CS_SIGMA] = sigma;
    cscal[CS_BETA] = beta;
    cscal[CS_TAU] = tau;
    cscal[CS_DEN] = den;
    Rc[(int64_t)s * n + p] = beta;
  }
}

// Partial g_j = A(rows, j)^T u for a group of GCOLS columns and one of RS
// row ranges per CTA (gpart[rs][j], summed in a fixed order by
// finalize_kernel).  Lanes take consecutive row quads (128-bit loads, two row
// quads of every column in flight per thread); FP32 data: exact FP32
// products with u as an FP32 pair, summed as FP32 pairs; FP64 data: FP64.
constexpr int GCOLS = 8;
constexpr int GV_THREADS = 256;
template <typename T>
__global__ void __launch_bounds__(GV_THREADS) gemv_kernel(
    const T* __restrict__ Ac, int64_t mc, int n, int s, int64_t chunk, int vec,
    const float* __restrict__ uh, const float* __restrict__ ul,
    double* __restrict__ gpart, const int* __restrict__ cint) {
  __shared__ double sh[GCOLS][GV_THREADS / 32];
  if (cint[CI_STOP]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ngroups = (n + GCOLS - 1) / GCOLS;
  const int grp = blockIdx.x % ngroups, rs = blockIdx.x / ngroups;
  const int j0 = grp * GCOLS;
  // rows above s + 1 hold u = 0: start at the row quad holding s + 1
  int64_t i0 = rs * chunk, i1 = i0 + chunk < mc ? i0 + chunk : mc;
  const int64_t lo_row = (int64_t)(s + 1) & ~(int64_t)3;
  if (i0 < lo_row) i0 = lo_row < i1 ? lo_row : i1;
  const T* cols[GCOLS];
#pragma unroll
  for (int q = 0; q < GCOLS; ++q) cols[q] = Ac + (int64_t)(j0 + q < n ? j0 + q : n - 1) * mc;
  double r[GCOLS];
  if constexpr (sizeof(T) == 4) {
    float hi[GCOLS], lo[GCOLS];
#pragma unroll
    for (int q = 0; q < GCOLS; ++q) hi[q] = lo[q] = 0.f;
    if (vec) {   // mc, chunk multiples of 4
      int64_t i = i0 + 4 * tid;
      for (; i + 4 * GV_THREADS < i1; i += 8 * GV_THREADS) {
        float4 x0[GCOLS], x1[GCOLS];
#pragma unroll
        for (int q = 0; q < GCOLS; ++q) {
          x0[q] = __ldcs(reinterpret_cast<const float4*>(cols[q] + i));
          x1[q] = __ldcs(reinterpret_cast<const float4*>(cols[q] + i + 4 * GV_THREADS));
        }
        const float4 h0 = *reinterpret_cast<const float4*>(uh + i);
        const float4 l0 = *reinterpret_cast<const float4*>(ul + i);
        const float4 h1 = *reinterpret_cast<const float4*>(uh + i + 4 * GV_THREADS);
        const float4 l1 = *reinterpret_cast<const float4*>(ul + i + 4 * GV_THREADS);
#pragma unroll
        for (int q = 0; q < GCOLS; ++q) {
          df_acc(hi[q], lo[q], x0[q].x, h0.x, l0.x);
          df_acc(hi[q], lo[q], x0[q].y, h0.y, l0.y);
          df_acc(hi[q], lo[q], x0[q].z, h0.z, l0.z);
          df_acc(hi[q], lo[q], x0[q].w, h0.w, l0.w);
          df_acc(hi[q], lo[q], x1[q].x, h1.x, l1.x);
          df_acc(hi[q], lo[q], x1[q].y, h1.y, l1.y);
          df_acc(hi[q], lo[q], x1[q].z, h1.z, l1.z);
          df_acc(hi[q], lo[q], x1[q].w, h1.w, l1.w);
        }
      }
      for (; i < i1; i += 4 * GV_THREADS) {
        const float4 h0 = *reinterpret_cast<const float4*>(uh + i);
        const float4 l0 = *reinterpret_cast<const float4*>(ul + i);
#pragma unroll
        for (int q = 0; q < GCOLS; ++q) {
          const float4 x = __ldcs(reinterpret_cast<const float4*>(cols[q] + i));
          df_acc(hi[q], lo[q], x.x, h0.x, l0.x);
          df_acc(hi[q], lo[q], x.y, h0.y, l0.y);
          df_acc(hi[q], lo[q], x.z, h0.z, l0.z);
          df_acc(hi[q], lo[q], x.w, h0.w, l0.w);
        }
      }
    } else {
      for (int64_t i = i0 + tid; i < i1; i += GV_THREADS) {
        const float bh = uh[i], bl = ul[i];
#pragma unroll
        for (int q = 0; q < GCOLS; ++q) df_acc(hi[q], lo[q], cols[q][i], bh, bl);
      }
    }
#pragma unroll
    for (int q = 0; q < GCOLS; ++q) r[q] = (double)hi[q] + (double)lo[q];
  } else {
#pragma unroll
    for (int q = 0; q < GCOLS; ++q) r[q] = 0.0;
    for (int64_t i = i0 + tid; i < i1; i += GV_THREADS) {
      const double b = (double)uh[i] + (double)ul[i];   // zero at and above row s
#pragma unroll
      for (int q = 0; q < GCOLS; ++q) r[q] = fma((double)cols[q][i], b, r[q]);
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
    for (int w = 0; w < GV_THREADS / 32; ++w) acc += sh[tid][w];
    gpart[(int64_t)rs * n + j0 + tid] = acc;
  }
}

// Streamed pass over FP32 A_c (m_c a multiple of 4): A_c^T u below row s
// (mode 0, u as the FP32 pair uh + ul) or the column sums of squares (mode 1).
// Work items are (group of SG_COLS columns, chunk of SG_ROWS rows) in
// group-major order; CTA b takes the contiguous item range
// [T b / G, T (b + 1) / G).  One producer thread bulk-copies each item's
// column pieces (and u's pair) into an SG_ST-stage shared-memory ring; eight
// consumer warps (thread t: row quads t, t + 256, ...) accumulate FP32-pair
// sums over the chunks of a group and, when the group changes, write one
// partial per (CTA, column): part[b][j].  stream_cta_range() gives the CTAs
// that touched a column, whose partials are then summed in CTA order.
constexpr int SG_COLS = 4, SG_ROWS = 4096, SG_ST = 2, SG_CONS = 8;
constexpr uint32_t SG_COLB = SG_ROWS * 4;                  // 16 KB column piece
constexpr uint32_t SG_STAGE = (SG_COLS + 2) * SG_COLB;     // + uh, ul
constexpr int SG_THREADS = (SG_CONS + 1) * 32;

__device__ __forceinline__ void mbar_expect_tx_arrive(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// CTAs [*b0, *b1] whose item ranges hold the items of column group g.
__host__ __device__ inline void stream_cta_range(int64_t T, int G, int64_t nchunks, int g,
                                                 int* b0, int* b1) {
  auto cta_of = [&](int64_t item) {
    int64_t b = item * G / T;
    while (b + 1 < G && T * (b + 1) / G <= item) ++b;
    while (b > 0 && T * b / G > item) --b;
    return (int)b;
  };
  *b0 = cta_of((int64_t)g * nchunks);
  *b1 = cta_of((int64_t)(g + 1) * nchunks - 1);
}

__global__ void __launch_bounds__(SG_THREADS, 1) stream_gemv_kernel(
    const float* __restrict__ Ac, int64_t mc, int n, int mode, const float* __restrict__ uh,
    const float* __restrict__ ul, double* __restrict__ part, int* __restrict__ status,
    const int* __restrict__ cint, int64_t keep_rows) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * SG_ST];
  __shared__ int abort_flag;
  __shared__ double red[SG_CONS][SG_COLS];
  if (mode == 0 && cint[CI_STOP]) return;
  const uint32_t base = (tc::smem_u32(smem_raw) + 127u) & ~127u;
  const uint8_t* basep = smem_raw + (base - tc::smem_u32(smem_raw));
  const uint32_t full0 = tc::smem_u32(&bars[0]), empty0 = tc::smem_u32(&bars[SG_ST]);
  const uint32_t abort_a = tc::smem_u32(&abort_flag);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ngroups = (n + SG_COLS - 1) / SG_COLS;
  const int64_t nchunks = (mc + SG_ROWS - 1) / SG_ROWS;
  const int64_t T = (int64_t)ngroups * nchunks;
  const int64_t it0 = T * blockIdx.x / gridDim.x, it1 = T * (blockIdx.x + 1) / gridDim.x;
  if (tid == 0) {
    for (int q = 0; q < SG_ST; ++q) {
      tc::mbar_init(full0 + 8u * q, 1);
      tc::mbar_init(empty0 + 8u * q, SG_CONS);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == SG_CONS) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      // rows [0, keep_rows) of every column stay in L2 from one pass to the
      // next (evict_last); the rest streams through (evict_first)
      const uint64_t pol_keep = tc::policy_evict_last(), pol_stream = tc::policy_evict_first();
      int u = 0;
      for (int64_t it = it0; it < it1; ++it, ++u) {
        const int st = u % SG_ST;
        if (u >= SG_ST && !tc::mbar_wait_spin(empty0 + 8u * st, ((u / SG_ST) - 1) & 1, abort_a))
          break;
        const int g = (int)(it / nchunks);
        const int64_t r0 = (it - (int64_t)g * nchunks) * SG_ROWS;
        const uint32_t bytes = (uint32_t)((mc - r0 < SG_ROWS ? mc - r0 : SG_ROWS) * 4);
        const int ncols = n - g * SG_COLS < SG_COLS ? n - g * SG_COLS : SG_COLS;
        const uint32_t dst = base + (uint32_t)st * SG_STAGE;
        mbar_expect_tx_arrive(full0 + 8u * st, bytes * (ncols + (mode == 0 ? 2 : 0)));
        const uint64_t pol = r0 < keep_rows ? pol_keep : pol_stream;
        for (int q = 0; q < ncols; ++q)
          tc::bulk_g2s_hint(dst + q * SG_COLB, Ac + (int64_t)(g * SG_COLS + q) * mc + r0, bytes,
                            full0 + 8u * st, pol);
        if (mode == 0) {
          tc::bulk_g2s_hint(dst + SG_COLS * SG_COLB, uh + r0, bytes, full0 + 8u * st, pol_keep);
          tc::bulk_g2s_hint(dst + (SG_COLS + 1) * SG_COLB, ul + r0, bytes, full0 + 8u * st,
                            pol_keep);
        }
      }
    }
  } else {
    // ---------------------------------------------------------- consumers
    float hi[SG_COLS], lo[SG_COLS];
    int cur = -1;
    auto flush = [&](int g) {
#pragma unroll
      for (int q = 0; q < SG_COLS; ++q) {
        double v = (double)hi[q] + (double)lo[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(SG_CONS * 32) : "memory");
      if (tid < SG_COLS && g * SG_COLS + tid < n) {
        double a = 0.0;
        for (int w = 0; w < SG_CONS; ++w) a += red[w][tid];
        part[(int64_t)blockIdx.x * n + g * SG_COLS + tid] = a;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(SG_CONS * 32) : "memory");
    };
    // one row quad of the stage into the accumulators
    auto quad = [&](const uint8_t* stage, int ncols, int r4) {
      float4 bh = make_float4(0.f, 0.f, 0.f, 0.f), bl = bh;
      if (mode == 0) {
        bh = *reinterpret_cast<const float4*>(stage + SG_COLS * SG_COLB + 4 * r4);
        bl = *reinterpret_cast<const float4*>(stage + (SG_COLS + 1) * SG_COLB + 4 * r4);
      }
      float4 x[SG_COLS];
#pragma unroll
      for (int q = 0; q < SG_COLS; ++q)
        x[q] = q < ncols ? *reinterpret_cast<const float4*>(stage + q * SG_COLB + 4 * r4)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < SG_COLS; ++q) {
        if (mode == 0) {
          df_acc(hi[q], lo[q], x[q].x, bh.x, bl.x);
          df_acc(hi[q], lo[q], x[q].y, bh.y, bl.y);
          df_acc(hi[q], lo[q], x[q].z, bh.z, bl.z);
          df_acc(hi[q], lo[q], x[q].w, bh.w, bl.w);
        } else {
          df_acc(hi[q], lo[q], x[q].x, x[q].x, 0.f);
          df_acc(hi[q], lo[q], x[q].y, x[q].y, 0.f);
          df_acc(hi[q], lo[q], x[q].z, x[q].z, 0.f);
          df_acc(hi[q], lo[q], x[q].w, x[q].w, 0.f);
        }
      }
    };
    int u = 0;
    for (int64_t it = it0; it < it1; ++it, ++u) {
      const int st = u % SG_ST;
      const int g = (int)(it / nchunks);
      if (g != cur) {
        if (cur >= 0) flush(cur);
        cur = g;
#pragma unroll
        for (int q = 0; q < SG_COLS; ++q) hi[q] = lo[q] = 0.f;
      }
      // after a timeout every consumer keeps the same loop (and flushes) but
      // skips the data, so that the named barriers in flush() stay matched
      const bool ok = tc::mbar_wait_spin(full0 + 8u * st, (u / SG_ST) & 1, abort_a);
      const int64_t r0 = (it - (int64_t)g * nchunks) * SG_ROWS;
      const int rows = (int)(mc - r0 < SG_ROWS ? mc - r0 : SG_ROWS);
      const int ncols = n - g * SG_COLS < SG_COLS ? n - g * SG_COLS : SG_COLS;
      const uint8_t* stage = basep + (size_t)st * SG_STAGE;
      for (int r4 = 4 * tid; ok && r4 < rows; r4 += 4 * SG_CONS * 32) quad(stage, ncols, r4);
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(empty0 + 8u * st);
    }
    if (cur >= 0) flush(cur);
  }
  __syncthreads();
  if (tid == 0 && abort_flag) atomicOr(status, 1);
}

// Column norms from the streamed sums of squares: nu2 = nu20 = sum over the
// CTAs that touched the column, in CTA order.
__global__ void norms_from_parts_kernel(const double* __restrict__ part, int64_t mc, int n, int G,
                                        double* __restrict__ nu2, double* __restrict__ nu20,
                                        int* __restrict__ colpos) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int ngroups = (n + SG_COLS - 1) / SG_COLS;
  const int64_t nchunks = (mc + SG_ROWS - 1) / SG_ROWS;
  int b0, b1;
  stream_cta_range((int64_t)ngroups * nchunks, G, nchunks, j / SG_COLS, &b0, &b1);
  double a = 0.0;
  for (int b = b0; b <= b1; ++b) a += part[(int64_t)b * n + j];
  nu2[j] = a;
  nu20[j] = a;
  colpos[j] = -1;
}

// Per column j (lane of warp 0): g_j = A(:, j)^T v_s from the CTA-ordered
// partials (G > 0: G row-split partials summed by the 8 warps over contiguous
// ranges, then in warp order; G < 0: the streamed partials of the -G CTAs of
// stream_gemv_kernel that touched the column), F(j, s), R(s, j) and the norm
// downdate.
constexpr int FIN_COLS = 32;
template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(
    const T* __restrict__ Ac, int64_t mc, int n, int s, int G, const float2* __restrict__ V,
    double* __restrict__ F, int64_t ldf, const double* __restrict__ gpart,
    const double* __restrict__ hvec, const int* __restrict__ colpos, double* __restrict__ Rc,
    double* __restrict__ nu2, const double* __restrict__ nu20, int* __restrict__ rlist,
    const double* __restrict__ cscal, int* __restrict__ cint) {
  __shared__ double part[8][FIN_COLS];
  __shared__ double pfh[8][FIN_COLS];
  __shared__ double prr[8][FIN_COLS];
  __shared__ double h[kLMax];
  __shared__ double vrow[kLMax];
  if (cint[CI_STOP]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j = blockIdx.x * FIN_COLS + lane;
  if (G > 0) {   // RS row-split partials: warp w sums a contiguous range
    const int b0 = (int)((int64_t)G * warp / 8), b1 = (int)((int64_t)G * (warp + 1) / 8);
    double a = 0.0;
    if (j < n)
      for (int b = b0; b < b1; ++b) a += gpart[(int64_t)b * n + j];
    part[warp][lane] = a;
  } else {       // streamed partials of the CTAs that touched column j
    double a = 0.0;
    if (warp == 0 && j < n) {
      const int ngroups = (n + SG_COLS - 1) / SG_COLS;
      const int64_t nchunks = (mc + SG_ROWS - 1) / SG_ROWS;
      int b0, b1;
      stream_cta_range((int64_t)ngroups * nchunks, -G, nchunks, j / SG_COLS, &b0, &b1);
      for (int b = b0; b <= b1; ++b) a += gpart[(int64_t)b * n + j];
    }
    part[warp][lane] = a;
  }
  for (int t = tid; t < s; t += 256) {
    h[t] = hvec[t];
    vrow[t] = df_val(V[(int64_t)t * mc + s]);
  }
  __syncthreads();
  // F(j, 0:s) h and V(s, 0:s) F(j, 0:s)^T: warp w takes t = w, w + 8, ...
  {
    double fh = 0.0, rr = 0.0;
    if (j < n) {
      double fv[kLMax / 8];   // all loads of the thread in flight
#pragma unroll
      for (int q = 0; q < kLMax / 8; ++q) {
        const int t = warp + 8 * q;
        fv[q] = t < s ? F[(int64_t)t * ldf + j] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < kLMax / 8; ++q) {
        const int t = warp + 8 * q;
        if (t < s) {
          fh += fv[q] * h[t];
          rr += vrow[t] * fv[q];
        }
      }
    }
    pfh[warp][lane] = fh;
    prr[warp][lane] = rr;
  }
  __syncthreads();
  if (warp == 0 && j < n) {
    double gsum = 0.0, fh = 0.0, rr = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      gsum += part[w][lane];
      fh += pfh[w][lane];
      rr += prr[w][lane];
    }
    const int cp = colpos[j];
    if (cp >= 0) {
      if (cp < s) Rc[(int64_t)s * n + j] = 0.0;   // R(s, p) itself was set with beta
    } else {
      const double tau = cscal[CS_TAU], den = cscal[CS_DEN], sigma = cscal[CS_SIGMA];
      const double asj = (double)Ac[s + (int64_t)j * mc];
      const double gj = sigma != 0.0 ? asj + gsum / den : asj;
      const double fjs = tau * (gj - fh);
      F[(int64_t)s * ldf + j] = fjs;
      const double r = asj - rr - fjs;   // v_s[s] = 1
      Rc[(int64_t)s * n + j] = r;
      const double nn = nu2[j] - r * r;
      nu2[j] = nn;
      if (nn <= kRecomputeFrac * nu20[j]) {
        const int slot = atomicAdd(&cint[CI_NREC], 1);
        rlist[slot] = j;
      }
    }
  }
}

// nu_j^2 = ||A^(s+1)(s+1:, j)||^2 from the definition, for the columns that
// finalize_kernel flagged (column s of V still holds u: v_s = u / den below
// row s).  Usually there are none and every CTA returns at once.
template <typename T>
__global__ void recompute_kernel(const T* __restrict__ Ac, int64_t mc, int s,
                                 const float2* __restrict__ V, const double* __restrict__ F,
                                 int64_t ldf, const int* __restrict__ rlist,
                                 double* __restrict__ nu2, double* __restrict__ nu20,
                                 const double* __restrict__ cscal, const int* __restrict__ cint) {
  __shared__ double fj[kLMax + 1];
  __shared__ double sh[33];
  if (cint[CI_STOP]) return;
  const int nrec = cint[CI_NREC];
  if (nrec == 0) return;
  const double sigma = cscal[CS_SIGMA];
  const double rden = sigma != 0.0 ? 1.0 / cscal[CS_DEN] : 0.0;
  for (int idx = blockIdx.x; idx < nrec; idx += gridDim.x) {
    const int j = rlist[idx];
    __syncthreads();
    for (int t = threadIdx.x; t <= s; t += blockDim.x) fj[t] = F[(int64_t)t * ldf + j];
    __syncthreads();
    double ss = 0.0;
    for (int64_t i = s + 1 + threadIdx.x; i < mc; i += blockDim.x) {
      double a = (double)Ac[i + (int64_t)j * mc];
      for (int t = 0; t < s; ++t) a -= df_val(V[(int64_t)t * mc + i]) * fj[t];
      const double vs = df_val(V[(int64_t)s * mc + i]) * rden;
      a -= vs * fj[s];
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

// Row ranges of step_kernel: G CTAs of rpc rows (a multiple of 4).
void step_grid(int64_t mc, int nsm, int* G, int64_t* rpc) {
  int64_t g = (mc + 63) / 64;   // at least 64 rows per CTA, two CTAs per SM at most
  g = std::max<int64_t>(1, std::min<int64_t>(g, 2 * (int64_t)nsm));
  int64_t r = (mc + g - 1) / g;
  r = (r + 3) / 4 * 4;
  *rpc = r;
  *G = (int)((mc + r - 1) / r);
}

// Row splits of gemv_kernel: about seven waves of two CTAs per SM over the
// column groups, rows split in multiples of 4.
void gemv_grid(int64_t mc, int n, int nsm, int max_rs, int* RS, int64_t* chunk) {
  const int ngroups = (n + GCOLS - 1) / GCOLS;
  int rs = (14 * nsm + ngroups - 1) / ngroups;
  rs = std::max(1, std::min(rs, max_rs));
  int64_t c = (mc + rs - 1) / rs;
  c = std::max<int64_t>(4, (c + 3) / 4 * 4);
  *chunk = c;
  *RS = (int)((mc + c - 1) / c);
}

template <typename T>
cudaError_t run(id_sketch* h, int64_t n64, cudaStream_t st) {
  const T* Ac = reinterpret_cast<const T*>(h->d_Ac);
  const int64_t mc = h->mc;
  const int n = (int)n64;
  const int k = h->k;
  const int kmax = (int)std::min<int64_t>(k, std::min<int64_t>(mc, n64));
  const int64_t ldf = h->n_max;
  int G, RS;
  int64_t rpc, chunk;
  step_grid(mc, h->nsm, &G, &rpc);
  gemv_grid(mc, n, h->nsm, h->coarse_blocks, &RS, &chunk);
  if (G > h->coarse_blocks || RS > h->coarse_blocks || h->nsm > h->coarse_blocks)
    return cudaErrorInvalidValue;
  const int vec = (sizeof(T) == 4 && (mc & 3) == 0) ? 1 : 0;
  const int ngroups = (n + GCOLS - 1) / GCOLS;
  const int fin_blocks = (n + FIN_COLS - 1) / FIN_COLS;
  float2* V2 = reinterpret_cast<float2*>(h->d_V);   // reflectors as FP32 pairs

  // FP32 data with m_c a multiple of 4 streams A_c through bulk copies
  const bool streamed = vec && getenv("IDSKETCH_COARSE_STREAM") == nullptr;
  const int SG = h->nsm;
  const size_t sg_smem = 128 + (size_t)SG_ST * SG_STAGE;
  // the leading rows of A_c that stay in L2 between the k passes: about 3/8
  // of L2 (the rest holds V, u and the partials), whole 4096-row chunks
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->dev) != cudaSuccess) {
    cudaGetLastError();
    l2 = 0;
  }
  const double keep_target = 0.375 * (double)l2 / (4.0 * (double)n);
  const int64_t keep_rows =
      std::min<int64_t>(mc, (int64_t)(keep_target / SG_ROWS + 0.5) * SG_ROWS);
  if (streamed) {
    cudaError_t e0 = cudaFuncSetAttribute(stream_gemv_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sg_smem);
    if (e0 != cudaSuccess) return e0;
    stream_gemv_kernel<<<SG, SG_THREADS, sg_smem, st>>>(
        reinterpret_cast<const float*>(Ac), mc, n, 1, nullptr, nullptr, h->d_gvec, h->d_status,
        h->d_cint, keep_rows);
    norms_from_parts_kernel<<<(n + 255) / 256, 256, 0, st>>>(h->d_gvec, mc, n, SG, h->d_nu2,
                                                             h->d_nu20, h->d_colposc);
  } else {
    init_norms_kernel<T><<<n, 256, 0, st>>>(Ac, mc, n, h->d_nu2, h->d_nu20, h->d_colposc);
  }
  init_tol_kernel<<<1, 1024, 0, st>>>(h->d_nu20, n, ID_RANK_TOL_FACTOR, h->d_cscal, h->d_cint);
  count_launches(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int s = 0; s < kmax; ++s) {
    step_kernel<T><<<G, ST_THREADS, 0, st>>>(Ac, mc, n, s, rpc, V2, h->d_F, ldf, h->d_vh,
                                             h->d_vl, h->d_upart, h->d_hvec, h->d_Rc,
                                             h->d_cscal, h->d_nu2, h->d_colposc, h->d_Jc,
                                             h->d_cint);
    if (streamed)
      stream_gemv_kernel<<<SG, SG_THREADS, sg_smem, st>>>(
          reinterpret_cast<const float*>(Ac), mc, n, 0, h->d_vh, h->d_vl, h->d_gvec,
          h->d_status, h->d_cint, keep_rows);
    else
      gemv_kernel<T><<<ngroups * RS, GV_THREADS, 0, st>>>(Ac, mc, n, s, chunk, vec, h->d_vh,
                                                          h->d_vl, h->d_gvec, h->d_cint);
    finalize_kernel<T><<<fin_blocks, 256, 0, st>>>(
        Ac, mc, n, s, streamed ? -SG : RS, V2, h->d_F, ldf, h->d_gvec, h->d_hvec,
        h->d_colposc, h->d_Rc, h->d_nu2, h->d_nu20, h->d_rlist, h->d_cscal, h->d_cint);
    recompute_kernel<T><<<64, 256, 0, st>>>(Ac, mc, s, V2, h->d_F, ldf, h->d_rlist, h->d_nu2,
                                            h->d_nu20, h->d_cscal, h->d_cint);
    count_launches(4);
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
  if (coarse_coop_ok(h)) {
    const cudaError_t e = launch_coarse_coop(h, n, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (h->cfg.dtype == ID_F64) return run<double>(h, n, st);
  return run<float>(h, n, st);
}

// Rows of the per-CTA partial buffers: step_kernel's CTAs, and one per SM for
// stream_gemv_kernel.
int coarse_blocks_needed(int64_t mc, int nsm) {
  int G;
  int64_t rpc;
  step_grid(mc, nsm, &G, &rpc);
  return std::max(G, nsm);
}

}  // namespace idsk
