// The coarse-grid pivoted QR (Algorithm 5 steps 3-7, transposed) as one
// cooperative, persistent launch: all k steps of the left-looking Householder
// QR of A_c (m_c x n FP32) in a single kernel, with grid-wide barriers
// between the dependent phases of a step instead of four dependent launches.
//
// Work split.  CTA b owns a fixed range of A_c's rows (whole row quads,
// about m_c / #SMs rows, at most 512) for the passes over rows, and a fixed
// range of columns for the per-column updates.  Per step s, with pivot p:
//   A  pivot from the norms (every CTA, same data, same choice); scale
//      column s-1 of V into v_{s-1}; for the CTA's rows
//        u = A(:, p) - V_s F(p, :)^T     (rows >= s; kept as column s of V),
//      the CTA's partials of V_s^T u and ||u||^2 (rows > s), and its share
//      of A^T u: its rows of every column (warp w takes columns w, w + 16,
//      ...; 128-bit loads two columns ahead of the sums, so that the warps
//      stream A_c independently of one another), one partial per (CTA,
//      column);
//   -- grid barrier --
//   B  every CTA sums the partials (in CTA order) into the Householder
//      scalars alpha = u_s, beta, tau, den = alpha - beta and h = V_s^T v_s;
//   C  for the CTA's columns: g_j = A(s, j) + (A^T u)_j / den, F(j, s),
//      R(s, j) and the norm downdate (a norm that lost more than 20 bits is
//      recomputed from its definition, rows split over the CTAs);
//   -- grid barrier --
// A^T v_s = A(s, :)^T + (A^T u below row s) / (u_s - beta) lets the pass over
// A_c run before the scalars exist, so a step needs two grid barriers.
// Arithmetic: the passes over rows and the sums of their per-CTA partials in
// FP32 pairs (about 48 bits); scalars, F, R and the norms in FP64; every sum
// in a fixed order.  GB300's FP64 pipe is narrow (a warp's FP64 instruction
// holds it for about 64 cycles), so nothing per row or per column of a pass
// runs in FP64.
//
// Waits are bounded: a grid barrier that gives up raises the status word, and
// every CTA then leaves its step loop.
#include <float.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "df.cuh"
#include "idsk_internal.h"
#include "tc_common.cuh"

namespace idsk {
namespace {

constexpr int CW = 16;               // consumer warps
constexpr int CT = CW * 32;          // threads (all of them consumers of the passes)
constexpr int NTH = CT;
constexpr int QMAX = 128;            // row quads per CTA (512 rows)
constexpr int HP = kLMax + 1;        // per-CTA partials: V^T u (kLMax), ||u||^2
constexpr double kRecomputeFrac = 1.0 / (1 << 20);
// cint slots (shared with coarse.cu's layout where the host reads them)
constexpr int CI_P = 0, CI_STOP = 1, CI_NREC = 2, CI_KOUT = 3, CI_BAR_CNT = 4, CI_BAR_GEN = 5,
              CI_NREC_ODD = 6;
// the recompute counter of step s: slot CI_NREC (even s) or CI_NREC_ODD (odd
// s); CTA 0 clears the slot of step s during step s, whose users all passed
// step s - 2's barriers long before
__device__ __forceinline__ int nrec_slot(int s) { return (s & 1) ? CI_NREC_ODD : CI_NREC; }
constexpr int CS_ALPHA = 0, CS_SIGMA = 1, CS_BETA = 2, CS_TAU = 3, CS_DEN = 4, CS_TOL = 5;

// Optional timeline of CTA 0 (clock64 at the phase boundaries of every step),
// compiled only when IDSK_CC_TRACE is defined by a profiling harness.
#ifdef IDSK_CC_TRACE
__device__ long long g_cc_trace[64 * 16];
#define CC_TRACE(s, point)                                                        \
  do {                                                                            \
    if (blockIdx.x == 0 && threadIdx.x == 0 && (s) < 64) g_cc_trace[(s) * 16 + (point)] = clock64(); \
  } while (0)
#else
#define CC_TRACE(s, point) \
  do {                     \
  } while (0)
#endif

struct CoopArgs {
  const float* Ac;
  int64_t mc;
  int n, kmax, k;
  int64_t ldf;
  float2* V;            // mc x k FP32 pairs, column-major
  double* F;            // F[t * ldf + j]
  double* Rc;           // k x n
  double* nu2;
  double* nu20;
  int* colpos;
  int* Jc;
  double* gpart;        // G x n: per-CTA column partials (FP32 pairs, or FP64 in the recompute)
  float2* upart;        // G x HP
  int* rlist;
  int* cint;
  double* cscal;
  int* status;
  int keep_cols;        // leading columns whose loads are kept in L2 (evict_last)
  double tol_factor;
};

// 128-bit read-only load with an L2 cache policy (createpolicy).
__device__ __forceinline__ float4 ld_f4_hint(const float* p, uint64_t policy) {
  float4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(policy));
  return v;
}

__device__ __forceinline__ unsigned long long norm_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? 0ull : b;
}

__device__ __forceinline__ void cons_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
}

// Grid-wide barrier of the consumer threads of every CTA (cooperative
// launch: all CTAs are resident).  Bounded (LIMIT clock64 cycles): false when
// it gave up (or another CTA did), with the status word raised.
template <long long LIMIT = tc::kWaitCycles>
__device__ bool grid_sync(const CoopArgs& a, int* sflag) {
  cons_sync();
  if (threadIdx.x == 0) {
    volatile int* gen = a.cint + CI_BAR_GEN;
    const int g = *gen;
    __threadfence();
    const int arrived = atomicAdd(a.cint + CI_BAR_CNT, 1);
    if (arrived == (int)gridDim.x - 1) {
      a.cint[CI_BAR_CNT] = 0;
      __threadfence();
      atomicAdd(a.cint + CI_BAR_GEN, 1);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (*(volatile int*)a.status) {
          *sflag = 1;
          break;
        }
        if (clock64() - t0 > LIMIT) {
          atomicOr(a.status, 1);
          *sflag = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  cons_sync();
  return *(volatile int*)sflag == 0;
}

// True when v holds in every consumer thread of the CTA (named barrier 1
// with a predicate AND), so that the CTA's threads take one branch.
__device__ __forceinline__ bool cons_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, %2, q;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(CT)
      : "memory");
  return r != 0;
}

// Fixed-order sum of a double over the consumer threads (warp trees, then
// warps in order); the result is returned to every consumer thread.
__device__ double cons_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  cons_sync();
  if (lane == 0) red[warp] = v;
  cons_sync();
  double s = 0.0;
  for (int w = 0; w < CW; ++w) s += red[w];
  return s;
}

__device__ __forceinline__ void warp_pair_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol);
  }
}

__global__ void __launch_bounds__(NTH, 1)
    coarse_coop_kernel(CoopArgs a) {
  __shared__ int sflag;
  __shared__ __align__(16) float uhs[QMAX * 4];
  __shared__ __align__(16) float uls[QMAX * 4];
  __shared__ float2 fp[kLMax];
  __shared__ double hs[HP], hvec[kLMax], vrow[kLMax];
  __shared__ double red[CW];
  __shared__ unsigned long long pk[CW];
  __shared__ int pi[CW];
  __shared__ double scal[6];   // alpha, sigma, beta, tau, den, tol
  __shared__ int piv, stop_now, nrec_s;
  // 1 / (u_s - beta) of the last step, in FP64 and as an FP32 pair: formed once
  // by thread 0 (an FP64 division per thread costs GB300's narrow FP64 pipe)
  __shared__ double rden_sh;
  __shared__ float2 rdf_sh;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x, b = blockIdx.x;
  const int64_t mc = a.mc;
  const int n = a.n;
  const int64_t Q = mc / 4;
  const int64_t q0 = Q * b / G, q1 = Q * (b + 1) / G;
  const int64_t r0 = 4 * q0;
  const int nrows = (int)(4 * (q1 - q0));
  const int nq = (int)(q1 - q0);
  const int c0 = (int)((int64_t)n * b / G), c1 = (int)((int64_t)n * (b + 1) / G);

  if (tid == 0) {
    sflag = 0;
    rden_sh = 0.0;
    rdf_sh = make_float2(0.f, 0.f);
  }
  __syncthreads();

  // ------------------------------------------------------------ consumers
  float2* const pairs = reinterpret_cast<float2*>(a.gpart);   // the passes' partials
  bool ok = true;
  // One pass over A_c for this CTA's rows: warp w takes columns w, w + CW,
  // ...; lane l loads row quads l, l + 32, ... of a column (128-bit loads,
  // the leading keep_cols columns with an evict-last L2 policy), two columns
  // ahead of the FP32-pair sums; each column's sum goes to its slot of the
  // CTA's partials.  mode 0: sums of squares; mode 1: A^T u with u from
  // uhs / uls.  Columns at or past n load nothing.
  auto pass = [&](int mode) -> bool {
    float4 uh4[QMAX / 32], ul4[QMAX / 32];
#pragma unroll
    for (int e = 0; e < QMAX / 32; ++e) {
      const int q = lane + 32 * e;
      const bool in = mode == 1 && q < nq;
      uh4[e] = in ? *reinterpret_cast<const float4*>(&uhs[4 * q]) : make_float4(0, 0, 0, 0);
      ul4[e] = in ? *reinterpret_cast<const float4*>(&uls[4 * q]) : make_float4(0, 0, 0, 0);
    }
    const uint64_t keep = tc::policy_evict_last(), stream = tc::policy_evict_first();
    auto load_col = [&](int j, float4 (&x)[QMAX / 32]) {
      const float* colp = a.Ac + (int64_t)j * mc + r0;
      const uint64_t pol = j < a.keep_cols ? keep : stream;
#pragma unroll
      for (int e = 0; e < QMAX / 32; ++e) {
        const int q = lane + 32 * e;
        x[e] = (j < n && q < nq) ? ld_f4_hint(colp + 4 * q, pol) : make_float4(0, 0, 0, 0);
      }
    };
    auto col_sum = [&](const float4 (&x)[QMAX / 32], int j) {
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int e = 0; e < QMAX / 32; ++e) {
        if (lane + 32 * e < nq) {
          if (mode == 0) {
            df_acc(hi, lo, x[e].x, x[e].x, 0.f);
            df_acc(hi, lo, x[e].y, x[e].y, 0.f);
            df_acc(hi, lo, x[e].z, x[e].z, 0.f);
            df_acc(hi, lo, x[e].w, x[e].w, 0.f);
          } else {
            df_acc(hi, lo, x[e].x, uh4[e].x, ul4[e].x);
            df_acc(hi, lo, x[e].y, uh4[e].y, ul4[e].y);
            df_acc(hi, lo, x[e].z, uh4[e].z, ul4[e].z);
            df_acc(hi, lo, x[e].w, uh4[e].w, ul4[e].w);
          }
        }
      }
      warp_pair_sum(hi, lo);
      if (lane == 0) pairs[(int64_t)b * n + j] = make_float2(hi, lo);
    };
    float4 x0[QMAX / 32], x1[QMAX / 32], x2[QMAX / 32];
    load_col(warp, x0);
    load_col(warp + CW, x1);
    for (int j = warp; j < n; j += 3 * CW) {
      load_col(j + 2 * CW, x2);
      col_sum(x0, j);
      if (j + CW >= n) break;
      load_col(j + 3 * CW, x0);
      col_sum(x1, j + CW);
      if (j + 2 * CW >= n) break;
      load_col(j + 4 * CW, x1);
      col_sum(x2, j + 2 * CW);
    }
    return true;
  };

  // ---- column norms (pass 0) and the rank tolerance
  ok = cons_all(pass(0));
  ok = grid_sync(a, &sflag) && ok;
  double nsum = 0.0;
  if (ok) {
    for (int j = c0 + tid; j < c1; j += CT) {
      float sh = 0.f, sl = 0.f;   // FP32-pair sum over the CTAs, in CTA order
      for (int bb = 0; bb < G; ++bb) {
        const float2 x = pairs[(int64_t)bb * n + j];
        df_add(sh, sl, x.x, x.y);
      }
      const double s2 = (double)sh + (double)sl;
      a.nu2[j] = s2;
      a.nu20[j] = s2;
      a.colpos[j] = -1;
      nsum += s2;
    }
  }
  nsum = cons_sum(nsum, red);
  if (tid == 0) reinterpret_cast<double*>(a.upart)[(int64_t)b * HP] = nsum;
  ok = ok && grid_sync(a, &sflag);
  if (ok) {
    double tot = 0.0;
    if (tid == 0) {
      for (int bb = 0; bb < G; ++bb) tot += reinterpret_cast<const double*>(a.upart)[(int64_t)bb * HP];
      scal[5] = a.tol_factor * DBL_EPSILON * sqrt(tot);
      if (b == 0) {
        a.cscal[CS_TOL] = scal[5];
        a.cint[CI_STOP] = 0;
        a.cint[CI_KOUT] = 0;
      }
    }
  }
  cons_sync();

  int s = 0;
  for (; ok && s < a.kmax; ++s) {
    // ---------------------------------------------------------- phase A
    // pivot: largest residual norm, ties to the lowest index
    CC_TRACE(s, 0);
    {
      unsigned long long v = 0ull;
      int idx = 0x7fffffff;
      for (int j = tid; j < n; j += CT) {
        const int cp = a.colpos[j];
        if (cp >= 0 && cp < s) continue;
        const unsigned long long key = norm_key(a.nu2[j]);
        if (idx == 0x7fffffff || key > v) {
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
      if (lane == 0) {
        pk[warp] = v;
        pi[warp] = idx;
      }
      cons_sync();
      if (tid == 0) {
        unsigned long long bv = pk[0];
        int p = pi[0];
        for (int w = 1; w < CW; ++w)
          if (pi[w] != 0x7fffffff && (p == 0x7fffffff || pk[w] > bv || (pk[w] == bv && pi[w] < p))) {
            bv = pk[w];
            p = pi[w];
          }
        const double tol = scal[5];
        const bool stop = p == 0x7fffffff || !(bv > norm_key(tol * tol));
        stop_now = stop ? 1 : 0;
        piv = stop ? -1 : p;
        if (b == 0) {
          if (stop) {
            a.cint[CI_STOP] = 1;
            a.cint[CI_KOUT] = s;
          } else {
            a.cint[CI_P] = p;
            a.Jc[s] = p;
            a.colpos[p] = s;
          }
          a.cint[nrec_slot(s)] = 0;
        }
      }
      cons_sync();
    }
    if (stop_now) break;
    CC_TRACE(s, 1);
    const int p = piv;
    for (int t = tid; t < s; t += CT) fp[t] = df_of(a.F[(int64_t)t * a.ldf + p]);
    cons_sync();
    // v_{s-1} from u_{s-1}, then u = A(:, p) - V_s F(p, :)^T for this CTA's rows
    float2 sig = make_float2(0.f, 0.f);
    const float2 prcp = rdf_sh;   // 1 / (u_{s-1} - beta_{s-1}); zero at s = 0
    for (int rr = tid; rr < nrows; rr += CT) {
      const int64_t i = r0 + rr;
      if (s > 0) {
        float2* vp = a.V + (int64_t)(s - 1) * mc + i;
        if (i == s - 1)
          *vp = make_float2(1.f, 0.f);
        else if (i > s - 1)
          *vp = df_mul(*vp, prcp);
      }
      float2 u = make_float2(0.f, 0.f);
      if (i >= s) {
        u = make_float2(a.Ac[i + (int64_t)p * mc], 0.f);
        for (int t0 = 0; t0 < s; t0 += 16) {
          float2 vv[16];
#pragma unroll
          for (int q = 0; q < 16; ++q)
            vv[q] = t0 + q < s ? a.V[(int64_t)(t0 + q) * mc + i] : make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (t0 + q < s) {
              const float2 pr = df_mul(vv[q], fp[t0 + q]);
              df_add(u.x, u.y, -pr.x, -pr.y);
            }
        }
        u = df_norm(u.x, u.y);
      }
      a.V[(int64_t)s * mc + i] = u;
      const float2 uu = i > s ? u : make_float2(0.f, 0.f);
      uhs[rr] = uu.x;
      uls[rr] = uu.y;
      const float2 u2 = df_mul(uu, uu);
      df_add(sig.x, sig.y, u2.x, u2.y);
    }
    for (int rr = nrows + tid; rr < 4 * QMAX; rr += CT) uhs[rr] = uls[rr] = 0.f;
    cons_sync();
    CC_TRACE(s, 2);
    // partials of V_s^T u (warp w: t = w, w + 16, ...) and ||u||^2; every
    // load of a lane's rows is in flight before the sums (rows lane + 32 e)
    for (int t = warp; t < s; t += CW) {
      float hh = 0.f, hl = 0.f;
      const float2* vc = a.V + (int64_t)t * mc + r0;
      float2 vv[QMAX * 4 / 32];
#pragma unroll
      for (int e = 0; e < QMAX * 4 / 32; ++e) {
        const int rr = lane + 32 * e;
        vv[e] = rr < nrows ? vc[rr] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int e = 0; e < QMAX * 4 / 32; ++e) {
        const int rr = lane + 32 * e;
        if (rr < nrows) {
          const float2 pr = df_mul(vv[e], make_float2(uhs[rr], uls[rr]));
          df_add(hh, hl, pr.x, pr.y);
        }
      }
      warp_pair_sum(hh, hl);
      if (lane == 0) a.upart[(int64_t)b * HP + t] = df_norm(hh, hl);
    }
    warp_pair_sum(sig.x, sig.y);
    if (lane == 0) reinterpret_cast<float2*>(red)[warp] = sig;   // red: CW doubles = CW float2
    cons_sync();
    if (tid == 0) {
      float2 acc = reinterpret_cast<const float2*>(red)[0];
      for (int w = 1; w < CW; ++w) {
        const float2 x = reinterpret_cast<const float2*>(red)[w];
        df_add(acc.x, acc.y, x.x, x.y);
      }
      a.upart[(int64_t)b * HP + kLMax] = df_norm(acc.x, acc.y);
    }
    CC_TRACE(s, 3);
    // A^T u over this CTA's rows (u is zero at and above row s): it needs
    // only this CTA's u, so it runs before the barrier
    ok = cons_all(pass(1));
    CC_TRACE(s, 4);
    if (!ok && tid == 0) atomicOr(a.status, 1);
    if (!grid_sync(a, &sflag) || !ok) {
      ok = false;
      break;
    }
    // ---------------------------------------------------------- phase B
    CC_TRACE(s, 5);
    // Householder scalars and h = V_s^T v_s, every CTA from the partials in
    // a fixed order: quantity g (V_t^T u for g = t < s, ||u||^2 for g = s) is
    // summed by the 8 threads 8 g .. 8 g + 7, thread j over the CTAs b = j
    // mod 8 (all its loads in flight), then a 3-level shuffle tree
    // The loads that do not depend on the sums go first: u_s (thread 0) and
    // v_t[s] (thread t < s; s < CT).
    const float2 us = tid == 0 ? a.V[(int64_t)s * mc + s] : make_float2(0.f, 0.f);
    const float2 vts = tid < s ? a.V[(int64_t)tid * mc + s] : make_float2(0.f, 0.f);
    // and the inputs of this warp's first column of phase C: the CTAs'
    // partials of (A^T u)_j and F(j, 0:s)
    const int jc = c0 + warp;
    float2 gv0[8];   // G <= 256
    double fv0[2];   // s <= 64
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int bb = lane + 32 * e;
      gv0[e] = (jc < c1 && bb < G) ? pairs[(int64_t)bb * n + jc] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int t = lane + 32 * e;
      fv0[e] = (jc < c1 && t < s) ? a.F[(int64_t)t * a.ldf + jc] : 0.0;
    }
    {
      const int g = tid >> 3, j = tid & 7;
      const int q = g < s ? g : (g == s ? kLMax : -1);
      float ah = 0.f, al = 0.f;
      for (int e0 = 0; e0 < (256 + 7) / 8; e0 += 16) {   // 16 loads in flight
        float2 xv[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int bb = j + 8 * (e0 + e);
          xv[e] = (q >= 0 && bb < G) ? a.upart[(int64_t)bb * HP + q] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (j + 8 * (e0 + e) < G) df_add(ah, al, xv[e].x, xv[e].y);
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, ah, o);
        const float ol = __shfl_xor_sync(0xffffffffu, al, o);
        df_add(ah, al, oh, ol);
      }
      if (j == 0 && q >= 0) hs[q] = (double)ah + (double)al;
    }
    cons_sync();
    if (tid == 0) {
      const double sigma = hs[kLMax];
      const double alpha = df_val(us);
      double beta = alpha, tau = 0.0, den = 0.0;
      if (sigma != 0.0) {
        const double nrm = sqrt(alpha * alpha + sigma);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        den = alpha - beta;
      }
      scal[0] = alpha;
      scal[1] = sigma;
      scal[2] = beta;
      scal[3] = tau;
      scal[4] = den;
      rden_sh = sigma != 0.0 ? 1.0 / den : 0.0;
      rdf_sh = df_of(rden_sh);
      if (b == 0) {
        a.cscal[CS_ALPHA] = alpha;
        a.cscal[CS_SIGMA] = sigma;
        a.cscal[CS_BETA] = beta;
        a.cscal[CS_TAU] = tau;
        a.cscal[CS_DEN] = den;
        a.Rc[(int64_t)s * n + p] = beta;
      }
    }
    cons_sync();
    if (tid < s) {
      const double vst = df_val(vts);   // v_t[s], t = tid
      hvec[tid] = vst + hs[tid] * rden_sh;
      vrow[tid] = vst;
    }
    cons_sync();
    // ---------------------------------------------------------- phase C
    // the CTA's columns: warp w takes c0 + w, c0 + w + 16, ...
    CC_TRACE(s, 6);
    {
      const double tau = scal[3], den = scal[4], sigma = scal[1];
      for (int j = c0 + warp; j < c1; j += CW) {
        float2 gv[8];   // every load of the lane in flight (G <= 256, s <= 64)
        double fv[2];
        if (j == jc) {   // loaded at the start of phase B
#pragma unroll
          for (int e = 0; e < 8; ++e) gv[e] = gv0[e];
          fv[0] = fv0[0];
          fv[1] = fv0[1];
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int bb = lane + 32 * e;
            gv[e] = bb < G ? pairs[(int64_t)bb * n + j] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int t = lane + 32 * e;
            fv[e] = t < s ? a.F[(int64_t)t * a.ldf + j] : 0.0;
          }
        }
        // (A^T u)_j: the CTAs' FP32-pair partials summed as FP32 pairs (lane
        // order, then a fixed shuffle tree), one FP64 value at the end
        float gh = 0.f, gl = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) df_add(gh, gl, gv[e].x, gv[e].y);
        warp_pair_sum(gh, gl);
        const double gs = (double)gh + (double)gl;
        double fh = 0.0, rr = 0.0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int t = lane + 32 * e;
          if (t < s) {
            fh += fv[e] * hvec[t];
            rr += vrow[t] * fv[e];
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fh += __shfl_xor_sync(0xffffffffu, fh, o);
          rr += __shfl_xor_sync(0xffffffffu, rr, o);
        }
        if (lane == 0) {
          const int cp = a.colpos[j];
          if (cp >= 0) {
            if (cp < s) a.Rc[(int64_t)s * n + j] = 0.0;   // R(s, p) itself is beta
          } else {
            const double asj = (double)a.Ac[s + (int64_t)j * mc];
            const double gj = sigma != 0.0 ? asj + gs / den : asj;
            const double fjs = tau * (gj - fh);
            a.F[(int64_t)s * a.ldf + j] = fjs;
            const double r = asj - rr - fjs;   // v_s[s] = 1
            a.Rc[(int64_t)s * n + j] = r;
            const double nn = a.nu2[j] - r * r;
            a.nu2[j] = nn;
            if (nn <= kRecomputeFrac * a.nu20[j]) {
              const int slot = atomicAdd(&a.cint[nrec_slot(s)], 1);
              a.rlist[slot] = j;
            }
          }
        }
      }
    }
    CC_TRACE(s, 7);
    if (!grid_sync(a, &sflag)) {
      ok = false;
      break;
    }
    CC_TRACE(s, 8);
    // norms that lost too many bits: recomputed from their definition
    // ||A^(s+1)(s+1:, j)||^2 in FP64, rows split over the CTAs
    if (tid == 0) nrec_s = *(volatile int*)&a.cint[nrec_slot(s)];
    cons_sync();
    const int nrec = nrec_s;
    if (nrec > 0) {
      const double rden = rden_sh;
      for (int idx = 0; idx < nrec; ++idx) {
        const int j = a.rlist[idx];
        double ssum = 0.0;
        for (int rr = tid; rr < nrows; rr += CT) {
          const int64_t i = r0 + rr;
          if (i <= s) continue;
          double x = (double)a.Ac[i + (int64_t)j * mc];
          for (int t = 0; t < s; ++t) x -= df_val(a.V[(int64_t)t * mc + i]) * a.F[(int64_t)t * a.ldf + j];
          x -= df_val(a.V[(int64_t)s * mc + i]) * rden * a.F[(int64_t)s * a.ldf + j];
          ssum += x * x;
        }
        ssum = cons_sum(ssum, red);
        if (tid == 0) a.gpart[(int64_t)b * n + idx] = ssum;
      }
      if (!grid_sync(a, &sflag)) {
        ok = false;
        break;
      }
      for (int idx = tid; idx < nrec; idx += CT) {
        const int j = a.rlist[idx];
        if (j < c0 || j >= c1) continue;
        double ssum = 0.0;
        for (int bb = 0; bb < G; ++bb) ssum += a.gpart[(int64_t)bb * n + idx];
        a.nu2[j] = ssum;
        a.nu20[j] = ssum;
      }
      if (!grid_sync(a, &sflag)) {
        ok = false;
        break;
      }
    }
  }
  // steps done (or stopped): k_out and the unused pivot slots
  if (ok && b == 0) {
    if (tid == 0 && !stop_now) a.cint[CI_KOUT] = s;
    cons_sync();
    const int kout = stop_now ? s : s;
    for (int q = kout + tid; q < a.k; q += CT) a.Jc[q] = -1;
  }
  if (!ok && tid == 0) atomicOr(a.status, 1);
}

// ------------------------------------------------------------------------
// Self-check of the bounded waits' give-up path (no fault, no hang): the
// waits of the kernels above, instantiated with a limit of ~1 ms, on a phase
// or a barrier that nothing completes, and the same waits on one that
// completes.  The status word is raised exactly as in the real kernels.
constexpr long long kCheckWaitCycles = 1ll << 21;
__device__ int g_check_words[8];   // barrier counters (CI_BAR_*) and, in slot 7, the status

// One CTA waits on phase 0 of an mbarrier; `complete`: thread 0 arrives
// first (the phase completes), else nobody does.
__global__ void mbar_check_kernel(int complete, int* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  const uint32_t b = tc::smem_u32(&bar), af = tc::smem_u32(&abort_flag);
  if (threadIdx.x == 0) {
    tc::mbar_init(b, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (complete && threadIdx.x == 0) tc::mbar_arrive(b);
  if (!tc::mbar_wait<kCheckWaitCycles>(b, 0, af)) atomicOr(status, 1);
}

// The coarse kernel's grid barrier over a cooperative launch; `skip`: the
// last CTA returns without reaching it.
__global__ void __launch_bounds__(CT, 1) grid_check_kernel(CoopArgs a, int skip) {
  __shared__ int sflag;
  if (threadIdx.x == 0) sflag = 0;
  __syncthreads();
  if (skip && blockIdx.x == gridDim.x - 1) return;
  if (!grid_sync<kCheckWaitCycles>(a, &sflag) && threadIdx.x == 0) atomicOr(a.status, 1);
}

}  // namespace

#ifdef IDSK_CC_TRACE
// Profiling harness only: clock64 of CTA 0 at the phase boundaries, entry
// [s * 16 + point]: 0 step start, 1 pivot chosen, 2 u formed, 3 partials
// written, 4 pass over A_c done, 5 after the first barrier, 6 scalars done,
// 7 columns finalized, 8 after the second barrier.
extern "C" int idsk_cc_trace_read(long long* host) {
  return (int)cudaMemcpyFromSymbol(host, g_cc_trace, sizeof(g_cc_trace));
}
#endif

// Whether the cooperative form serves this handle: FP32 A_c with m_c a
// multiple of 4 (16-byte row quads) and at most 512 rows per CTA.
bool coarse_coop_ok(const id_sketch* h) { return coarse_coop_ok_ctas(h, 0); }

// The same with at most max_ctas CTAs (0: one per SM).
bool coarse_coop_ok_ctas(const id_sketch* h, int max_ctas) {
  if (h->cfg.dtype != ID_F32 || (h->mc & 3) != 0 || getenv("IDSKETCH_COARSE_MULTI")) return false;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev) != cudaSuccess ||
      !coop) {
    cudaGetLastError();
    return false;
  }
  const int64_t Q = h->mc / 4;
  const int cap = max_ctas > 0 ? std::min(max_ctas, h->nsm) : h->nsm;
  const int64_t G = std::min<int64_t>(cap, Q);
  return Q >= 1 && G >= 1 && G <= 256 && (Q + G - 1) / G <= QMAX && h->coarse_blocks >= G;
}

// Runs one self-check of the bounded waits (modes as id_check_wait) on
// stream st; *gave_up = 1 when the wait gave up and raised the status word.
cudaError_t run_wait_check(int mode, cudaStream_t st, int* gave_up) {
  int* words = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&words, g_check_words);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(words, 0, sizeof(g_check_words), st)) != cudaSuccess) return e;
  if (mode == 0 || mode == 1) {
    mbar_check_kernel<<<1, 32, 0, st>>>(mode == 1, words + 7);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    CoopArgs a;
    memset(&a, 0, sizeof(a));
    a.cint = words;
    a.status = words + 7;
    int skip = mode == 2;
    void* args[] = {&a, &skip};
    e = cudaLaunchCooperativeKernel((const void*)grid_check_kernel, dim3(2), dim3(CT), args, 0,
                                   st);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  int h = 0;
  if ((e = cudaMemcpyAsync(&h, words + 7, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  *gave_up = h != 0;
  return cudaSuccess;
}

cudaError_t launch_coarse_coop(id_sketch* h, int64_t n64, cudaStream_t st, int max_ctas) {
  const int n = (int)n64;
  const int64_t Q = h->mc / 4;
  const int cap = max_ctas > 0 ? std::min(max_ctas, h->nsm) : h->nsm;
  const int G = (int)std::min<int64_t>(cap, Q);   // every CTA owns a row quad
  CoopArgs a;
  a.Ac = reinterpret_cast<const float*>(h->d_Ac);
  a.mc = h->mc;
  a.n = n;
  a.k = h->k;
  a.kmax = (int)std::min<int64_t>(h->k, std::min<int64_t>(h->mc, n64));
  a.ldf = h->n_max;
  a.V = reinterpret_cast<float2*>(h->d_V);
  a.F = h->d_F;
  a.Rc = h->d_Rc;
  a.nu2 = h->d_nu2;
  a.nu20 = h->d_nu20;
  a.colpos = h->d_colposc;
  a.Jc = h->d_Jc;
  a.gpart = h->d_gvec;
  a.upart = reinterpret_cast<float2*>(h->d_upart);
  a.rlist = h->d_rlist;
  a.cint = h->d_cint;
  a.cscal = h->d_cscal;
  a.status = h->d_status;
  a.tol_factor = ID_RANK_TOL_FACTOR;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->dev) != cudaSuccess) {
    cudaGetLastError();
    l2 = 0;
  }
  // about 3/8 of L2 holds the leading columns of A_c from one step to the next
  double keep = 0.375;
  if (const char* env = getenv("IDSKETCH_COARSE_L2_KEEP")) keep = atof(env);
  a.keep_cols = (int)std::min<int64_t>(
      n, (int64_t)(std::max(0.0, std::min(1.0, keep)) * l2 / (4.0 * (double)h->mc)));
  cudaError_t e = cudaMemsetAsync(h->d_cint, 0, 8 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)coarse_coop_kernel, dim3(G), dim3(NTH), args, 0,
                                  st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return launch_solve_p(h->d_Rc, h->d_Jc, h->d_colposc, h->d_cint + CI_KOUT, h->k, n, h->d_Pc,
                        st);
}

}  // namespace idsk
