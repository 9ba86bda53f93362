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
//      of A^T u: its rows of every column, streamed from HBM in TMA boxes
//      through a shared-memory ring (the producer warp runs ahead across
//      steps: A_c does not change), one partial per (CTA, column);
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
// Waits are bounded: a grid barrier or a ring wait that gives up raises the
// status word; every CTA then leaves its step loop and waits (bounded) for
// its own bulk copies before it exits.
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
constexpr int CT = CW * 32;          // consumer threads
constexpr int NTH = CT + 32;         // + the producer warp
constexpr int RING = 6;              // stages of the A_c ring
constexpr int PF_STAGES = 8;         // stages streamed into L2 ahead of the ring loads
constexpr uint32_t STAGE_MAX = 32768;
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
  int keep_cols;        // columns whose ring loads are kept in L2 (evict_last)
  int sgc;              // columns per ring stage
  int box_rows;         // rows per TMA box (two boxes cover a CTA's rows)
  double tol_factor;
};

__device__ __forceinline__ unsigned long long norm_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? 0ull : b;
}

__device__ __forceinline__ void cons_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(CT) : "memory");
}

// Grid-wide barrier of the consumer threads of every CTA (cooperative
// launch: all CTAs are resident).  Bounded: false when it gave up (or another
// CTA did), with the status word raised.
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
        if (clock64() - t0 > tc::kWaitCycles) {
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
    coarse_coop_kernel(CoopArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * RING];
  __shared__ int abort_flag, stop_flag, sflag;
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

  const uint32_t ring = (tc::smem_u32(smem_raw) + 127u) & ~127u;
  const uint8_t* ringp = smem_raw + (ring - tc::smem_u32(smem_raw));
  const uint32_t full0 = tc::smem_u32(&bars[0]), empty0 = tc::smem_u32(&bars[RING]);
  const uint32_t abort_a = tc::smem_u32(&abort_flag);
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
  const int sgc = a.sgc;
  const int box_rows = a.box_rows;
  const uint32_t box_bytes = (uint32_t)(box_rows * sgc * 4);
  const int nstage = (n + sgc - 1) / sgc;
  const uint32_t stage_bytes = 2u * box_bytes;

  if (tid == 0) {
    for (int q = 0; q < RING; ++q) {
      tc::mbar_init(full0 + 8u * q, 1);
      tc::mbar_init(empty0 + 8u * q, CW);
    }
    abort_flag = 0;
    stop_flag = 0;
    sflag = 0;
    rden_sh = 0.0;
    rdf_sh = make_float2(0.f, 0.f);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == CW) {
    // ------------------------------------------------------------ producer
    // Stage u holds columns [sgc * (u % nstage), ...) of this CTA's rows, for
    // pass u / nstage (pass 0: the norms, pass 1 + s: step s), as two TMA
    // boxes of box_rows rows x sgc columns (column-major, zero fill past the
    // matrix).  A_c does not change, so the producer runs ahead across steps,
    // bounded by the ring.
    if (lane == 0) {
      const uint64_t tm = reinterpret_cast<uint64_t>(&tmap);
      const uint64_t keep = tc::policy_evict_last(), stream = tc::policy_evict_first();
      const int64_t total = (int64_t)(1 + a.kmax) * nstage;
      int64_t u = 0, pf = 1;   // pf: next stage to prefetch into L2
      for (; u < total; ++u) {
        const int slot = (int)(u % RING);
        // keep PF_STAGES stages ahead of this load on their way into L2 (the
        // kept columns are there already), so that the ring's loads hit L2
        // also right after the scalar and column phases of a step
        for (; pf <= u + PF_STAGES && pf < total; ++pf) {
          const int pj0 = (int)(pf % nstage) * sgc;
          if (pj0 >= a.keep_cols) {
            tc::tma_prefetch_2d(tm, (int)r0, pj0);
            tc::tma_prefetch_2d(tm, (int)r0 + box_rows, pj0);
          }
        }
        if (u >= RING) {
          const uint32_t par = (uint32_t)(((u / RING) - 1) & 1);
          const long long t0 = clock64();
          bool ok = true;
          while (!tc::mbar_try(empty0 + 8u * slot, par)) {
            if (*(volatile int*)&stop_flag || *(volatile int*)&abort_flag) {
              ok = false;
              break;
            }
            if (clock64() - t0 > tc::kWaitCycles) {
              tc::st_volatile_shared(abort_a, 1);
              ok = false;
              break;
            }
          }
          if (!ok) break;
        }
        const int st = (int)(u % nstage);
        const int j0 = st * sgc;
        const uint64_t pol = j0 < a.keep_cols ? keep : stream;
        tc::mbar_expect_tx(full0 + 8u * slot, stage_bytes);
        tc::tma_load_2d(ring + (uint32_t)slot * stage_bytes, tm, (int)r0, j0, full0 + 8u * slot,
                        pol);
        tc::tma_load_2d(ring + (uint32_t)slot * stage_bytes + box_bytes, tm, (int)r0 + box_rows,
                        j0, full0 + 8u * slot, pol);
      }
      // every issued copy has landed before the CTA exits (bounded)
      const int64_t issued = u;
      const int64_t first = issued > RING ? issued - RING : 0;
      for (int64_t v = first; v < issued; ++v) {
        const int slot = (int)(v % RING);
        const long long t0 = clock64();
        while (!tc::mbar_try(full0 + 8u * slot, (uint32_t)((v / RING) & 1)))
          if (clock64() - t0 > tc::kWaitCycles) break;
      }
    }
    return;
  }

  // ------------------------------------------------------------ consumers
  int64_t ucons = 0;   // next ring stage to consume
  float2* const pairs = reinterpret_cast<float2*>(a.gpart);   // the passes' partials
  bool ok = true;
  // One pass over the ring for this CTA's rows: f(column, warp partial pair)
  // receives the warp's FP32-pair sum over the rows of that column.
  // mode 0: sum of squares; mode 1: A^T u with u from uhs / uls.
  auto pass = [&](int mode) -> bool {
    float4 uh4[QMAX / 32], ul4[QMAX / 32];
    if (mode == 1) {
#pragma unroll
      for (int e = 0; e < QMAX / 32; ++e) {
        const int q = lane + 32 * e;
        uh4[e] = q < nq ? *reinterpret_cast<const float4*>(&uhs[4 * q]) : make_float4(0, 0, 0, 0);
        ul4[e] = q < nq ? *reinterpret_cast<const float4*>(&uls[4 * q]) : make_float4(0, 0, 0, 0);
      }
    }
    for (int st = 0; st < nstage; ++st, ++ucons) {
      const int slot = (int)(ucons % RING);
      if (!tc::mbar_wait_spin(full0 + 8u * slot, (uint32_t)((ucons / RING) & 1), abort_a))
        return false;
      const int j0 = st * sgc;
      const int ncols = min(sgc, n - j0);
      for (int c = warp; c < ncols; c += CW) {
        // row quad q of column c: box 0 (rows < box_rows) or box 1
        const uint8_t* col0 = ringp + (size_t)slot * stage_bytes + (size_t)c * box_rows * 4;
        const uint8_t* col1 = col0 + box_bytes - (size_t)box_rows * 4;
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int e = 0; e < QMAX / 32; ++e) {
          const int q = lane + 32 * e;
          if (q < nq) {
            const float4 x = *reinterpret_cast<const float4*>(
                4 * q < box_rows ? col0 + 16 * q : col1 + 16 * q);
            if (mode == 0) {
              df_acc(hi, lo, x.x, x.x, 0.f);
              df_acc(hi, lo, x.y, x.y, 0.f);
              df_acc(hi, lo, x.z, x.z, 0.f);
              df_acc(hi, lo, x.w, x.w, 0.f);
            } else {
              df_acc(hi, lo, x.x, uh4[e].x, ul4[e].x);
              df_acc(hi, lo, x.y, uh4[e].y, ul4[e].y);
              df_acc(hi, lo, x.z, uh4[e].z, ul4[e].z);
              df_acc(hi, lo, x.w, uh4[e].w, ul4[e].w);
            }
          }
        }
        warp_pair_sum(hi, lo);
        // the pair itself: GB300's FP64 units are too narrow for a conversion
        // per column here (a warp's FP64 instruction holds its pipe ~64 cycles)
        if (lane == 0) pairs[(int64_t)b * n + j0 + c] = make_float2(hi, lo);
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(empty0 + 8u * slot);
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
      const double alpha = df_val(a.V[(int64_t)s * mc + s]);
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
    {
      const double rden = rden_sh;
      for (int t = tid; t < s; t += CT) {
        const double vst = df_val(a.V[(int64_t)t * mc + s]);   // v_t[s]
        hvec[t] = vst + hs[t] * rden;
        vrow[t] = vst;
      }
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
  // release the producer (it may wait for ring slots nobody will consume)
  if (tid == 0) tc::st_volatile_shared(tc::smem_u32(&stop_flag), 1);
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
bool coarse_coop_ok(const id_sketch* h) {
  if (h->cfg.dtype != ID_F32 || (h->mc & 3) != 0 || getenv("IDSKETCH_COARSE_MULTI")) return false;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev) != cudaSuccess ||
      !coop) {
    cudaGetLastError();
    return false;
  }
  const int64_t Q = h->mc / 4;
  const int64_t G = std::min<int64_t>(h->nsm, Q);
  return Q >= 1 && G <= 256 && (Q + G - 1) / G <= QMAX && h->coarse_blocks >= G;
}

cudaError_t launch_coarse_coop(id_sketch* h, int64_t n64, cudaStream_t st) {
  const int n = (int)n64;
  const int64_t Q = h->mc / 4;
  const int G = (int)std::min<int64_t>(h->nsm, Q);   // every CTA owns a row quad
  const int64_t qmax = (Q + G - 1) / G;
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
  a.box_rows = (int)(4 * ((qmax + 1) / 2));   // two boxes of at most 256 rows
  a.sgc = (int)std::max<int64_t>(1, std::min<int64_t>(16, STAGE_MAX / (8 * a.box_rows)));
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  if (!make_tmap_f32_2d(h->d_Ac, h->mc, n, h->mc, a.box_rows, a.sgc, &tm))
    return cudaErrorNotSupported;   // the multi-launch path serves it
  a.tol_factor = ID_RANK_TOL_FACTOR;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->dev) != cudaSuccess) {
    cudaGetLastError();
    l2 = 0;
  }
  // about 3/8 of L2 holds the leading columns of A_c from one step to the next
  a.keep_cols = (int)std::min<int64_t>(n, (int64_t)(0.375 * l2 / (4.0 * (double)h->mc)));
  const size_t smem = 128 + (size_t)RING * 8 * a.box_rows * a.sgc;
  cudaError_t e = cudaFuncSetAttribute(coarse_coop_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(h->d_cint, 0, 8 * sizeof(int), st)) != cudaSuccess) return e;
  void* args[] = {&a, &tm};
  e = cudaLaunchCooperativeKernel((const void*)coarse_coop_kernel, dim3(G), dim3(NTH), args,
                                  smem, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return launch_solve_p(h->d_Rc, h->d_Jc, h->d_colposc, h->d_cint + CI_KOUT, h->k, n, h->d_Pc,
                        st);
}

}  // namespace idsk
