// Fused reconstruction-error pass on the tcgen05 tensor cores (FP32 data).
//
// One read of A gives ||A - A(:,J) P||_F^2, ||A||_F^2 and
// max |A_ij - A_hat_ij| / |A_ij| over A_ij != 0 (the Frobenius metric of
// Sec. 3.3 and the entry-wise metric of Sec. 3.1), A_hat = A(:,J) P being the
// ID of eq. eqn:id written for columns.
//
// Each CTA owns one 256-column tile C and a contiguous range of 128-row
// blocks R (the CTAs of one row range run side by side, so the skeleton rows
// A(R, J) they all gather come from L2 after the first read):
//   A_hat(R, C) = A(R, J) P(:, C)   M = 128 rows, N = 256 columns, K = k <= 64
// Precision: A(R, J) (FP32) and P (FP64) are each split into three bfloat16
// pieces and the six products with an exponent sum up to 2^-16 are formed
// (a0p0, a0p1, a1p0, a0p2, a1p1, a2p0), which reproduces A_hat to about FP32
// accuracy; the residual and its square are then taken in FP32 against A
// itself, read once from global memory by the epilogue.
//
// Warp roles:
//   warps 0-7   epilogue: stream A(R, C) (warp w: TMEM lane quarter w % 4,
//               128 columns w / 4), read A_hat from TMEM, accumulate the
//               statistics
//   warps 8-11  gather A(R, J): one row per thread, all k loads of the row
//               issued at once, split, store the pieces (double-buffered)
//   warp 12     TMEM allocation and the single-thread tcgen05.mma issue
//   warp 13     (TMA form) streams A(R, C) in boxes of 128 rows x 32 columns
//               through a 4-stage shared-memory ring for the epilogue
// At most 4 warps per SM sub-partition (128 registers each).  The TMA form
// (A 16-byte aligned, lda a multiple of 4) keeps 80 KB of A in flight per SM
// and single-buffers the skeleton pieces to make room; the other form loads
// A in the epilogue warps directly.
// Waits are bounded as in the sketch kernel; on timeout the status word is
// set and the host reports ID_ERR_TIMEOUT.
#include <cuda_bf16.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "idsk_internal.h"
#include "tc_common.cuh"

namespace idsk {
namespace {

using namespace tc;

constexpr int TR = 128;
constexpr int TN = 256;                  // columns per CTA tile
constexpr int KP = 64;                   // padded rank
constexpr int NEPI = 8;
constexpr int NGAT = 4;
constexpr int MMA_WARP = NEPI + NGAT;    // 12
constexpr int NTHREADS = (NEPI + NGAT + 1) * 32;
constexpr int PROD_WARP = MMA_WARP + 1;  // TMA producer (TMA form only)
constexpr int NTHREADS_TMA = NTHREADS + 32;
constexpr int NST = 5;                   // A boxes of 128 rows x 32 columns in flight
constexpr uint32_t RAW_BYTES = TR * 32 * 4;   // 16 KB
constexpr uint32_t S_PIECE = TR * KP * 2;   // 16 KB
constexpr uint32_t P_PIECE = TN * KP * 2;   // 32 KB
constexpr uint32_t IDESC = idesc_bf16(TR, TN, 0);

enum { B_SF0 = 0, B_SF1, B_SE0, B_SE1, B_DF0, B_DF1, B_DE0, B_DE1, B_DONE, B_RF0,
       B_RE0 = B_RF0 + NST, NBAR = B_RE0 + NST };

// Optional timeline of CTA 0, compiled only when IDSK_RC_TRACE is defined by a
// profiling harness.
#ifdef IDSK_RC_TRACE
__device__ long long g_rc_trace[4][4096];
#define RC_TRACE(role, idx)                                                   \
  do {                                                                        \
    if (blockIdx.x == 0 && (idx) < 4096) g_rc_trace[role][idx] = clock64();   \
  } while (0)
#else
#define RC_TRACE(role, idx) \
  do {                      \
  } while (0)
#endif


template <typename T>
struct Kahan {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

__device__ __forceinline__ void split3(float x, uint16_t& p0, uint16_t& p1, uint16_t& p2) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h0);
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h1);
  const __nv_bfloat16 h2 = __float2bfloat16_rn(r2);
  p0 = *reinterpret_cast<const uint16_t*>(&h0);
  p1 = *reinterpret_cast<const uint16_t*>(&h1);
  p2 = *reinterpret_cast<const uint16_t*>(&h2);
}

// TMA: A(R, C) reaches the epilogue through an NST-stage ring of TMA boxes
// (producer warp 13) and the skeleton pieces are single-buffered to make room;
// otherwise the epilogue loads A itself and the pieces are double-buffered.
// INTERP: the skeleton rows are interpolated from the coarse skeleton
// (single-pass ID) instead of gathered from A; a separate instantiation, so
// that the plain error pass carries none of that code (the kernel's roles
// share the instruction cache).
template <bool TMA, bool INTERP>
__global__ void __launch_bounds__(TMA ? NTHREADS_TMA : NTHREADS, 1)
    recon_tc_kernel(const float* __restrict__ A, int64_t lda, int64_t m, int n,
                    const int* __restrict__ J, const double* __restrict__ P, int k,
                    double* __restrict__ part, int* __restrict__ status, InterpGeom geo,
                    const __grid_constant__ CUtensorMap tmap) {
  constexpr int NSB = TMA ? 1 : 2;                 // skeleton piece buffers
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t s_p = base;                       // P pieces: 3 x 32 KB
  const uint32_t s_s = s_p + 3u * P_PIECE;         // S pieces: NSB buffers x 3 x 16 KB
  const uint32_t s_raw = s_s + (uint32_t)NSB * 3u * S_PIECE;   // TMA: NST x 16 KB
  const uint32_t bars = s_raw + (TMA ? NST * RAW_BYTES : 0u);
  const uint32_t tmem_slot = bars + NBAR * 8u;
  const uint32_t abort_flag = tmem_slot + 4u;
  __shared__ int Js[kRecKMax];
  __shared__ double red[3][NEPI];
  auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_ct = (n + TN - 1) / TN;
  const int ct = blockIdx.x % n_ct;
  const int rr = blockIdx.x / n_ct;
  const int nrr = gridDim.x / n_ct;
  const int64_t nrb = (m + TR - 1) / TR;
  const int64_t rb_begin = nrb * rr / nrr, rb_end = nrb * (rr + 1) / nrr;
  const int nloc = (int)(rb_end - rb_begin);
  const int c0 = ct * TN;

  if (tid == 0) {
    mbar_init(bar(B_SF0), NGAT);
    mbar_init(bar(B_SF1), NGAT);
    mbar_init(bar(B_SE0), 1);
    mbar_init(bar(B_SE1), 1);
    mbar_init(bar(B_DF0), 1);
    mbar_init(bar(B_DF1), 1);
    mbar_init(bar(B_DE0), NEPI);
    mbar_init(bar(B_DE1), NEPI);
    mbar_init(bar(B_DONE), 1);
    if (TMA) {
      for (int q = 0; q < NST; ++q) {
        mbar_init(bar(B_RF0 + q), 1);
        mbar_init(bar(B_RE0 + q), NEPI / 2);   // the 4 warps of one column half
      }
    }
    st_volatile_shared(abort_flag, 0);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int u = tid; u < k; u += NTHREADS) Js[u] = J[u];
  // P(:, C) split into three bf16 pieces: K-major B operand, row = column c
  for (int e = tid; e < TN * KP; e += NTHREADS) {
    const int c = e / KP, t = e % KP;
    double v = 0.0;
    if (t < k && c0 + c < n) v = P[(int64_t)t * n + c0 + c];
    // the three 8-bit pieces hold 24 bits: split the FP32 rounding of P on
    // the FP32 units (the FP64 split cost a sizeable share of a launch)
    uint16_t p0, p1, p2;
    split3((float)v, p0, p1, p2);
    const uint32_t off = swz((uint32_t)c, (uint32_t)t, 1024u);
    st_shared_u16(s_p + off, p0);
    st_shared_u16(s_p + P_PIECE + off, p1);
    st_shared_u16(s_p + 2u * P_PIECE + off, p2);
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     tmem_slot)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(tmem_slot) : "memory");

  if (warp < NEPI) {
    // -------------------------------------------------------------- epilogue
    const int q = warp & 3;                  // TMEM lane quarter
    const int ch = warp >> 2;                // column half of the tile (128 columns)
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    Kahan<float> res, tot;
    float mx = 0.f;
    // per row block: four chunks of 32 columns; the 32 loads of a chunk are
    // issued before its TMEM read.
    // Per element: one residual, two FMAs into chunk sums (folded into the
    // Kahan accumulators once per chunk), and a division-free running maximum
    // of |e| / |a| kept as the pair (bn, bd) = (|e|, |a|) of the best entry.
    float bn = 0.f, bd = 1.f;
    bool ok = true;
    for (int i = 0; i < nloc && ok; ++i) {
      const int b = i & 1;
      const int64_t r = (rb_begin + i) * TR + q * 32 + lane;
      const bool rok = r < m;
#pragma unroll 1
      for (int c4 = 0; c4 < 4; ++c4) {
        const int cb = c0 + ch * 128 + c4 * 32;
        const bool full = rok && (cb + 31 < n);
        float v[32];
        if constexpr (TMA) {
          // box u of the ring sequence: row block i, column half ch, chunk c4
          // (zero-filled outside the matrix)
          const int u = i * 8 + 2 * c4 + ch, st = u % NST;
          if (!mbar_wait(bar(B_RF0 + st), (u / NST) & 1, abort_flag, 64)) {
            ok = false;
            break;
          }
          const float* box =
              reinterpret_cast<const float*>(smem_raw + (s_raw - smem_u32(smem_raw))) +
              st * (RAW_BYTES / 4) + q * 32 + lane;
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = box[j * TR];
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_RE0 + st));
        } else if (full) {
          const float* p = A + r + (int64_t)cb * lda;
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __ldcs(p + (int64_t)j * lda);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            v[j] = (rok && cb + j < n) ? __ldcs(A + r + (int64_t)(cb + j) * lda) : 0.f;
        }
        if (c4 == 0) {
          if (!mbar_wait(bar(B_DF0 + b), (i >> 1) & 1, abort_flag, 128)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        float d[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(b * TN + ch * 128 + c4 * 32), d);
        if (!full) {   // entries outside the matrix contribute nothing
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (!(rok && cb + j < n)) d[j] = 0.f;
        }
        float se = 0.f, sa = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float a = v[j];
          const float e = a - d[j];
          se = fmaf(e, e, se);
          sa = fmaf(a, a, sa);
          const float ae = fabsf(e), aa = fabsf(a);
          const bool better = (aa != 0.f) && (ae * bd > bn * aa);
          bn = better ? ae : bn;
          bd = better ? aa : bd;
        }
        res.add(se);
        tot.add(sa);
      }
      if (!ok) break;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_DE0 + b));
      if (warp == 0 && lane == 0) RC_TRACE(0, i);
    }
    mx = bn / bd;
    double s0 = (double)res.s - (double)res.c, s1 = (double)tot.s - (double)tot.c, s2 = mx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 = fmax(s2, __shfl_xor_sync(0xffffffffu, s2, o));
    }
    if (lane == 0) {
      red[0][warp] = s0;
      red[1][warp] = s1;
      red[2][warp] = s2;
    }
  } else if (warp < MMA_WARP) {
    // ---------------------------------------------------------------- gather
    const int rl = tid - NEPI * 32;          // row of the block owned by this thread
    uint8_t* sm_gen = smem_raw + (s_s - smem_u32(smem_raw));
    // 8 skeleton values of this row, entries t0..t0+7: split into the three
    // pieces and stored as one 16-byte chunk of each piece
    auto store8 = [&](uint8_t* sbp, int t0, const float* x8) {
      uint32_t w[3][4];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        uint16_t a0, a1, a2, b0, b1, b2;
        split3(x8[u], a0, a1, a2);
        split3(x8[u + 1], b0, b1, b2);
        w[0][u >> 1] = (uint32_t)a0 | ((uint32_t)b0 << 16);
        w[1][u >> 1] = (uint32_t)a1 | ((uint32_t)b1 << 16);
        w[2][u >> 1] = (uint32_t)a2 | ((uint32_t)b2 << 16);
      }
      const uint32_t off = swz((uint32_t)rl, (uint32_t)t0, 1024u);   // 16 bytes
#pragma unroll
      for (int p = 0; p < 3; ++p)
        *reinterpret_cast<uint4*>(sbp + p * S_PIECE + off) =
            make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    };
    bool gok = true;
    for (int i = 0; i < nloc && gok; ++i) {
      const int b = i % NSB, use = i / NSB;
      const int64_t r = (rb_begin + i) * TR + rl;
      const bool rok = r < m;
      uint8_t* sbp = sm_gen + (size_t)b * 3u * S_PIECE;
      if constexpr (!INTERP) {
        // all k loads of the row in flight at once (the gather warps are on
        // the error pass's critical path), then split and stored
        float x[KP];
#pragma unroll
        for (int t = 0; t < KP; ++t) x[t] = (t < k && rok) ? A[r + (int64_t)Js[t] * lda] : 0.f;
        if (use >= 1 && !mbar_wait(bar(B_SE0 + b), (use - 1) & 1, abort_flag, 64)) {
          gok = false;
          break;
        }
#pragma unroll
        for (int t0 = 0; t0 < KP; t0 += 8) store8(sbp, t0, x + t0);
      } else {   // single-pass ID: the skeleton row interpolated from the coarse one
        float x[KP];
#pragma unroll
        for (int t = 0; t < KP; ++t) x[t] = 0.f;
        if (rok) {
          int64_t idx[8];
          float w[8];
          interp_corners<float>(r, geo, idx, w);
          const float4* sc = reinterpret_cast<const float4*>(geo.Sc);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4* row = sc + idx[q] * (kSkelLd / 4);
#pragma unroll
            for (int t4 = 0; t4 < KP / 4; ++t4) {
              if (4 * t4 < k) {
                const float4 v = row[t4];
                x[4 * t4] = fmaf(w[q], v.x, x[4 * t4]);
                x[4 * t4 + 1] = fmaf(w[q], v.y, x[4 * t4 + 1]);
                x[4 * t4 + 2] = fmaf(w[q], v.z, x[4 * t4 + 2]);
                x[4 * t4 + 3] = fmaf(w[q], v.w, x[4 * t4 + 3]);
              }
            }
          }
        }
        if (use >= 1 && !mbar_wait(bar(B_SE0 + b), (use - 1) & 1, abort_flag, 64)) {
          gok = false;
          break;
        }
#pragma unroll
        for (int t0 = 0; t0 < KP; t0 += 8) store8(sbp, t0, x + t0);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_SF0 + b));
      if (rl == 0) RC_TRACE(1, i);
    }
  } else if (warp == MMA_WARP && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    for (int i = 0; i < nloc; ++i) {
      const int b = i & 1;                  // TMEM accumulator
      const int sbuf = i % NSB, suse = i / NSB;   // skeleton piece buffer
      if (!mbar_wait(bar(B_SF0 + sbuf), suse & 1, abort_flag, 64)) break;
      if (i >= 2 && !mbar_wait(bar(B_DE0 + b), ((i >> 1) - 1) & 1, abort_flag, 64)) break;
      tc_fence_after();
      RC_TRACE(2, i);
      const uint32_t sb = s_s + (uint32_t)sbuf * 3u * S_PIECE;
      const uint32_t d = tmem + (uint32_t)(b * TN);
      // base descriptors of the three pieces of each operand; a K step only
      // moves the start-address field (32 bytes = 2 units of 16)
      const uint64_t dS0 = sdesc(sb, 0u, 1024u), dP0 = sdesc(s_p, 0u, 1024u);
      constexpr uint64_t kS = S_PIECE >> 4, kPp = P_PIECE >> 4;
      for (int kk = 0; kk < KP / 16; ++kk) {
        const uint64_t ko = (uint64_t)(2 * kk);
        // piece products a0p0, a0p1, a1p0, a0p2, a1p1, a2p0
        mma_bf16(d, dS0 + ko, dP0 + ko, IDESC, (uint32_t)kk);
        mma_bf16(d, dS0 + ko, dP0 + kPp + ko, IDESC, 1u);
        mma_bf16(d, dS0 + kS + ko, dP0 + ko, IDESC, 1u);
        mma_bf16(d, dS0 + ko, dP0 + 2 * kPp + ko, IDESC, 1u);
        mma_bf16(d, dS0 + kS + ko, dP0 + kPp + ko, IDESC, 1u);
        mma_bf16(d, dS0 + 2 * kS + ko, dP0 + ko, IDESC, 1u);
      }
      mma_commit(bar(B_DF0 + b));
      mma_commit(bar(B_SE0 + sbuf));
    }
    mma_commit(bar(B_DONE));
    const long long t0 = clock64();
    while (!mbar_try(bar(B_DONE), 0)) {
      if (clock64() - t0 > kWaitCycles) {
        st_volatile_shared(abort_flag, 1);
        break;
      }
    }
  } else if (TMA && warp == PROD_WARP && lane == 0) {
    // ------------------------------------------------------- TMA producer
    const uint64_t tm = reinterpret_cast<uint64_t>(&tmap);
    const uint64_t once = policy_evict_first();
    int u = 0;
    bool ok = true;
    for (int i = 0; i < nloc && ok; ++i) {
      const int row = (int)((rb_begin + i) * TR);
      for (int bi = 0; bi < 8; ++bi, ++u) {   // chunk c4 = bi / 2 of column half bi % 2
        const int st = u % NST;
        if (u >= NST && !mbar_wait(bar(B_RE0 + st), ((u / NST) - 1) & 1, abort_flag, 32)) {
          ok = false;
          break;
        }
        mbar_expect_tx(bar(B_RF0 + st), RAW_BYTES);
        tma_load_2d(s_raw + (uint32_t)st * RAW_BYTES, tm, row, c0 + (bi & 1) * 128 + (bi >> 1) * 32,
                    bar(B_RF0 + st), once);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
  if (tid == 0) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int w = 0; w < NEPI; ++w) {
      a0 += red[0][w];
      a1 += red[1][w];
      a2 = fmax(a2, red[2][w]);
    }
    part[3 * blockIdx.x + 0] = a0;
    part[3 * blockIdx.x + 1] = a1;
    part[3 * blockIdx.x + 2] = a2;
    if (ld_volatile_shared(abort_flag)) atomicOr(status, 1);
  }
}

}  // namespace

int recon_tc_grid(int64_t m, int64_t n, int nsm) {
  const int n_ct = (int)((n + TN - 1) / TN);
  const int64_t nrb = (m + TR - 1) / TR;
  const int rr = (int)std::max<int64_t>(1, std::min<int64_t>(nrb, nsm / std::max(1, n_ct)));
  return n_ct * rr;
}

cudaError_t launch_recon_tc(const float* A, int64_t lda, int64_t m, int64_t n, const int* J,
                            const double* P, int k, double* part, int grid, int* status,
                            cudaStream_t st, KernelTimer* timer, const InterpGeom* interp) {
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  const char* env = getenv("IDSKETCH_RECON_TMA");
  const bool tma = !(env && env[0] == '0') && make_tmap_f32_2d(A, m, n, lda, TR, 32, &tm);
  const size_t sm = 1024 + 3u * P_PIECE + (tma ? 3u * S_PIECE + NST * RAW_BYTES : 6u * S_PIECE) +
                    NBAR * 8 + 16;
  const bool ip = interp != nullptr && interp->Sc != nullptr;
  auto kern = tma ? (ip ? recon_tc_kernel<true, true> : recon_tc_kernel<true, false>)
                  : (ip ? recon_tc_kernel<false, true> : recon_tc_kernel<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (timer && (e = timer->mark(st)) != cudaSuccess) return e;
  const InterpGeom geo = interp ? *interp : InterpGeom{};
  kern<<<grid, tma ? NTHREADS_TMA : NTHREADS, sm, st>>>(A, lda, m, (int)n, J, P, k, part, status,
                                                         geo, tm);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (timer) e = timer->mark(st);
  return e;
}

}  // namespace idsk
