// Learned skeleton proposal: the network's training and inference kernels.
// No counterpart in the paper (which motivates the ID as the selection of the
// most important snapshots, Sec. 4); the network is
//   s = w2 . gelu(x W1 + b1) + b2,  gelu(z) = z Phi(z)  (exact GELU),
// on features x of a snapshot column (its values on a coarse sub-grid),
// trained on the skeletons of the plain randomized ID with the mean binary
// cross entropy of sigmoid(s).
//
// Kernels (every sum in a fixed order, no atomics on data):
//   features_kernel  X(j, f) = scale * A(rows[f], j)
//   tc_gemm_kernel   the two dense products on the tcgen05 tensor cores,
//                    bfloat16 operands (weights and features) with FP32
//                    accumulation: forward Z = X W1 + b1 with G = gelu(Z) in
//                    the epilogue; backward dW1 = X^T dZ
//   score_kernel     s = G w2 + b2, one warp per column, shuffle tree
//   dscore_kernel    ds = d loss / d s
//   dz_kernel        dZ = ds w2^T .* gelu'(Z)
//   colsum_kernel    column sums (db1 = sum dZ, dw2 = G^T ds)
//   sgd_kernel       p -= lr g
#include <limits.h>
#include <math.h>

#include <atomic>

#include <algorithm>

#include "idsk_internal.h"
#include "tc_common.cuh"

namespace idsk {
extern std::atomic<int> g_last_cuda_error;
}

using namespace idsk;

namespace {

__device__ __forceinline__ float gelu_f(float z) { return z * normcdff(z); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return normcdff(z) + z * (expf(-0.5f * z * z) * 0.3989422804014327f);
}

// A row index outside [0, m) gives a NaN feature (never an out-of-bounds read).
template <typename T>
__global__ void features_kernel(const T* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                const int64_t* __restrict__ rows, int64_t F, float scale,
                                float* __restrict__ X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * F) return;
  const int64_t j = e / F, f = e - j * F;
  const int64_t r = rows[f];
  X[e] = (r >= 0 && r < m) ? scale * (float)A[r + j * lda] : __int_as_float(0x7fc00000);
}

// ---------------------------------------------------------------------------
// The two dense products of the network on the tcgen05 tensor cores, with
// bfloat16 operands and FP32 accumulation in TMEM:
//   forward   Z (n x H) = X (n x F) W1 (F x H)       [+ b1, G = gelu(Z)]
//   backward  gW1 (F x H) = X^T (F x n) dZ (n x H)
// C (M x N, row-major FP32, ldc = N) = A (M x K) B (K x N), where element
// (i, k) of A is A[i * a_si + k * a_sk] and element (k, j) of B is
// B[k * b_sk + j * b_sj] (FP32 in global memory; any of the two layouts of
// each operand).  Every operand value is rounded to bfloat16 as it is staged,
// so the weights and the features enter the products in bfloat16 and every
// product accumulates in FP32.
//
// One CTA (4 warps) per 128 x 128 output tile: all warps stage 64-wide K
// chunks of A and B (row i of the A tile, row j of the B^T tile) as K-major
// 128-byte-swizzled bfloat16 tiles in two shared-memory stages; one thread
// issues four kind::f16 MMAs (M = N = 128, K = 16) per chunk into a 128-column
// TMEM accumulator and commits them to the stage's mbarrier, so the next
// chunk is staged while the MMAs run.  The epilogue reads the accumulator
// (row i = TMEM lane i) and adds the bias / applies the GELU.  Every output
// is the sum of its K products in ascending chunks: the result does not
// depend on scheduling.  The waits are bounded: on timeout the kernel raises
// g_mlp_abort, writes NaN to its tile and frees its TMEM.
constexpr int TG_M = 128, TG_N = 128, TG_K = 64, TG_THREADS = 128;
constexpr uint32_t TG_TILE_BYTES = TG_M * TG_K * 2;   // 16 KB per operand and stage
constexpr uint32_t TG_IDESC = tc::idesc_bf16(TG_M, TG_N, 0);

__device__ int g_mlp_abort;

// Stage rows [r0, r0 + 128) x K chunk [k0, k0 + 64) of a strided FP32 operand
// (element (r, k) at X[r * s_r + k * s_k], zero outside rows x K) into a
// K-major swizzled bfloat16 tile: each thread writes 16-byte groups of 8
// consecutive k of one row.  With s_k == 1 the 8 lanes of a row read one
// contiguous 32-byte run each; otherwise consecutive lanes take consecutive
// rows (coalesced along r).
__device__ __forceinline__ void stage_tile(const float* __restrict__ X, int64_t s_r,
                                           int64_t s_k, int rows, int K, int r0, int k0,
                                           uint32_t dst) {
  const int tid = threadIdx.x;
  for (int c = tid; c < TG_M * (TG_K / 8); c += TG_THREADS) {
    int rr, q;
    if (s_k == 1) {
      rr = c >> 3;
      q = c & 7;
    } else {
      rr = c & (TG_M - 1);
      q = c >> 7;
    }
    const int r = r0 + rr, kb = k0 + 8 * q;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kb + e;
      v[e] = (r < rows && k < K) ? X[(int64_t)r * s_r + (int64_t)k * s_k] : 0.f;
    }
    const uint32_t off = tc::swz((uint32_t)rr, (uint32_t)(8 * q), 1024u);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + off),
                 "r"(tc::pack_bf16x2(v[0], v[1])), "r"(tc::pack_bf16x2(v[2], v[3])),
                 "r"(tc::pack_bf16x2(v[4], v[5])), "r"(tc::pack_bf16x2(v[6], v[7]))
                 : "memory");
  }
}

// mode 1: C = A B + bias[j] and G = gelu(C); mode 0: C = A B.
__global__ void __launch_bounds__(TG_THREADS, 1) tc_gemm_kernel(
    const float* __restrict__ A, int64_t a_si, int64_t a_sk, const float* __restrict__ B,
    int64_t b_sk, int64_t b_sj, int M, int N, int K, const float* __restrict__ bias,
    float* __restrict__ C, float* __restrict__ G, int mode) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[3];   // two stages, all MMAs done
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const uint32_t base = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sa = base, sb = base + 2 * TG_TILE_BYTES;   // [2][16 KB] each
  const uint32_t bar0 = tc::smem_u32(&bars[0]);
  const uint32_t abort_a = tc::smem_u32(&abort_flag);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.y * TG_M, j0 = blockIdx.x * TG_N;
  if (tid == 0) {
    tc::mbar_init(bar0, 1);
    tc::mbar_init(bar0 + 8, 1);
    tc::mbar_init(bar0 + 16, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&tmem_slot)),
                 "n"(TG_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int nk = (K + TG_K - 1) / TG_K;
  bool ok = true;
  for (int kc = 0; kc < nk; ++kc) {
    const int st = kc & 1;
    // the MMAs of chunk kc - 2 have read this stage
    if (kc >= 2 && !tc::mbar_wait(bar0 + 8u * st, ((kc >> 1) - 1) & 1, abort_a)) ok = false;
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    stage_tile(A, a_si, a_sk, M, K, i0, kc * TG_K, sa + st * TG_TILE_BYTES);
    stage_tile(B, b_sj, b_sk, N, K, j0, kc * TG_K, sb + st * TG_TILE_BYTES);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < TG_K / 16; ++kk)
        tc::mma_bf16(tmem, tc::sdesc(sa + st * TG_TILE_BYTES + 32u * kk, 0u, 1024u),
                     tc::sdesc(sb + st * TG_TILE_BYTES + 32u * kk, 0u, 1024u), TG_IDESC,
                     (uint32_t)(kc | kk));
      tc::mma_commit(bar0 + 8u * st);
    }
  }
  // the last chunk's commit covers every MMA issued before it
  if (ok && nk > 0 && !tc::mbar_wait(bar0 + 8u * ((nk - 1) & 1), ((nk - 1) >> 1) & 1, abort_a))
    ok = false;
  ok = !__syncthreads_or(!ok);
  tc::tc_fence_after();
  const int i = i0 + 32 * warp + lane;   // TMEM lane = output row
  for (int c0 = 0; c0 < TG_N; c0 += 32) {
    float v[32];
    tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
    if (i < M) {
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int j = j0 + c0 + e;
        if (j < N) {
          float z = ok ? v[e] : __int_as_float(0x7fc00000);
          if (mode == 1) {
            z += bias[j];
            G[(int64_t)i * N + j] = gelu_f(z);
          }
          C[(int64_t)i * N + j] = z;
        }
      }
    }
  }
  // every MMA this CTA issued has completed before its TMEM is released
  // (after a timeout as well: bounded)
  if (tid == 0) {
    tc::mma_commit(bar0 + 16);
    const long long t0 = clock64();
    while (!tc::mbar_try(bar0 + 16, 0))
      if (clock64() - t0 > tc::kWaitCycles) {
        ok = false;
        break;
      }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TG_N)
                 : "memory");
  if (tid == 0 && !ok) atomicOr(&g_mlp_abort, 1);
}

constexpr size_t kTgSmem = 1024 + 4 * (size_t)TG_TILE_BYTES;

cudaError_t launch_tc_gemm(const float* A, int64_t a_si, int64_t a_sk, const float* B,
                           int64_t b_sk, int64_t b_sj, int M, int N, int K, const float* bias,
                           float* C, float* G, int mode, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTgSmem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((N + TG_N - 1) / TG_N), (unsigned)((M + TG_M - 1) / TG_M));
  tc_gemm_kernel<<<grid, TG_THREADS, kTgSmem, st>>>(A, a_si, a_sk, B, b_sk, b_sj, M, N, K, bias,
                                                     C, G, mode);
  return cudaGetLastError();
}

// s[j] = sum_h G[j, h] w2[h] + b2: one warp per row, lanes stride h, then a
// fixed shuffle tree.
__global__ void score_kernel(const float* __restrict__ G, int64_t n, int H,
                             const float* __restrict__ w2, const float* __restrict__ b2,
                             float* __restrict__ s) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  float a = 0.f;
  for (int h = lane; h < H; h += 32) a = fmaf(G[j * H + h], w2[h], a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) s[j] = a + b2[0];
}

// ds[j] = d/ds_j of mean_j [ w y softplus(-s) + (1 - y) softplus(s) ]
__global__ void dscore_kernel(const float* __restrict__ s, const float* __restrict__ y,
                              int64_t n, float pos_weight, float* __restrict__ ds) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float v = s[j];
  const float sg = v >= 0.f ? 1.f / (1.f + expf(-v)) : expf(v) / (1.f + expf(v));
  ds[j] = (-pos_weight * y[j] * (1.f - sg) + (1.f - y[j]) * sg) / (float)n;
}

__global__ void dz_kernel(const float* __restrict__ Z, const float* __restrict__ ds,
                          const float* __restrict__ w2, int64_t n, int H,
                          float* __restrict__ dZ) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * H) return;
  const int64_t j = e / H;
  const int h = (int)(e - j * H);
  dZ[e] = ds[j] * w2[h] * gelu_grad_f(Z[e]);
}

// out[h] = sum_j M[j, h] * (v ? v[j] : 1), j ascending (one thread per h)
__global__ void colsum_kernel(const float* __restrict__ Mx, const float* __restrict__ v,
                              int64_t n, int H, float* __restrict__ out) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  float a = 0.f;
  for (int64_t j = 0; j < n; ++j) a = fmaf(Mx[j * H + h], v ? v[j] : 1.f, a);
  out[h] = a;
}

__global__ void sgd_kernel(float* __restrict__ p, const float* __restrict__ g, int64_t count,
                           float lr) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) p[e] -= lr * g[e];
}

// The count columns of highest score, ties to the lower index, written in
// increasing column order (the learned proposal's candidates).  One CTA:
// column j is taken when fewer than count columns rank above it (score
// greater, or equal with a lower index); its output slot is the number of
// taken columns before it.  A NaN score ranks below every number.
constexpr int PR_THREADS = 1024, PR_MAX = 4096;

__device__ __forceinline__ int score_key(float v) {
  if (v != v) return INT_MIN;   // NaN lowest
  if (v == 0.f) return 0;       // -0 ties with +0
  const int b = __float_as_int(v);
  return b >= 0 ? b : (int)(0x80000000u - (unsigned)b) - 1;   // monotone in v
}

// strata > 1: the columns form `strata` consecutive ranges [q n / strata,
// (q + 1) n / strata) and column j competes only within its range for `count`
// places (the stratified proposal); strata = 1: one range.
__global__ void __launch_bounds__(PR_THREADS) propose_kernel(const float* __restrict__ s, int n,
                                                              int count, int strata,
                                                              int* __restrict__ cand,
                                                              int* __restrict__ ncand) {
  __shared__ int key[PR_MAX];
  __shared__ unsigned char take[PR_MAX];
  __shared__ int wsum[PR_THREADS / 32];
  for (int j = threadIdx.x; j < n; j += PR_THREADS) key[j] = score_key(s[j]);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += PR_THREADS) {
    const int kj = key[j];
    // the range holding j: the largest q with q n / strata <= j
    int q = (int)(((int64_t)j * strata) / n);
    while (q + 1 < strata && ((int64_t)(q + 1) * n) / strata <= j) ++q;
    while (q > 0 && ((int64_t)q * n) / strata > j) --q;
    const int lo = (int)(((int64_t)q * n) / strata), hi = (int)(((int64_t)(q + 1) * n) / strata);
    int above = 0;
    for (int i = lo; i < hi; ++i) above += (key[i] > kj) || (key[i] == kj && i < j);
    take[j] = above < count;
  }
  __syncthreads();
  // exclusive prefix count of take[] over j, in chunks of PR_THREADS
  int base = 0;
  for (int c0 = 0; c0 < n; c0 += PR_THREADS) {
    const int j = c0 + threadIdx.x;
    const int t = j < n ? take[j] : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (t) cand[base + before + incl - 1] = j;
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < PR_THREADS / 32; ++w) tot += wsum[w];
    base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && ncand) *ncand = base;
}

id_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ID_OK;
  g_last_cuda_error.store((int)e);
  return ID_ERR_CUDA;
}

int blocks_for(int64_t count, int threads) { return (int)((count + threads - 1) / threads); }

bool gemm_dims_ok(int64_t M, int64_t N, int64_t K) {
  return M >= 1 && N >= 1 && K >= 1 && M <= (1 << 24) && N <= (1 << 24) && K <= (1 << 24) &&
         (M + TG_M - 1) / TG_M <= 65535;
}

// The element-wise kernels take one thread per entry of an n x H (or n x 32)
// array: their grid (blocks of 256) must stay below 2^31 blocks.
bool elementwise_grid_ok(int64_t n, int64_t H) {
  return n * std::max<int64_t>(H, 32) / 256 + 1 < ((int64_t)1 << 31);
}

}  // namespace

extern "C" {

id_status id_mlp_features(const void* d_A, int64_t lda, int64_t m, int64_t n, int32_t dtype,
                          const int64_t* d_rows, int64_t F, float scale, float* d_X,
                          void* cuda_stream) {
  if (!d_A || !d_rows || !d_X || m < 1 || n < 1 || F < 1 || lda < m ||
      (dtype != ID_F32 && dtype != ID_F64) || n * F > ((int64_t)1 << 40))
    return ID_ERR_INVALID_ARG;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t tot = n * F;
  if (tot / 256 + 1 > ((int64_t)1 << 31) - 1) return ID_ERR_INVALID_ARG;
  if (dtype == ID_F64)
    features_kernel<double><<<blocks_for(tot, 256), 256, 0, st>>>(
        reinterpret_cast<const double*>(d_A), lda, m, n, d_rows, F, scale, d_X);
  else
    features_kernel<float><<<blocks_for(tot, 256), 256, 0, st>>>(
        reinterpret_cast<const float*>(d_A), lda, m, n, d_rows, F, scale, d_X);
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

id_status id_mlp_forward(const float* d_X, int64_t n, int64_t F, int32_t H, const float* d_W1,
                         const float* d_b1, const float* d_w2, const float* d_b2, float* d_Z,
                         float* d_G, float* d_s, void* cuda_stream) {
  if (!d_X || !d_W1 || !d_b1 || !d_w2 || !d_b2 || !d_Z || !d_G || !d_s || H < 1 ||
      !gemm_dims_ok(n, H, F) || !elementwise_grid_ok(n, H))
    return ID_ERR_INVALID_ARG;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  // Z = X W1: A = X (n x F, row-major), B = W1 (F x H, row-major)
  cudaError_t e = launch_tc_gemm(d_X, F, 1, d_W1, H, 1, (int)n, H, (int)F, d_b1, d_Z, d_G, 1, st);
  if (e != cudaSuccess) return cuda_status(e);
  score_kernel<<<blocks_for(n * 32, 256), 256, 0, st>>>(d_G, n, H, d_w2, d_b2, d_s);
  count_launches(2);
  return cuda_status(cudaGetLastError());
}

id_status id_mlp_backward(const float* d_X, int64_t n, int64_t F, int32_t H, const float* d_Z,
                          const float* d_G, const float* d_w2, const float* d_s,
                          const float* d_y, float pos_weight, float* d_gW1, float* d_gb1,
                          float* d_gw2, float* d_gb2, float* d_ds, float* d_dZ,
                          void* cuda_stream) {
  if (!d_X || !d_Z || !d_G || !d_w2 || !d_s || !d_y || !d_gW1 || !d_gb1 || !d_gw2 || !d_gb2 ||
      !d_ds || !d_dZ || H < 1 || !gemm_dims_ok(F, H, n) || !elementwise_grid_ok(n, H) ||
      !(pos_weight >= 0.f))
    return ID_ERR_INVALID_ARG;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  dscore_kernel<<<blocks_for(n, 256), 256, 0, st>>>(d_s, d_y, n, pos_weight, d_ds);
  dz_kernel<<<blocks_for(n * H, 256), 256, 0, st>>>(d_Z, d_ds, d_w2, n, H, d_dZ);
  colsum_kernel<<<blocks_for(H, 128), 128, 0, st>>>(d_G, d_ds, n, H, d_gw2);    // G^T ds
  colsum_kernel<<<blocks_for(H, 128), 128, 0, st>>>(d_dZ, nullptr, n, H, d_gb1);
  colsum_kernel<<<1, 128, 0, st>>>(d_ds, nullptr, n, 1, d_gb2);                 // sum ds
  // gW1 = X^T dZ: A = X^T (element (f, j) at X[j F + f]), B = dZ (n x H)
  const cudaError_t e =
      launch_tc_gemm(d_X, 1, F, d_dZ, H, 1, (int)F, H, (int)n, nullptr, d_gW1, nullptr, 0, st);
  if (e != cudaSuccess) return cuda_status(e);
  count_launches(6);
  return cuda_status(cudaGetLastError());
}

id_status id_mlp_propose(const float* d_s, int64_t n, int32_t count, int32_t* d_cand,
                         void* cuda_stream) {
  if (!d_s || !d_cand || n < 1 || n > PR_MAX || count < 1 || count > n)
    return ID_ERR_INVALID_ARG;
  propose_kernel<<<1, PR_THREADS, 0, (cudaStream_t)cuda_stream>>>(d_s, (int)n, count, 1, d_cand,
                                                                   nullptr);
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

id_status id_mlp_propose_stratified(const float* d_s, int64_t n, int32_t strata, int32_t per,
                                    int32_t* d_cand, int32_t* d_ncand, void* cuda_stream) {
  if (!d_s || !d_cand || n < 1 || n > PR_MAX || strata < 1 || strata > n || per < 1)
    return ID_ERR_INVALID_ARG;
  propose_kernel<<<1, PR_THREADS, 0, (cudaStream_t)cuda_stream>>>(d_s, (int)n, per, strata,
                                                                   d_cand, d_ncand);
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

id_status id_mlp_check(void* cuda_stream) {
  if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess)
    return cuda_status(cudaGetLastError());
  int flag = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbol(&flag, g_mlp_abort, sizeof(int)) != cudaSuccess ||
      (flag && cudaMemcpyToSymbol(g_mlp_abort, &zero, sizeof(int)) != cudaSuccess))
    return cuda_status(cudaGetLastError());
  return flag ? ID_ERR_TIMEOUT : ID_OK;
}

id_status id_mlp_sgd(float* d_p, const float* d_g, int64_t count, float lr, void* cuda_stream) {
  if (!d_p || !d_g || count < 1 || !isfinite(lr)) return ID_ERR_INVALID_ARG;
  if (count / 256 + 1 > ((int64_t)1 << 31) - 1) return ID_ERR_INVALID_ARG;
  sgd_kernel<<<blocks_for(count, 256), 256, 0, (cudaStream_t)cuda_stream>>>(d_p, d_g, count, lr);
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
