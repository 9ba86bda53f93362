// Learned skeleton proposal: the network's training and inference kernels.
// No counterpart in the paper (which motivates the ID as the selection of the
// most important snapshots, Sec. 4); the network is
//   s = w2 . gelu(x W1 + b1) + b2,  gelu(z) = z Phi(z)  (exact GELU),
// on features x of a snapshot column (its values on a coarse sub-grid),
// trained on the skeletons of the plain randomized ID with the mean binary
// cross entropy of sigmoid(s).
//
// Kernels (FP32, every sum in a fixed order, no atomics):
//   features_kernel  X(j, f) = scale * A(rows[f], j)
//   gemm_kernel      C = op(A) B on 32 x 32 output tiles staged in shared
//                    memory (K ascending per output); forward: Z = X W1 + b1
//                    with G = gelu(Z) in the epilogue; backward: dW1 = X^T dZ
//   score_kernel     s = G w2 + b2, one warp per column, shuffle tree
//   dscore_kernel    ds = d loss / d s
//   dz_kernel        dZ = ds w2^T .* gelu'(Z)
//   colsum_kernel    column sums (db1 = sum dZ, dw2 = G^T ds)
//   sgd_kernel       p -= lr g
#include <math.h>

#include <atomic>

#include <algorithm>

#include "idsk_internal.h"

namespace idsk {
extern std::atomic<int> g_last_cuda_error;
}

using namespace idsk;

namespace {

constexpr int GT = 32;   // GEMM output tile

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

// C (M x N, row-major, ldc = N) = op(A) (M x K) B (K x N, row-major), op(A)
// read as A[i * K + k] or, transposed, A[k * M + i].  mode 1: C += bias[col],
// G = gelu(C) written to G (ldg = N).
__global__ void __launch_bounds__(256) gemm_kernel(const float* __restrict__ A,
                                                   const float* __restrict__ B, int M, int N,
                                                   int K, int transA,
                                                   const float* __restrict__ bias,
                                                   float* __restrict__ C, float* __restrict__ G,
                                                   int mode) {
  __shared__ float As[GT][GT + 1];   // As[k][i]
  __shared__ float Bs[GT][GT + 1];   // Bs[k][j]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < K; k0 += GT) {
    // consecutive threads read consecutive addresses: along i for A^T and
    // for B's columns, along k for A
    for (int e = threadIdx.x; e < GT * GT; e += 256) {
      const int q = e / GT, r = e % GT;
      if (transA) {
        const int i = i0 + r, k = k0 + q;
        As[q][r] = (i < M && k < K) ? A[(int64_t)k * M + i] : 0.f;
      } else {
        const int i = i0 + q, k = k0 + r;
        As[r][q] = (i < M && k < K) ? A[(int64_t)i * K + k] : 0.f;
      }
      const int k = k0 + q, j = j0 + r;
      Bs[q][r] = (k < K && j < N) ? B[(int64_t)k * N + j] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GT; ++kk) {
      const float a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const float b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      if (i < M && j < N) {
        float v = acc[r][c];
        if (mode == 1) {
          v += bias[j];
          G[(int64_t)i * N + j] = gelu_f(v);
        }
        C[(int64_t)i * N + j] = v;
      }
    }
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

id_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ID_OK;
  g_last_cuda_error.store((int)e);
  return ID_ERR_CUDA;
}

int blocks_for(int64_t count, int threads) { return (int)((count + threads - 1) / threads); }

bool gemm_dims_ok(int64_t M, int64_t N, int64_t K) {
  return M >= 1 && N >= 1 && K >= 1 && M <= (1 << 24) && N <= (1 << 24) && K <= (1 << 24) &&
         (M + GT - 1) / GT <= 65535;
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
  const dim3 grid((unsigned)((H + GT - 1) / GT), (unsigned)((n + GT - 1) / GT));
  gemm_kernel<<<grid, 256, 0, st>>>(d_X, d_W1, (int)n, H, (int)F, 0, d_b1, d_Z, d_G, 1);
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
  const dim3 grid((unsigned)((H + GT - 1) / GT), (unsigned)((F + GT - 1) / GT));
  gemm_kernel<<<grid, 256, 0, st>>>(d_X, d_dZ, (int)F, H, (int)n, 1, nullptr, d_gW1, nullptr,
                                    0);                                          // X^T dZ
  count_launches(6);
  return cuda_status(cudaGetLastError());
}

id_status id_mlp_sgd(float* d_p, const float* d_g, int64_t count, float lr, void* cuda_stream) {
  if (!d_p || !d_g || count < 1 || !isfinite(lr)) return ID_ERR_INVALID_ARG;
  if (count / 256 + 1 > ((int64_t)1 << 31) - 1) return ID_ERR_INVALID_ARG;
  sgd_kernel<<<blocks_for(count, 256), 256, 0, (cudaStream_t)cuda_stream>>>(d_p, d_g, count, lr);
  count_launches(1);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
