// Fused reconstruction-error pass: one read of A gives
//   ||A - A(:,J) P||_F^2, ||A||_F^2 and max_ij |A_ij - A_hat_ij| / |A_ij|
// (Frobenius metric of Sec. 3.3; entry-wise metric of Sec. 3.1, skipping
// A_ij == 0 where the ratio is undefined).  The reconstruction
// A_hat = A(:,J) P is the ID of eq. eqn:id written for columns; the skeleton
// block A(R, J) is gathered once per row tile R.
//
// FP32 data: products and the residual in FP32 (P rounded to FP32), squares
// summed with Kahan compensation in FP32 per thread, then FP64 across threads
// and CTAs.  FP64 data: FP64 throughout.  The cross-CTA sum runs in a fixed
// order, so the result is deterministic.
#include <algorithm>

#include "idsk_internal.h"

namespace idsk {
namespace {

constexpr int TM = 64;
constexpr int TC = 32;
constexpr int NT = 256;

template <typename T>
struct Acc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {   // Kahan-Babuska step
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

template <typename T>
__global__ void __launch_bounds__(NT) recon_kernel(const T* __restrict__ A, int64_t lda,
                                                   int64_t m, int64_t n,
                                                   const int* __restrict__ J,
                                                   const double* __restrict__ P, int k,
                                                   double* __restrict__ part, InterpGeom geo) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* sk = reinterpret_cast<T*>(smem);   // k x TM   : A(R, J)
  T* as = sk + kRecKMax * TM;           // TC x (TM+1)
  T* ps = as + TC * (TM + 1);           // k x TC   : P(:, chunk)
  __shared__ int Js[kRecKMax];
  __shared__ double red[3][NT / 32];

  const int t = threadIdx.x;
  for (int u = t; u < k; u += NT) Js[u] = J[u];
  const int c = t & (TC - 1);
  const int rb = t >> 5;
  Acc<T> res, tot;
  T mx = T(0);
  const int64_t ntiles = (m + TM - 1) / TM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * TM;
    __syncthreads();
    if (geo.Sc == nullptr) {
      for (int e = t; e < k * TM; e += NT) {
        const int u = e / TM, r = e % TM;
        sk[e] = (r0 + r < m) ? A[(r0 + r) + (int64_t)Js[u] * lda] : T(0);
      }
    } else {   // single-pass ID: skeleton rows interpolated from the coarse ones
      const int r = t % TM;
      int64_t idx[8];
      T w[8];
      if (r0 + r < m) interp_corners<T>(r0 + r, geo, idx, w);
      const T* sc = reinterpret_cast<const T*>(geo.Sc);
      for (int u = t / TM; u < k; u += NT / TM) {
        T acc = T(0);
        if (r0 + r < m) {
#pragma unroll
          for (int q = 0; q < 8; ++q) acc += w[q] * sc[idx[q] * kSkelLd + u];
        }
        sk[u * TM + r] = acc;
      }
    }
    for (int64_t cc = 0; cc < n; cc += TC) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < (TC * TM) / NT; ++q) {
        const int e = t + q * NT;
        const int cl = e >> 6, r = e & (TM - 1);
        as[cl * (TM + 1) + r] =
            (r0 + r < m && cc + cl < n) ? A[(r0 + r) + (cc + cl) * lda] : T(0);
      }
      for (int e = t; e < k * TC; e += NT) {
        const int u = e / TC, cl = e % TC;
        ps[e] = (cc + cl < n) ? (T)P[(int64_t)u * n + cc + cl] : T(0);
      }
      __syncthreads();
      if (cc + c < n) {
        T ah[TM / 8];
#pragma unroll
        for (int q = 0; q < TM / 8; ++q) ah[q] = T(0);
        for (int u = 0; u < k; ++u) {
          const T pv = ps[u * TC + c];
#pragma unroll
          for (int q = 0; q < TM / 8; ++q) ah[q] += sk[u * TM + rb + 8 * q] * pv;
        }
#pragma unroll
        for (int q = 0; q < TM / 8; ++q) {
          const int r = rb + 8 * q;
          if (r0 + r < m) {
            const T a = as[c * (TM + 1) + r];
            const T d = a - ah[q];
            res.add(d * d);
            tot.add(a * a);
            const T ad = d < T(0) ? -d : d;
            const T aa = a < T(0) ? -a : a;
            if (a != T(0) && ad > mx * aa) mx = ad / aa;
          }
        }
      }
    }
  }
  // block reduction (fixed order)
  double v0 = (double)res.s - (double)res.c, v1 = (double)tot.s - (double)tot.c, v2 = (double)mx;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    v2 = fmax(v2, __shfl_xor_sync(0xffffffffu, v2, o));
  }
  const int lane = t & 31, warp = t >> 5;
  __syncthreads();
  if (lane == 0) {
    red[0][warp] = v0;
    red[1][warp] = v1;
    red[2][warp] = v2;
  }
  __syncthreads();
  if (t == 0) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      a0 += red[0][w];
      a1 += red[1][w];
      a2 = fmax(a2, red[2][w]);
    }
    part[3 * blockIdx.x + 0] = a0;
    part[3 * blockIdx.x + 1] = a1;
    part[3 * blockIdx.x + 2] = a2;
  }
}

__global__ void recon_finalize_kernel(const double* __restrict__ part, int nblk,
                                      double* __restrict__ out3) {
  if (threadIdx.x != 0) return;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int b = 0; b < nblk; ++b) {
    a0 += part[3 * b];
    a1 += part[3 * b + 1];
    a2 = fmax(a2, part[3 * b + 2]);
  }
  out3[0] = a0;
  out3[1] = a1;
  out3[2] = a2;
}

template <typename T>
size_t recon_smem(void) {
  return sizeof(T) * (kRecKMax * TM + TC * (TM + 1) + kRecKMax * TC);
}

}  // namespace

cudaError_t launch_recon_error(const void* A, int64_t lda, int64_t m, int64_t n, int dtype,
                               const int* J, const double* P, int k, double* part, int nblk,
                               double* out3, int* status, cudaStream_t st, KernelTimer* timer,
                               const InterpGeom* interp) {
  const InterpGeom geo = interp ? *interp : InterpGeom{};
  cudaError_t e;
  if (dtype == ID_F32 && m >= 128) {
    // FP32 data: tensor-core pass (products split into bf16 pieces)
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = std::min(recon_tc_grid(m, n, nsm), nblk);
    if (grid * 1 < (int)((n + 255) / 256)) return cudaErrorInvalidValue;
    e = launch_recon_tc(reinterpret_cast<const float*>(A), lda, m, n, J, P, k, part, grid,
                        status, st, timer, interp);
    if (e != cudaSuccess) return e;
    recon_finalize_kernel<<<1, 32, 0, st>>>(part, grid, out3);
    count_launches(1);
    return cudaGetLastError();
  }
  const int64_t ntiles = (m + TM - 1) / TM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, nblk));
  if (timer && (e = timer->mark(st)) != cudaSuccess) return e;
  if (dtype == ID_F64) {
    const size_t sm = recon_smem<double>();
    e = cudaFuncSetAttribute(recon_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
    recon_kernel<double><<<grid, NT, sm, st>>>(reinterpret_cast<const double*>(A), lda, m, n, J,
                                               P, k, part, geo);
  } else {
    const size_t sm = recon_smem<float>();
    e = cudaFuncSetAttribute(recon_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
    if (e != cudaSuccess) return e;
    recon_kernel<float><<<grid, NT, sm, st>>>(reinterpret_cast<const float*>(A), lda, m, n, J, P,
                                              k, part, geo);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (timer && (e = timer->mark(st)) != cudaSuccess) return e;
  recon_finalize_kernel<<<1, 32, 0, st>>>(part, grid, out3);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace idsk
