// Single-pass ID (Algorithm 6, Sec. 2.6, eq. eqn:single_ID), column
// orientation: A ~ M A_c(:, J_c) P_c.  The fine skeleton is not read from A a
// second time; the coarse skeleton A_c(:, J_c) is interpolated back to the
// fine grid by the coarse-to-fine operator M (Algorithm 6 step 4).
//
// M is trilinear interpolation on the mesh (t = 8 coarse points per fine
// point), applied as a tensor product of one-dimensional rules:
//   * coarse points are every s-th index from 0 in each direction (the direct
//     injection of Sec. 2.5);
//   * between two coarse points the weight of the upper one is the fraction
//     of the physical distance, (x_i - x_lo) / (x_hi - x_lo);
//   * past the last coarse point a periodic direction wraps to coarse point 0
//     at x_0 + period, a non-periodic one extrapolates linearly from its last
//     two coarse points.
// M is never stored: each fine row finds its 8 corners from three small
// per-direction tables (interp_corners).
#include <cmath>

#include "idsk_internal.h"

namespace idsk {

void build_axis_weights(const double* x, int n, int stride, double period, AxisW* out) {
  const int c = (n + stride - 1) / stride;
  for (int i = 0; i < n; ++i) {
    const int a = i / stride;
    AxisW e{a, a, 0.0};
    if (i % stride != 0) {
      if (a + 1 < c) {
        e.hi = a + 1;
        e.w = (x[i] - x[a * stride]) / (x[(a + 1) * stride] - x[a * stride]);
      } else if (period > 0.0) {
        e.hi = 0;
        e.w = (x[i] - x[a * stride]) / (x[0] + period - x[a * stride]);
      } else if (c >= 2) {
        e.lo = c - 2;
        e.hi = c - 1;
        e.w = (x[i] - x[(c - 2) * stride]) / (x[(c - 1) * stride] - x[(c - 2) * stride]);
      } else {
        e.lo = e.hi = 0;
      }
    }
    out[i] = e;
  }
}

namespace {

// Sc(i, u) = A_c(i, J_c[u]) for u < k, 0 for k <= u < kSkelLd (row-major).
template <typename T>
__global__ void skeleton_compact_kernel(const T* __restrict__ Ac, int64_t mc,
                                        const int* __restrict__ Jc, int k, T* __restrict__ Sc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mc * kSkelLd) return;
  const int64_t i = e / kSkelLd;
  const int u = (int)(e - i * kSkelLd);
  Sc[e] = u < k ? Ac[i + (int64_t)Jc[u] * mc] : T(0);
}

// S(r, u) = sum over the 8 corners of w * Sc(corner, u), column-major m x k.
// FP32 data interpolates in FP32 (weights rounded), FP64 data in FP64.
template <typename T>
__global__ void lift_kernel(InterpGeom g, int64_t m, int k, T* __restrict__ S) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  int64_t idx[8];
  T w[8];
  interp_corners<T>(r, g, idx, w);
  const T* Sc = reinterpret_cast<const T*>(g.Sc);
  for (int u = 0; u < k; ++u) {
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += w[q] * Sc[idx[q] * kSkelLd + u];
    S[r + (int64_t)u * m] = acc;
  }
}

}  // namespace

cudaError_t launch_skeleton_compact(const void* Ac, int64_t mc, int dtype, const int* Jc, int k,
                                    void* Sc, cudaStream_t st) {
  const int64_t tot = mc * kSkelLd;
  const int blocks = (int)((tot + 255) / 256);
  if (dtype == ID_F64)
    skeleton_compact_kernel<double><<<blocks, 256, 0, st>>>(
        reinterpret_cast<const double*>(Ac), mc, Jc, k, reinterpret_cast<double*>(Sc));
  else
    skeleton_compact_kernel<float><<<blocks, 256, 0, st>>>(
        reinterpret_cast<const float*>(Ac), mc, Jc, k, reinterpret_cast<float*>(Sc));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_single_pass_lift(const InterpGeom& g, int64_t m, int dtype, int k, void* S,
                                    cudaStream_t st) {
  const int blocks = (int)((m + 255) / 256);
  if (dtype == ID_F64)
    lift_kernel<double><<<blocks, 256, 0, st>>>(g, m, k, reinterpret_cast<double*>(S));
  else
    lift_kernel<float><<<blocks, 256, 0, st>>>(g, m, k, reinterpret_cast<float*>(S));
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace idsk
