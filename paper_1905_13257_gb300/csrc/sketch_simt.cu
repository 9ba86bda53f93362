// Fused single-read sketch, CUDA-core (SIMT) form, and the Gaussian fill.
//
// One read of each tile of A forms both randomized sketches of the streamed
// columns (Algorithm 4 step 3, transposed orientation, and eq. eq:sampmatrix):
//   W(:, cols) = Psi A(:, cols)        (l x ncols, FP64 accumulation)
//   Y         += A(:, cols) Omega(cols, :)   (m x l)
// and, when asked, gathers the coarse-grid rows A_c = A(rows_c, cols) of
// Algorithm 5 step 3 from the same tile.  Psi is never stored: each CTA draws
// Psi(:, R) for its row tile R from the counter generator.
//
// This form serves FP64 data and any shape; the tensor-core form in
// sketch_tc.cu serves FP32 data at HBM speed.
#include <cuda_bf16.h>

#include <algorithm>

#include "idsk_internal.h"

namespace idsk {
namespace {

constexpr int TM = 64;    // rows per tile
constexpr int TC = 32;    // columns per chunk
constexpr int NT = 256;   // threads per CTA

__global__ void gaussian_fill_kernel(uint32_t which, uint32_t k0, uint32_t k1, int64_t first,
                                     int64_t count, int width, const float* __restrict__ table,
                                     float* __restrict__ out) {
  const int nblk = (width + 9) / 10;
  const int64_t total = count * nblk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nblk;
    const int sb = (int)(e % nblk);
    float g[10];
    gauss10((uint64_t)(first + i), (uint32_t)sb, which, k0, k1, table, g);
#pragma unroll
    for (int f = 0; f < 10; ++f) {
      const int s = sb * 10 + f;
      if (s < width) out[i * width + s] = g[f];
    }
  }
}

__device__ __forceinline__ float to_bf16_rn(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

template <typename T>
__device__ __forceinline__ T maybe_bf16(T v, int on) {
  return v;
}
template <>
__device__ __forceinline__ float maybe_bf16<float>(float v, int on) {
  return on ? to_bf16_rn(v) : v;
}

__device__ __forceinline__ int64_t coarse_index(int64_t r, const CoarseGeom& g) {
  const int64_t i = r % g.nx;
  const int64_t rest = r / g.nx;
  const int64_t z = rest % g.nz;
  const int64_t rest2 = rest / g.nz;
  const int64_t j = rest2 % g.ny;
  const int64_t c = rest2 / g.ny;
  if (i % g.sx || j % g.sy || z % g.sz) return -1;
  return ((c * g.cy + j / g.sy) * g.cz + z / g.sz) * g.cx + i / g.sx;
}

// Shared layout (bytes): table 16384 | psi 64xTM f32 | omega TCx64 f32 |
// A tile TC x (TM+1) T | rc TM i64 | colptr TC | wacc 64 x ncols f64
template <typename T>
__global__ void __launch_bounds__(NT, 1) sketch_simt_kernel(SketchArgs a, Window w) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* tab = reinterpret_cast<float*>(smem);
  float* psi_s = tab + kTableSize;
  float* om_s = psi_s + kLMax * TM;
  T* a_s = reinterpret_cast<T*>(om_s + TC * kLMax);
  int64_t* rc_s = reinterpret_cast<int64_t*>(a_s + TC * (TM + 1) + (sizeof(T) == 4 ? TC : 0));
  const T** cptr_s = reinterpret_cast<const T**>(rc_s + TM);
  double* wacc = reinterpret_cast<double*>(cptr_s + TC);

  const int t = threadIdx.x;
  const int ncols = w.ncols;
  const int lpad = a.lpad;
  const int l = a.l;

  for (int e = t; e < kTableSize; e += NT) tab[e] = a.table[e];
  for (int e = t; e < kLMax * ncols; e += NT) wacc[e] = 0.0;

  const int64_t ntiles = (a.m + TM - 1) / TM;
  const int yrow = t & (TM - 1);
  const int yg = t >> 6;               // 4 groups of 16 sketch columns
  const int wc = t & (TC - 1);         // W: column inside the chunk
  const int ws = t >> 5;               // W: first sketch row (stride 8)

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * TM;
    __syncthreads();   // previous tile fully consumed
    // Psi(:, R) from the counter generator
    {
      const int64_t i = r0 + yrow;
      for (int sb = yg; sb * 10 < lpad; sb += 4) {
        float g[10];
        if (i < a.m) {
          gauss10((uint64_t)i, (uint32_t)sb, kStreamPsi, a.k0, a.k1, tab, g);
        } else {
#pragma unroll
          for (int f = 0; f < 10; ++f) g[f] = 0.f;
        }
#pragma unroll
        for (int f = 0; f < 10; ++f) {
          const int s = sb * 10 + f;
          if (s < lpad) psi_s[s * TM + yrow] = (s < l) ? g[f] : 0.f;
        }
      }
      if (t < TM) rc_s[t] = (a.cg.on && r0 + t < a.m) ? coarse_index(r0 + t, a.cg) : -1;
    }
    T yacc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) yacc[q] = T(0);

    for (int cc = 0; cc < ncols; cc += TC) {
      __syncthreads();
      if (t < TC) {
        const int c = cc + t;
        const T* p = nullptr;
        if (c < ncols) {
          for (int s = 0; s < w.nseg; ++s) {
            const Seg& sg = w.seg[s];
            if (c >= sg.col0 && c < sg.col0 + sg.ncols) {
              p = reinterpret_cast<const T*>(sg.ptr) + (int64_t)(c - sg.col0) * sg.ld;
              break;
            }
          }
        }
        cptr_s[t] = p;
      }
      for (int e = t; e < TC * kLMax; e += NT) {
        const int c = e / kLMax, s = e % kLMax;
        om_s[e] = (cc + c < ncols && s < l) ? a.omega[(w.col_base + cc + c) * l + s] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < (TC * TM) / NT; ++q) {
        const int e = t + q * NT;
        const int c = e >> 6, r = e & (TM - 1);
        const T* p = cptr_s[c];
        T v = T(0);
        if (p != nullptr && r0 + r < a.m) {
          v = p[r0 + r];
          const int64_t rc = rc_s[r];
          if (rc >= 0) reinterpret_cast<T*>(a.Ac)[rc + a.cg.mc * (w.col_base + cc + c)] = v;
          v = maybe_bf16(v, a.bf16);
        }
        a_s[c * (TM + 1) + r] = v;
      }
      __syncthreads();
      // Y(R, :) += A(R, chunk) Omega(chunk, :)
      if (a.want_Y) {
#pragma unroll 4
        for (int c = 0; c < TC; ++c) {
          const T av = a_s[c * (TM + 1) + yrow];
#pragma unroll
          for (int q = 0; q < 16; ++q) yacc[q] += av * (T)om_s[c * kLMax + yg * 16 + q];
        }
      }
      // W(:, chunk) += Psi(:, R) A(R, chunk)
      if (cc + wc < ncols) {
#pragma unroll
        for (int q = 0; q < kLMax / 8; ++q) {
          const int s = ws + 8 * q;
          if (s < l) {
            T acc = T(0);
#pragma unroll 8
            for (int r = 0; r < TM; ++r) acc += (T)psi_s[s * TM + r] * a_s[wc * (TM + 1) + r];
            wacc[s * ncols + cc + wc] += (double)acc;
          }
        }
      }
    }
    if (a.want_Y) {
      const int64_t i = r0 + yrow;
      if (i < a.m) {
        T* Y = reinterpret_cast<T*>(a.Y);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int s = yg * 16 + q;
          if (s < l) {
            const int64_t o = i + s * a.m;
            Y[o] = a.y_accumulate ? Y[o] + yacc[q] : yacc[q];
          }
        }
      }
    }
  }
  __syncthreads();
  for (int e = t; e < l * ncols; e += NT) {
    const int s = e / ncols, c = e % ncols;
    atomicAdd(&a.W[s * a.ldw + w.col_base + c], wacc[s * ncols + c]);
  }
}

template <typename T>
size_t simt_smem_bytes(int ncols) {
  return sizeof(float) * (kTableSize + kLMax * TM + TC * kLMax) +
         sizeof(T) * (TC * (TM + 1) + (sizeof(T) == 4 ? TC : 0)) + sizeof(int64_t) * TM +
         sizeof(void*) * TC + sizeof(double) * kLMax * (size_t)ncols;
}

}  // namespace

cudaError_t launch_gaussian_fill(uint32_t which, uint32_t k0, uint32_t k1, int64_t first,
                                 int64_t count, int width, const float* table, float* out,
                                 cudaStream_t st) {
  if (count <= 0 || width <= 0) return cudaSuccess;
  const int64_t total = count * ((width + 9) / 10);
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  gaussian_fill_kernel<<<blocks, 256, 0, st>>>(which, k0, k1, first, count, width, table, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sketch_simt(const SketchArgs& a, const Window& w, int dtype, int nsm,
                               cudaStream_t st) {
  if (w.ncols <= 0) return cudaSuccess;
  const int64_t ntiles = (a.m + TM - 1) / TM;
  const int grid = (int)std::min<int64_t>(ntiles, nsm);
  if (dtype == ID_F64) {
    const size_t sm = simt_smem_bytes<double>(w.ncols);
    cudaError_t e = cudaFuncSetAttribute(sketch_simt_kernel<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    sketch_simt_kernel<double><<<grid, NT, sm, st>>>(a, w);
  } else {
    const size_t sm = simt_smem_bytes<float>(w.ncols);
    cudaError_t e = cudaFuncSetAttribute(sketch_simt_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    sketch_simt_kernel<float><<<grid, NT, sm, st>>>(a, w);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace idsk
