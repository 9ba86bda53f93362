// Internal declarations of the idsketch library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "idsketch.h"

namespace idsk {

// ------------------------------------------------------------------ limits
constexpr int kLMax = 64;             // sketch width l (padded to 16 on device)
// Wider sketches, l <= kLMaxW (so k <= 86 at l = k + 10): FP32 data on the
// tensor-core sketch without Y, in passes of at most kPassRows rows of Psi
// (one more read of each window per pass); the one-CTA pivoted QR and the
// solve take up to kLMaxW rows and pivots.  Everything else keeps k, l <= 64.
constexpr int kLMaxW = 96;
constexpr int kPassRows = 60;         // a multiple of 10: Psi's counter blocks
constexpr int kMaxSegs = 64;          // column segments per sketch launch
constexpr int kSimtWindowMax = 320;   // columns per SIMT sketch launch
constexpr int kTcMaxTiles = 4;        // 128-column tiles per tensor-core launch (TMEM budget)
constexpr int kRecKMax = 64;          // rank handled by the error pass
constexpr int kTableSize = 4096;

// -------------------------------------------------- counter-based Gaussian
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies with the round multipliers below; the key advances by the Weyl
// increments after every round.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kStreamPsi = 1;
constexpr uint32_t kStreamOmega = 2;

#ifdef __CUDACC__
__host__ __device__ __forceinline__ void philox10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                                  uint32_t& c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
}

// Field f (bits 12f .. 12f+11) of the 128-bit block c0 | c1<<32 | c2<<64 | c3<<96.
__host__ __device__ __forceinline__ uint32_t field12(uint32_t c0, uint32_t c1, uint32_t c2,
                                                     uint32_t c3, int f) {
  const uint64_t lo = (uint64_t)c0 | ((uint64_t)c1 << 32);
  const uint64_t hi = (uint64_t)c2 | ((uint64_t)c3 << 32);
  const int b = 12 * f;
  if (b + 12 <= 64) return (uint32_t)(lo >> b) & 0xFFFu;
  if (b < 64) return (uint32_t)((lo >> b) | (hi << (64 - b))) & 0xFFFu;
  return (uint32_t)(hi >> (b - 64)) & 0xFFFu;
}

// Ten consecutive entries G(index, 10*sb .. 10*sb+9) of stream `which`.
__device__ __forceinline__ void gauss10(uint64_t index, uint32_t sb, uint32_t which, uint32_t k0,
                                        uint32_t k1, const float* __restrict__ tab,
                                        float out[10]) {
  uint32_t c0 = (uint32_t)index, c1 = (uint32_t)(index >> 32), c2 = sb, c3 = which;
  philox10(c0, c1, c2, c3, k0, k1);
#pragma unroll
  for (int f = 0; f < 10; ++f) out[f] = tab[field12(c0, c1, c2, c3, f)];
}
#endif

// ------------------------------------------------------------- launch args
struct Seg {
  const void* ptr;   // first element of the segment's first column
  int64_t ld;        // leading dimension (elements)
  int32_t col0;      // first column of the segment inside the window
  int32_t ncols;
};

struct Window {
  int32_t nseg;
  int32_t ncols;      // columns in the window
  int64_t col_base;   // global index of the window's first column
  Seg seg[kMaxSegs];
};

struct CoarseGeom {
  int32_t on;
  int32_t nx, ny, nz, sx, sy, sz, cx, cy, cz;   // c* = coarse points per direction
  int64_t mc;
};

struct SketchArgs {
  int64_t m;
  int32_t l, lpad;
  uint32_t k0, k1;
  const float* table;   // 4096 quantiles (FP32, bf16-exact)
  const float* omega;   // n_max x l, row-major
  double* W;            // l x ldw, row-major (accumulated with atomics)
  int64_t ldw;
  void* Y;              // m x l, column-major, dtype
  int32_t want_Y, y_accumulate;
  void* Ac;             // mc x n_max, column-major, dtype
  CoarseGeom cg;
  int32_t bf16;         // round A to bfloat16 before the products
  float* wpart;         // tensor-core kernel: per-CTA FP32 W^T slabs [nsm][512][w_width]
  const int64_t* crow;  // tensor-core path: fine row of each coarse row (the A_c copy)
  const float* colscale;   // FP8 form: 2^e_c of each column of the window (window column 0 first)
  int32_t fp8;             // FP8-E4M3 form (tensor-core path, one bfloat16 piece)
  int32_t s0;           // first row of Psi drawn by this launch (a multiple of 10)
};

// Width of the tensor-core sketch's W^T accumulators and partial slabs: 64
// columns, or 96 when Y is not formed and l > 64 (the whole sketch in one
// pass over A).
__host__ __device__ constexpr inline int w_width(int l, bool want_Y) {
  return (!want_Y && l > kLMax) ? kLMaxW : kLMax;
}

// ------------------------------------------- batched form (work list)
// The sketch of one matrix of a batch: all a.l <= 96 rows of Psi in one
// pass, no Y and no coarse gather.  Its W goes to Wd (row-major, a.l x
// ncols, leading dimension ncols).
struct BatchJob {
  SketchArgs a;
  int32_t ncols;          // n of the matrix (<= 512)
  int32_t np;             // bfloat16 pieces of A: 2 (FP32-accurate) or 1 (BF16 form)
  int32_t prob;           // problem index (its status flag)
  int32_t item0, nitem;   // its work items, contiguous in the item table
  int32_t pad;
  double* Wd;
};
// A work item: row blocks rb0 .. rb0 + nrb - 1 of one job, its W^T partials
// into the FP32 slab at float offset `slab` ([ceil(ncols / 128) * 128][lw],
// lw = w_width(l, false)).
struct BatchItem {
  int64_t rb0;
  int64_t slab;
  int32_t nrb, job;
};
// Pivoted QR of one batched W (l x n row-major, leading dimension n) and the
// solve for P, written straight into the batch's packed outputs.
struct QrJob {
  double* M;
  double* R;
  int32_t* J;
  int32_t* colpos;
  int32_t* kout;
  double* P;
  int32_t rows, n, k, pad;
};

// ------------------------------------------------ single-pass ID (Alg. 6)
// Coarse-to-fine interpolation of one direction at fine index i: the value is
// (1 - w) f[lo] + w f[hi] with lo, hi coarse indices (a fine index on a coarse
// point has lo = hi, w = 0; a periodic direction wraps past its last coarse
// point; a non-periodic one extrapolates from its last two coarse points).
struct AxisW {
  int32_t lo, hi;
  double w;
};

// Trilinear interpolation of the coarse skeleton Sc = A_c(:, J_c) (m_c rows of
// kSkelLd entries, row-major, data type) to fine row r.
constexpr int kSkelLd = 64;
struct InterpGeom {
  const AxisW* ax = nullptr;   // nx entries
  const AxisW* ay = nullptr;   // ny entries
  const AxisW* az = nullptr;   // nz entries
  const void* Sc = nullptr;    // null: no interpolation (gather A(:, J) instead)
  int32_t nx = 0, ny = 0, nz = 0, cx = 0, cy = 0, cz = 0;
};

// The 8 corners of fine row r = ((c ny + j) nz + kz) nx + i: coarse rows
// ((c cy + jy) cz + kc) cx + ic and their trilinear weights, formed in the
// arithmetic of W (the data type of the interpolation).
template <typename W>
__host__ __device__ inline void interp_corners(int64_t r, const InterpGeom& g, int64_t (&idx)[8],
                                               W (&w)[8]) {
  const int64_t i = r % g.nx;
  int64_t rest = r / g.nx;
  const int64_t kz = rest % g.nz;
  rest /= g.nz;
  const int64_t j = rest % g.ny;
  const int64_t c = rest / g.ny;
  const AxisW X = g.ax[i], Y = g.ay[j], Z = g.az[kz];
  int q = 0;
  for (int b = 0; b < 2; ++b) {
    const int64_t iy = b ? Y.hi : Y.lo;
    const W fy = b ? (W)Y.w : (W)1 - (W)Y.w;
    for (int d = 0; d < 2; ++d) {
      const int64_t iz = d ? Z.hi : Z.lo;
      const W fz = d ? (W)Z.w : (W)1 - (W)Z.w;
      for (int a = 0; a < 2; ++a) {
        const int64_t ix = a ? X.hi : X.lo;
        const W fx = a ? (W)X.w : (W)1 - (W)X.w;
        idx[q] = ((c * g.cy + iy) * g.cz + iz) * g.cx + ix;
        w[q] = fx * fy * fz;
        ++q;
      }
    }
  }
}

// CUDA events recorded around the main kernel of a launcher, on the launching
// stream (optional measurement; the launchers take a null pointer when off).
struct KernelTimer {
  std::vector<cudaEvent_t> ev;   // start, stop, start, stop, ...
  size_t used = 0;               // events recorded since the last read
  cudaError_t mark(cudaStream_t st) {
    if (used == ev.size()) {
      cudaEvent_t e;
      const cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      ev.push_back(e);
    }
    return cudaEventRecord(ev[used++], st);
  }
  // Sum of the recorded (stop - start) intervals in ms; waits for the last
  // event and starts a new accumulation.
  cudaError_t read(double* ms, int64_t* pairs) {
    double tot = 0.0;
    const size_t np = used / 2;
    if (np > 0) {
      cudaError_t r = cudaEventSynchronize(ev[2 * np - 1]);
      if (r != cudaSuccess) return r;
      for (size_t q = 0; q < np; ++q) {
        float t = 0.f;
        r = cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]);
        if (r != cudaSuccess) return r;
        tot += t;
      }
    }
    used = 0;
    *ms = tot;
    *pairs = (int64_t)np;
    return cudaSuccess;
  }
  ~KernelTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

}  // namespace idsk

// ------------------------------------------------------------------ handle
struct id_sketch {
  id_config cfg;
  cudaStream_t st = nullptr;
  int dev = 0, nsm = 0;
  int64_t m = 0, n_max = 0, mc = 0;
  int k = 0, l = 0, lpad = 0;
  size_t esz = 4;
  uint32_t key0 = 0, key1 = 0;
  idsk::CoarseGeom cg{};

  float* d_table = nullptr;
  float* d_omega = nullptr;
  double* d_W = nullptr;
  void* d_Y = nullptr;
  void* d_Ac = nullptr;
  int64_t* d_crow = nullptr;   // fine row of each coarse-grid row (FP32, want_coarse)
  float* d_colscale = nullptr;  // FP8 form: per-column power-of-two scales (n_max)

  std::vector<idsk::Seg> pend;   // borrowed chunks, window-relative col0
  int64_t pend_cols = 0;
  int64_t n_seen = 0;            // columns accepted (launched + pending)
  int64_t n_launched = 0;
  bool y_started = false;
  bool poisoned = false;
  int sketch_kernel = 0;         // 0 auto, 1 tensor cores, 2 SIMT (IDSKETCH_SKETCH)
  int drain_blocks = 8;          // row blocks between FP64 flushes of W^T (tensor cores)
  int grid_cap = 0;              // CTAs of a sketch launch at most (0: one per SM)
  int* d_status = nullptr;       // nonzero: a bounded device wait gave up
  float* d_wpart = nullptr;      // per-CTA W^T slabs of the tensor-core sketch

  // factor workspace
  double* d_work = nullptr;   // l x n_max copy of W
  double* d_R = nullptr;      // max(k) x n_max
  double* d_P = nullptr;      // k x n_max
  int* d_J = nullptr;         // k
  int* d_colpos = nullptr;    // n_max
  int* d_kout = nullptr;      // 1
  int* d_cand = nullptr;      // n_max: candidate columns (id_factor_restricted)
  double* d_fq = nullptr;     // l k + k + k k: reflectors, tau, R of W(:, J)
  // coarse workspace (allocated with the handle when want_coarse)
  double* d_V = nullptr;      // mc x k: reflectors as FP32 pairs (8 bytes each)
  double* d_F = nullptr;      // n_max x k
  double* d_nu2 = nullptr;    // n_max
  double* d_nu20 = nullptr;   // n_max
  double* d_gvec = nullptr;   // coarse_blocks x n_max: row-range partials of A_c^T u
  double* d_hvec = nullptr;   // kLMax: V_s^T v_s
  float* d_vh = nullptr;      // mc: u below row s as an FP32 pair (hi)
  float* d_vl = nullptr;      // mc: (lo)
  double* d_upart = nullptr;  // coarse_blocks x (kLMax + 1): partials of V_s^T u, ||u||^2
  double* d_cscal = nullptr;  // 8 scalars
  int* d_cint = nullptr;      // 8 ints: pivot, stop, nrecompute, k_out, 2 CTA counters
  int* d_rlist = nullptr;     // n_max
  double* d_Rc = nullptr;     // k x n_max
  double* d_Pc = nullptr;     // k x n_max
  int* d_Jc = nullptr;        // k
  int* d_colposc = nullptr;   // n_max
  int coarse_blocks = 0;
  // The coarse QR of the same columns started by id_factor on a side stream
  // (want_coarse, FP32, cooperative form): it runs beside the small QR of W
  // and id_coarse_factor only waits for it.
  cudaStream_t st2 = nullptr;     // side stream (created with the handle)
  cudaEvent_t ev_sk = nullptr;    // the sketch of the columns is complete
  cudaEvent_t ev_cq = nullptr;    // the side stream's coarse QR is complete
  int64_t coarse_spec = -1;       // n_seen of the started coarse QR (-1: none)
  bool cq_pending = false;        // side-stream work not yet ordered before h->st
  // error-pass workspace
  double* d_part = nullptr;   // rec_blocks x 3
  double* d_out3 = nullptr;   // 3
  int* d_Jin = nullptr;       // kRecKMax
  double* d_Pin = nullptr;    // kRecKMax x pin_cap
  int64_t pin_cap = 0;
  int rec_blocks = 0;
  // id_timing_enable: events around the fused sketch kernel and the error-pass
  // kernel
  idsk::KernelTimer* timer_sketch = nullptr;
  idsk::KernelTimer* timer_recon = nullptr;
  // id_set_mesh: per-direction interpolation tables and the compact coarse
  // skeleton of the single-pass ID
  idsk::AxisW* d_axis = nullptr;   // nx + ny + nz entries
  void* d_Sc = nullptr;            // m_c x kSkelLd, dtype
  bool mesh_set = false;
};

// ------------------------------------------------------------- launchers
namespace idsk {
// The coarse rows of the tensor-core path (sketch_tc.cu): crow[coarse index]
// = fine row, once per handle; A_c(:, window) = A(crow, window) after each
// window's sketch.
cudaError_t launch_coarse_rows(const CoarseGeom& g, int64_t m, int64_t* crow, cudaStream_t st);
cudaError_t launch_coarse_gather(const Window& w, const int64_t* crow, int64_t mc, float* Ac,
                                 cudaStream_t st);
// FP8 form (sketch_tc.cu): the power-of-two scale of each column of the
// window into scale[0 .. w.ncols - 1] (one read of the window).
cudaError_t launch_fp8_scales(const Window& w, int64_t m, float* scale, cudaStream_t st);
cudaError_t launch_gaussian_fill(uint32_t which, uint32_t k0, uint32_t k1, int64_t first,
                                 int64_t count, int width, const float* table, float* out,
                                 cudaStream_t st);
cudaError_t launch_sketch_simt(const SketchArgs& a, const Window& w, int dtype, int nsm,
                               cudaStream_t st);
cudaError_t launch_sketch_tc(const SketchArgs& a, const Window& w, int npieces, int nsm,
                             int drain_blocks, int* status, cudaStream_t st,
                             KernelTimer* timer = nullptr);
// Batched form (sketch_tc.cu): the whole work list in one persistent launch
// (grid CTAs; items taken in `order`; counters[0] the item counter and
// counters[1 + j] job j's completed items, all zeroed by the caller); the CTA
// that completes a job's last item sums its slabs into W and runs its QR and
// solve (qjobs[j]).
size_t sketch_batch_smem_bytes();
cudaError_t launch_sketch_batch(const BatchJob* jobs, const CUtensorMap* tmaps,
                                const BatchItem* items, const int32_t* order, int nitems,
                                float* slabs, int* counters, const QrJob* qjobs,
                                double tol_factor, int* stat, int grid, int drain_blocks,
                                cudaStream_t st);
cudaError_t launch_cpqr_small(double* M, int rows, int n, int ld, int k, double tol_factor,
                              double* R, int* J, int* colpos, int* kout, cudaStream_t st,
                              bool one_cta = false);
cudaError_t launch_solve_p(const double* R, const int* J, const int* colpos, const int* kout,
                           int k, int n, double* P, cudaStream_t st);
cudaError_t launch_coarse_cpqr(id_sketch* h, int64_t n, cudaStream_t st);
// The coarse QR as one cooperative launch (coarse_coop.cu): FP32 A_c, m_c a
// multiple of 4, at most 512 rows per CTA.
bool coarse_coop_ok(const id_sketch* h);
cudaError_t launch_coarse_coop(id_sketch* h, int64_t n, cudaStream_t st, int max_ctas = 0);
bool coarse_coop_ok_ctas(const id_sketch* h, int max_ctas);
cudaError_t run_wait_check(int mode, cudaStream_t st, int* gave_up);
cudaError_t launch_recon_error(const void* A, int64_t lda, int64_t m, int64_t n, int dtype,
                               const int* J, const double* P, int k, double* part, int nblk,
                               double* out3, int* status, cudaStream_t st,
                               KernelTimer* timer = nullptr, const InterpGeom* interp = nullptr);
int recon_tc_grid(int64_t m, int64_t n, int nsm);
cudaError_t launch_recon_tc(const float* A, int64_t lda, int64_t m, int64_t n, const int* J,
                            const double* P, int k, double* part, int grid, int* status,
                            cudaStream_t st, KernelTimer* timer = nullptr,
                            const InterpGeom* interp = nullptr);
void build_axis_weights(const double* x, int n, int stride, double period, AxisW* out);
// Tensor map of an FP32 column-major matrix (rows contiguous, leading
// dimension ld), boxes of box_rows x box_cols, zero fill outside; false when
// it cannot be built (alignment, no driver entry point).
bool make_tmap_f32_2d(const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                      int box_cols, CUtensorMap* tm);
cudaError_t launch_skeleton_compact(const void* Ac, int64_t mc, int dtype, const int* Jc, int k,
                                    void* Sc, cudaStream_t st);
cudaError_t launch_single_pass_lift(const InterpGeom& g, int64_t m, int dtype, int k, void* S,
                                    cudaStream_t st);
void gaussian_table_host(float* vals, uint16_t* bits);
void count_launches(int64_t n);
cudaError_t launch_gather_cols(const double* W, int64_t ldw, int l, const int* cand, int ncand,
                               double* Wc, cudaStream_t st);
cudaError_t launch_map_pivots(const int* Jc, const int* cand, const int* kout, int k, int* J,
                              cudaStream_t st);
cudaError_t launch_fixed_solve(const double* W, int64_t ldw, int l, int n, const int* J,
                               const int* kout, int k, double* fq, double* P, cudaStream_t st);
// Launch the sketch of every pending column window of the handle (capi.cu).
id_status launch_pending(id_sketch* h);
// Enqueue the randomized ID of the streamed columns (pivoted QR of W and the
// solve for P) into h->d_J, h->d_P, h->d_kout, with no host synchronisation
// (capi.cu).  ID_ERR_STATE when no column was streamed.
id_status factor_enqueue(id_sketch* h, bool one_cta = false);
}  // namespace idsk
