// Fused single-read sketch on the tcgen05 tensor cores (FP32 data).
//
// One read of each 128 x 128 tile of A forms both randomized sketches of the
// window's columns (Algorithm 4 step 3, transposed orientation; eq.
// eq:sampmatrix):
//   W^T(c, :) += A(R, c)^T Psi(:, R)^T   (128 columns x 64, TMEM accumulator)
//   Y(R, :)   += A(R, C) Omega(C, :)     (128 rows x 64, TMEM accumulator)
// The coarse-grid rows of Algorithm 5 step 3 are copied to A_c by a small
// kernel right after each window's sketch (coarse_gather_kernel): it reads
// only the row blocks that hold coarse rows (1/16 of A on a grid with
// stride 4 in y and z).  Copied inside this kernel they cost far more: by
// the converters 0.45 ms per 512-column window of 4.7M rows (their loop on
// the critical path), by a dedicated warp 2.1 ms (the raw ring waits for
// it), against 2.1 ms for the whole window without them.
//
// Precision.  A (FP32) is split once per tile into NP bfloat16 pieces,
// A = a0 + a1 (+ rounding below 2^-16 |A|); Psi and Omega are exact in
// bfloat16 (quantile table), so every tensor-core product is exact and the
// sketches carry only the split error (about 2.4e-6 relative in Frobenius
// norm for NP = 2) and the FP32 accumulation.  NP = 1 is the bfloat16
// precision form.  The tensor cores' FP32 accumulator error grows with the
// length of the sum, so W^T partials leave TMEM every few row blocks; they
// are added (round to nearest) into a per-CTA FP32 slab, about 30 partials
// per entry, and the slabs are summed in FP32 pairs (about 48 bits).
//
// Shared-memory layout.  A piece tile is stored in 128-byte-swizzled 1 KB
// atoms of 8 columns x 64 rows (rows contiguous).  Read as K-major it is the
// A operand of the W^T product (M = columns, K = rows); read as MN-major it is
// the A operand of the Y product (M = rows, K = columns): one copy serves both
// products.  Psi(:, R)^T and Omega(C, :)^T are K-major B operands.
//
// Warp roles (one CTA per SM, persistent over a contiguous range of row
// blocks):
//   warps 0-7    converters: load A with 128-bit coalesced loads in half
//                tiles (two register buffers: one half tile in flight),
//                split into pieces, store them to the swizzled piece buffer
//                (double-buffered)
//   warps 8-11   epilogue: draw Psi for upcoming row blocks (counter
//                generator), drain Y to global memory, flush W^T partials
//                into a per-CTA FP32 slab in L2 (one 128-column tile at a
//                time, staggered over the row blocks: a tile's accumulator
//                is handed back to the MMAs as soon as it is in registers,
//                before its reductions)
//   warp 12      TMEM allocation and the single-thread tcgen05.mma issue
//   warp 13      (TMA form: a single-segment window with 16-byte aligned
//                columns) streams raw FP32 boxes of 128 rows x 32 columns
//                through an NST-stage shared-memory ring; the converters
//                then read A from the ring and fill two single-piece slots
//                in turn, so that the MMAs of one piece overlap the
//                conversion of the other
// At most 4 warps per SM sub-partition, so a thread may hold up to 128
// registers.
// Every mbarrier wait is bounded: on timeout the CTA raises an abort flag,
// every role leaves its loop, in-flight MMAs are waited for (bounded) and the
// TMEM is freed; the host reads the status word and reports ID_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "cta_qr.cuh"
#include "df.cuh"
#include "idsk_internal.h"
#include "tc_common.cuh"

namespace idsk {
namespace {

using namespace tc;

constexpr int TR = 128;                 // rows per tile
constexpr int TCOLS = 128;              // columns per tile
constexpr int NCONV = 8;                // converter warps
constexpr int NEPI = 4;                 // epilogue warps
constexpr int MMA_WARP = NCONV + NEPI;  // 12
constexpr int NTHREADS = (NCONV + NEPI + 1) * 32;
constexpr int PROD_WARP = MMA_WARP + 1;   // TMA producer (TMA form only)
constexpr int NTHREADS_TMA = NTHREADS + 32;
constexpr int NST = 4;                    // raw FP32 stages of 128 rows x 32 columns
constexpr uint32_t RAW_BYTES = TR * 32 * 4;   // 16 KB
constexpr int LP = 64;                  // padded sketch width: N of both products
constexpr uint32_t PIECE_BYTES = TR * TCOLS * 2;     // 32 KB
constexpr uint32_t PSI_BYTES = LP * TR * 2;          // 16 KB
constexpr uint32_t OMEGA_TILE_BYTES = LP * TCOLS * 2;  // 16 KB
constexpr int TMEM_COLS = 512;
constexpr uint32_t IDESC_W = tc::idesc_bf16(128, LP, 0);   // A^T K-major (K = rows)
constexpr uint32_t IDESC_W96 = tc::idesc_bf16(128, 96, 0);  // the same, 96 sketch rows
constexpr uint32_t IDESC_Y = tc::idesc_bf16(128, LP, 1);   // A MN-major (M = rows)
constexpr int TMEM_Y = kTcMaxTiles * LP;             // Y accumulators after W^T

// Optional timeline of CTA 0 (clock64 stamps per role), compiled only when
// IDSK_TC_TRACE is defined by a profiling harness.
#ifdef IDSK_TC_TRACE
__device__ long long g_tc_trace[4][8192];
#define TC_TRACE(role, idx)                                              \
  do {                                                                   \
    if (blockIdx.x == 0 && (idx) < 8192) g_tc_trace[role][idx] = clock64(); \
  } while (0)
#else
#define TC_TRACE(role, idx) \
  do {                      \
  } while (0)
#endif

// barrier slots
enum { B_FULL0 = 0, B_FULL1, B_FREE0, B_FREE1, B_PSIF0, B_PSIE0 = B_PSIF0 + 4,
       B_YF0 = B_PSIE0 + 4, B_YF1, B_YE0, B_YE1, B_WF0, B_WE0 = B_WF0 + kTcMaxTiles,
       B_DONE = B_WE0 + kTcMaxTiles, B_RF0, B_RE0 = B_RF0 + NST, NBAR = B_RE0 + NST };

struct Smem {
  uint32_t pieces;   // [2 buffers][NP][PIECE_BYTES] (TMA form: [2 slots][PIECE_BYTES])
  uint32_t raw;      // TMA form: [NST][RAW_BYTES]
  uint32_t omega;    // [kTcMaxTiles][OMEGA_TILE_BYTES]
  uint32_t psi;      // [2][PSI_BYTES]
  uint32_t bars;     // NBAR x 8 bytes
  uint32_t tmem_slot;
  uint32_t abort_flag;
};

__device__ __forceinline__ void st_v4_f32_hint(float* p, float a, float b, float c, float d,
                                               uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(a),
               "f"(b), "f"(c), "f"(d), "l"(policy)
               : "memory");
}
__device__ __forceinline__ void red_add_v4_f32(float* p, float a, float b, float c, float d,
                                               uint64_t policy) {
  asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p),
               "f"(a), "f"(b), "f"(c), "f"(d), "l"(policy)
               : "memory");
}

__device__ __forceinline__ int64_t coarse_index_tc(int64_t r, const CoarseGeom& g) {
  const int64_t i = r % g.nx;
  const int64_t rest = r / g.nx;
  const int64_t z = rest % g.nz;
  const int64_t rest2 = rest / g.nz;
  const int64_t j = rest2 % g.ny;
  const int64_t c = rest2 / g.ny;
  if (i % g.sx || j % g.sy || z % g.sz) return -1;
  return ((c * g.cy + j / g.sy) * g.cz + z / g.sz) * g.cx + i / g.sx;
}

__device__ __forceinline__ const float* column_ptr(const Window& w, int c) {
  for (int s = 0; s < w.nseg; ++s) {
    const Seg& sg = w.seg[s];
    if (c >= sg.col0 && c < sg.col0 + sg.ncols)
      return reinterpret_cast<const float*>(sg.ptr) + (int64_t)(c - sg.col0) * sg.ld;
  }
  return nullptr;
}

// The loaded value of column c, rows r0..r0+3, with out-of-range entries zero
// (ragged last row block: the valid rows are read here, element by element).
__device__ __forceinline__ float4 split_source(const SketchArgs& a, const Window& w, int64_t r0,
                                               int c, float4 x) {
  if (r0 + 3 < a.m && c < w.ncols) return x;
  float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c < w.ncols && r0 < a.m) {
    const float* p = column_ptr(w, c) + r0;
    y.x = p[0];
    if (r0 + 1 < a.m) y.y = p[1];
    if (r0 + 2 < a.m) y.z = p[2];
  }
  return y;
}

// FP8 form: two values rounded to the nearest FP8-E4M3 value, ties to even,
// saturating at +-448 (the hardware conversion), and widened back exactly
// through half precision (E4M3 values are exact in half and in bfloat16);
// lo goes to the low half.
__device__ __forceinline__ float2 e4m3x2(float lo, float hi) {
  uint16_t p;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(p) : "f"(hi), "f"(lo));
  uint32_t h;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h) : "h"(p));
  return __half22float2(*reinterpret_cast<const __half2*>(&h));
}

__device__ __forceinline__ float4 e4m3_scaled(float4 x, float sc) {
  const float2 a = e4m3x2(x.x * sc, x.y * sc), b = e4m3x2(x.z * sc, x.w * sc);
  return make_float4(a.x, a.y, b.x, b.y);
}

// Psi(0 .. l-1, r) of row r into column rl of a K-major Psi tile (zero past
// the last row), in groups of ten draws: only the ceil(l / 10) groups that
// hold rows below l are drawn.  The tile's rows from there to LWT - 1 keep
// whatever they hold; they only feed the W^T accumulator columns past l,
// which no sum reads.  The loop over the groups stays rolled:
// unrolled, the longer epilogue code made the sketch slower for every n but
// the smallest (measured: 2.64 against 2.76 ms per launch with Y; 1.75
// against 1.77 us per tile at n = 512 without Y; 3.16 against 2.73 us at
// n = 64, one 128-column tile per row block).
template <int LWT>
__device__ __forceinline__ void psi_row(const SketchArgs& a, int64_t r, int rl, uint32_t dst) {
  const int ngroups = (min(a.l, LWT) + 9) / 10;
#pragma unroll 1
  for (int sb = 0; sb < ngroups; ++sb) {
    float g[10];
    if (r < a.m) {
      gauss10((uint64_t)r, (uint32_t)(sb + a.s0 / 10), kStreamPsi, a.k0, a.k1, a.table, g);
    } else {
#pragma unroll
      for (int f = 0; f < 10; ++f) g[f] = 0.f;
    }
#pragma unroll
    for (int f = 0; f < 10; ++f) {
      const int s = sb * 10 + f;
      if (s < LWT)
        st_shared_u16(dst + swz((uint32_t)s, (uint32_t)rl, 2048u), bf16_bits(s < a.l ? g[f] : 0.f));
    }
  }
}

// Shared-memory carve-up (1024-byte aligned base).  The batched kernel uses
// the TMA form's layout and keeps its current job's arguments after the
// abort flag.
template <int NP, bool TMA>
__device__ __forceinline__ Smem carve(uint32_t base) {
  Smem S;
  S.pieces = base;
  S.omega = S.pieces + (TMA ? 2u : 2u * NP) * PIECE_BYTES;
  S.psi = S.omega + kTcMaxTiles * OMEGA_TILE_BYTES;
  S.raw = S.psi + 2u * PSI_BYTES;
  S.bars = S.raw + (TMA ? NST * RAW_BYTES : 0u);
  S.tmem_slot = S.bars + NBAR * 8u;
  S.abort_flag = S.tmem_slot + 4u;
  return S;
}

// The CTA's barrier set (thread 0, once per kernel).
template <bool TMA>
__device__ __forceinline__ void init_bars(const Smem& S) {
  auto bar = [&](int i) { return S.bars + 8u * (uint32_t)i; };
  mbar_init(bar(B_FULL0), NCONV);
  mbar_init(bar(B_FULL1), NCONV);
  mbar_init(bar(B_FREE0), 1);
  mbar_init(bar(B_FREE1), 1);
  for (int pb = 0; pb < 4; ++pb) {
    mbar_init(bar(B_PSIF0 + pb), NEPI);
    mbar_init(bar(B_PSIE0 + pb), 1);
  }
  mbar_init(bar(B_YF0), 1);
  mbar_init(bar(B_YF1), 1);
  mbar_init(bar(B_YE0), NEPI);
  mbar_init(bar(B_YE1), NEPI);
  for (int ct = 0; ct < kTcMaxTiles; ++ct) {
    mbar_init(bar(B_WF0 + ct), 1);
    mbar_init(bar(B_WE0 + ct), NEPI);
  }
  mbar_init(bar(B_DONE), 1);
  if (TMA) {
    for (int st = 0; st < NST; ++st) {
      mbar_init(bar(B_RF0 + st), 1);
      mbar_init(bar(B_RE0 + st), NCONV);
    }
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Running counts of each role across the row ranges that one CTA processes
// (the persistent batched kernel runs many ranges with one barrier set, so
// every barrier phase follows from these counts; a single range starts them
// at zero).  A thread keeps only its own role's counts.
struct RoleCounters {
  int g = 0;           // row blocks (epilogue, MMA issuer)
  int u = 0;           // bfloat16 piece units (TMA converters, MMA issuer)
  int t = 0;           // tiles (register-form converters and MMA issuer)
  int box = 0;         // raw TMA boxes (TMA converters, producer)
  int done = 0;        // completed ranges (MMA issuer: phase of B_DONE)
  uint32_t wpar = 0;   // per W^T tile: parity of its flushes (epilogue, MMA issuer)
  uint32_t wpend = 0;  // MMA issuer: tiles handed to the epilogue, not yet read back
};

// The roles of one CTA over row blocks rb_begin .. rb_begin + nloc - 1 of
// one window (ncols columns), its W^T
// partials into the FP32 slab `slab` ([nct * 128][64]).  tm: generic address
// of the window's tensor map (TMA form); w: the window's segments (register
// form only).
template <int NP, bool TMA, bool WY, bool Q8 = false>
__device__ __forceinline__ void sketch_roles(const SketchArgs& a, const Window* wp, int ncols,
                                             uint64_t tm, int64_t rb_begin,
                                             int nloc, float* slab, int drain_blocks,
                                             const Smem& S, uint32_t tmem, uint8_t* smem_raw,
                                             RoleCounters& rc) {
  auto bar = [&](int i) { return S.bars + 8u * (uint32_t)i; };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nct = (ncols + TCOLS - 1) / TCOLS;
  const int ntile = nloc * nct;
  // Widths and the Psi ring: with Y, W^T tiles of 64 columns and two Psi
  // buffers; without Y, W^T tiles of 64 or 96 columns (l <= 96 in one pass:
  // the Y accumulators' TMEM is free) and four Psi buffers in the shared
  // memory that Omega would use (and the usual Psi buffers after it).
  constexpr bool wy = WY;   // a.want_Y, fixed per instantiation
  const int lw = WY ? LP : w_width(a.l, false);
  constexpr int npsi = WY ? 2 : 4;
  const uint32_t psi0 = WY ? S.psi : S.omega;
  const uint32_t psi_bytes = (uint32_t)lw * TR * 2u;

  // W^T tile ct is flushed after row block i when drain_due(i, ct): every
  // drain_blocks row blocks, the tiles offset from one another so that the
  // flushes spread over the row blocks, and all tiles after the last one
  auto drain_due = [&](int i, int ct) {
    return ((i + 1 + (ct * drain_blocks) / kTcMaxTiles) % drain_blocks) == 0 || i == nloc - 1;
  };

  if (warp < NCONV) {
    if constexpr (TMA) {
    // ------------------------------------------------------ converters (TMA)
    // Raw FP32 boxes (32 columns x 128 rows, 512 B per column) arrive in an
    // NST-stage ring; thread (warp w, lane l) splits one column, rows
    // 4(l%8) + 32g of each box into the (single) piece buffer.  The eight
    // lanes of a quarter warp share a column; the two quarters of each half
    // warp take columns 4 apart, so that every 8-byte store phase covers all
    // 32 banks of the 128-byte-swizzled piece (columns c and c + 4 have
    // disjoint 16-byte chunk positions for rows 0-31).
    const int cl = (warp >> 1) * 8 + (warp & 1) * 2 + ((lane >> 3) & 1) * 4 + (lane >> 4);
    const int rq = (lane & 7) * 4;
    const uint8_t* rawp = smem_raw + (S.raw - smem_u32(smem_raw));
    int U = rc.u, X = rc.box;
    bool ok = true;
    for (int i = 0; i < nloc && ok; ++i) {
      for (int ct = 0; ct < nct && ok; ++ct, U += NP, X += 4) {
        // Piece units u take the two piece slots in turn (slot u & 1, its
        // (u >> 1)-th use): with NP = 2 the MMAs of one piece run while the
        // converters write the other.
        const int u0 = U, s0 = u0 & 1;
        if (u0 >= 2 && !mbar_wait(bar(B_FREE0 + s0), ((u0 >> 1) - 1) & 1, S.abort_flag, 16)) {
          ok = false;
          break;
        }
        if (warp == 0 && lane == 0) TC_TRACE(0, 4 * u0);
        const uint32_t hi_buf = S.pieces + (uint32_t)s0 * PIECE_BYTES;
        uint32_t lo_keep[NP > 1 ? 32 : 1];   // second piece, packed, until its slot frees
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int xb = X + j, st = xb % NST;
          if (ok && !mbar_wait(bar(B_RF0 + st), (xb / NST) & 1, S.abort_flag)) ok = false;
          if (!ok) continue;
          const float* raw = reinterpret_cast<const float*>(rawp + st * RAW_BYTES);
          const int cc = 32 * j + cl;              // column inside the tile
          float sc = 1.f;                          // FP8 form: the column's scale
          if (Q8 && ct * TCOLS + cc < ncols) sc = a.colscale[ct * TCOLS + cc];
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int rr = 32 * g + rq;
            float4 x = *reinterpret_cast<const float4*>(raw + cl * TR + rr);
            if (Q8) x = e4m3_scaled(x, sc);
            const uint32_t off = swz((uint32_t)cc, (uint32_t)rr, 2048u);
            const uint32_t h01 = pack_bf16x2(x.x, x.y), h23 = pack_bf16x2(x.z, x.w);
            st_shared_v2(hi_buf + off, h01, h23);
            if (NP > 1) {
              const float2 f01 =
                  __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h01));
              const float2 f23 =
                  __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h23));
              lo_keep[(j * 4 + g) * 2] = pack_bf16x2(x.x - f01.x, x.y - f01.y);
              lo_keep[(j * 4 + g) * 2 + 1] = pack_bf16x2(x.z - f23.x, x.w - f23.y);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_RE0 + st));
        }
        if (!ok) break;
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_FULL0 + s0));
        if (warp == 0 && lane == 0) TC_TRACE(0, 4 * u0 + 1);
        if (NP > 1) {
          const int u1 = u0 + 1, s1 = u1 & 1;   // the other slot
          if (u1 >= 2 && !mbar_wait(bar(B_FREE0 + s1), ((u1 >> 1) - 1) & 1, S.abort_flag, 16)) {
            ok = false;
            break;
          }
          if (warp == 0 && lane == 0) TC_TRACE(0, 4 * u0 + 2);
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int g = 0; g < 4; ++g)
              st_shared_v2(S.pieces + (uint32_t)s1 * PIECE_BYTES +
                               swz((uint32_t)(32 * j + cl), (uint32_t)(32 * g + rq), 2048u),
                           lo_keep[(j * 4 + g) * 2], lo_keep[(j * 4 + g) * 2 + 1]);
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_FULL0 + s1));
        }
        if (warp == 0 && lane == 0) TC_TRACE(0, 4 * u0 + 3);
      }
    }
    rc.u = U;
    rc.box = X;
    } else {
    // ------------------------------------------------------------ converters
    // A tile is two half tiles of 64 columns; each thread owns 8 columns x 4
    // rows of a half tile.  The loads of the next half tile are issued before
    // the current one is split and stored (ping-pong register buffers), with
    // plain address arithmetic on the window's single segment when it has one.
    const Window& w = *wp;
    const int row_off = lane * 4;
    const bool one_seg = (w.nseg == 1);
    const float* seg_base = reinterpret_cast<const float*>(w.seg[0].ptr);
    const int64_t seg_ld = w.seg[0].ld;
    auto load_half = [&](int64_t r0, int c0, float4 (&v)[8]) {
      const bool rows_ok = r0 + 3 < a.m;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = c0 + j;
        const float* p = seg_base;
        if (rows_ok && c < w.ncols)
          p = one_seg ? seg_base + (int64_t)c * seg_ld + r0 : column_ptr(w, c) + r0;
        v[j] = __ldcs(reinterpret_cast<const float4*>(p));
      }
    };
    auto store_half = [&](uint32_t pbuf, int64_t r0, int c0, int col_off,
                          const float4 (&v)[8]) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float4 x = split_source(a, w, r0, c0 + j, v[j]);
        if (Q8) x = e4m3_scaled(x, c0 + j < w.ncols ? a.colscale[c0 + j] : 1.f);
        const uint32_t off = swz((uint32_t)(col_off + j), (uint32_t)row_off, 2048u);
        const uint32_t h01 = pack_bf16x2(x.x, x.y), h23 = pack_bf16x2(x.z, x.w);
        st_shared_v2(pbuf + off, h01, h23);
        if (NP > 1) {
          const float2 f01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h01));
          const float2 f23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h23));
          st_shared_v2(pbuf + PIECE_BYTES + off, pack_bf16x2(x.x - f01.x, x.y - f01.y),
                       pack_bf16x2(x.z - f23.x, x.w - f23.y));
        }
      }
    };
    const int c_lo = warp * 8;         // half 0 columns of this warp
    const int c_hi = 64 + warp * 8;    // half 1 columns
    float4 bufA[8], bufB[8];
    if (ntile > 0) load_half(rb_begin * TR + row_off, c_lo, bufA);
    int tl = 0;   // tile index inside the range; rc.t + tl: the running count
    bool ok = true;
    for (int i = 0; i < nloc && ok; ++i) {
      const int64_t r0 = (rb_begin + i) * TR + row_off;
      for (int ct = 0; ct < nct; ++ct, ++tl) {
        const int cbase = ct * TCOLS;
        load_half(r0, cbase + c_hi, bufB);                       // half 1 of this tile
        const int t = rc.t + tl, b = t & 1;
        if (t >= 2 && !mbar_wait(bar(B_FREE0 + b), ((t >> 1) - 1) & 1, S.abort_flag)) {
          ok = false;
          break;
        }
        const uint32_t pbuf = S.pieces + (uint32_t)b * NP * PIECE_BYTES;
        store_half(pbuf, r0, cbase + c_lo, c_lo, bufA);          // half 0
        if (tl + 1 < ntile) {                                     // half 0 of the next tile
          const bool last_ct = (ct + 1 == nct);
          load_half(last_ct ? r0 + TR : r0, last_ct ? c_lo : cbase + TCOLS + c_lo, bufA);
        }
        store_half(pbuf, r0, cbase + c_hi, c_hi, bufB);          // half 1
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_FULL0 + b));
        if (warp == 0 && lane == 0) TC_TRACE(0, t);
      }
    }
    rc.t += ntile;
    }
  } else if (warp < MMA_WARP) {
    // -------------------------------------------------------------- epilogue
    const int q = warp - NCONV;           // TMEM lane quarter
    const int rl = q * 32 + lane;         // row (Y) / column (W^T) inside the tile
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int g0 = rc.g;   // running row-block count: Psi buffer and Y accumulator phases
    // Psi of row block i of the range into buffer (g0 + i) mod npsi, once
    // the MMAs of the row block npsi earlier (maybe of an earlier range)
    // have completed; false when the wait gave up
    auto gen_psi = [&](int i) {
      const int g = g0 + i, pb = g & (npsi - 1);
      if (g >= npsi &&
          !mbar_wait(bar(B_PSIE0 + pb), ((g / npsi) - 1) & 1, S.abort_flag, 256))
        return false;
      const int64_t r = (rb_begin + i) * TR + rl;
      const uint32_t dst = psi0 + (uint32_t)pb * psi_bytes;
      if (WY || lw == 64)
        psi_row<64>(a, r, rl, dst);
      else
        psi_row<96>(a, r, rl, dst);
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_PSIF0 + pb));
      return true;
    };
    bool pok = true;
    for (int i = 0; i < npsi && i < nloc && pok; ++i) pok = gen_psi(i);
    uint32_t wpar = rc.wpar, wseen = 0;   // per W^T tile: flush parity, flushed in this range
    for (int i = 0; i < nloc && pok; ++i) {
      const int g = g0 + i, yb = g & 1;
      // a later window adds into Y: its old values of row block i + 2 are
      // prefetched into L2 now (the warp's 32 rows of every sketch column),
      // so that the read-modify-write at the drain waits for L2, not HBM
      // (a bulk prefetch needs 16-byte aligned addresses: m a multiple of 4)
      if (wy && a.y_accumulate && (a.m & 3) == 0 && i + 2 < nloc) {
        const int64_t r2 = (rb_begin + i + 2) * TR + q * 32;
        if (r2 + 32 <= a.m)
          for (int j = lane; j < a.l; j += 32)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], 128;" ::"l"(
                             reinterpret_cast<const float*>(a.Y) + r2 + (int64_t)j * a.m)
                         : "memory");
      }
      // flushes due after this row block first: each W^T tile's barrier is
      // committed right after that tile's MMAs, and the next row block's
      // MMAs wait for the tile to be read out
      bool wok = true;
      for (int ct = 0; ct < nct; ++ct) {
        if (!drain_due(i, ct)) continue;
        if (!mbar_wait(bar(B_WF0 + ct), (wpar >> ct) & 1u, S.abort_flag, 256)) {
          wok = false;
          break;
        }
        tc_fence_after();
        // the tile's 128 x lw partials into registers (32 columns at a
        // time); the accumulator goes back to the MMAs once the last chunk
        // is in registers, and the partials are added to this range's FP32
        // slab [c][s] (the first flush of a tile stores, later ones add in
        // L2, four entries per reduction; each slab entry is written by one
        // thread only, in program order, so the sum has a fixed order)
        const uint64_t keep = policy_evict_last();
        float* dst = slab + (int64_t)(ct * TCOLS + rl) * lw;
        const bool first = !((wseen >> ct) & 1u);
        auto put = [&](const float(&v)[32], int c0) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            if (first)
              st_v4_f32_hint(dst + c0 + j, v[j], v[j + 1], v[j + 2], v[j + 3], keep);
            else
              red_add_v4_f32(dst + c0 + j, v[j], v[j + 1], v[j + 2], v[j + 3], keep);
          }
        };
        float v[2][32];
        const uint32_t tcol = tmem + lane_base + (uint32_t)(ct * lw);
        tmem_ld32(tcol, v[0]);
        tmem_ld32(tcol + 32, v[1]);
        if (lw == 64) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_WE0 + ct));
        }
        put(v[0], 0);
        put(v[1], 32);
        if (lw == 96) {
          tmem_ld32(tcol + 64, v[0]);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_WE0 + ct));
          put(v[0], 64);
        }
        wpar ^= 1u << ct;
        wseen |= 1u << ct;
      }
      if (!wok) break;
      if (q == 0 && lane == 0) TC_TRACE(2, 4 * i);
      if (wy) {   // Y of row block i: accumulator yb
        if (!mbar_wait(bar(B_YF0 + yb), (g >> 1) & 1, S.abort_flag, 256)) break;
        tc_fence_after();
        if (q == 0 && lane == 0) TC_TRACE(2, 4 * i + 1);
        const int64_t r = (rb_begin + i) * TR + rl;
        float* Y = reinterpret_cast<float*>(a.Y);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[32];
          tmem_ld32(tmem + lane_base + (uint32_t)(TMEM_Y + yb * LP + h * 32), v);
          if (r < a.m) {
            float* yr = Y + r + (int64_t)(h * 32) * a.m;
            if (a.y_accumulate) {   // all loads in flight before the stores
              float old[32];
#pragma unroll
              for (int j = 0; j < 32; ++j)
                old[j] = (h * 32 + j < a.l) ? __ldcs(yr + (int64_t)j * a.m) : 0.f;
#pragma unroll
              for (int j = 0; j < 32; ++j) v[j] += old[j];
            }
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (h * 32 + j < a.l) __stcs(yr + (int64_t)j * a.m, v[j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_YE0 + yb));
      }
      if (q == 0 && lane == 0) TC_TRACE(2, 4 * i + 2);
      if (i + npsi < nloc && !gen_psi(i + npsi)) break;   // into row block i's buffer
      if (q == 0 && lane == 0) TC_TRACE(2, 4 * i + 3);
    }
    rc.g = g0 + nloc;
    rc.wpar = wpar;
  } else if (warp == MMA_WARP && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    uint32_t accw = 0;          // bit ct: W^T accumulator of tile ct holds data
    uint32_t wpend = rc.wpend;  // bit ct: tile ct handed to the epilogue, not yet read out
    uint32_t wpar = rc.wpar;    // bit ct: parity of the flushes of tile ct handed out
    const uint32_t idesc_w = lw == 96 ? IDESC_W96 : IDESC_W;
    int t = rc.t, U = rc.u;
    bool ok = true;
    for (int i = 0; i < nloc && ok; ++i) {
      const int g = rc.g + i, pb = g & (npsi - 1), yb = g & 1;
      if (!mbar_wait(bar(B_PSIF0 + pb), (g / npsi) & 1, S.abort_flag)) break;
      if (wy && g >= 2 && !mbar_wait(bar(B_YE0 + yb), ((g >> 1) - 1) & 1, S.abort_flag)) break;
      tc_fence_after();
      const uint32_t psi_s = psi0 + (uint32_t)pb * psi_bytes;
      const uint32_t ytm = tmem + (uint32_t)(TMEM_Y + yb * LP);
      for (int ct = 0; ct < nct; ++ct, ++t, U += NP) {
        const int b = t & 1;
        if (!TMA && !mbar_wait(bar(B_FULL0 + b), (t >> 1) & 1, S.abort_flag)) {
          ok = false;
          break;
        }
        if ((wpend >> ct) & 1u) {   // the epilogue must have read the last flush
          if (!mbar_wait(bar(B_WE0 + ct), ((wpar >> ct) & 1u) ^ 1u, S.abort_flag)) {
            ok = false;
            break;
          }
          wpend &= ~(1u << ct);
        }
        tc_fence_after();
        const uint32_t pbuf = S.pieces + (uint32_t)b * NP * PIECE_BYTES;
        const uint32_t wtm = tmem + (uint32_t)(ct * lw);
        const uint32_t om = S.omega + (uint32_t)ct * OMEGA_TILE_BYTES;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          uint32_t pa = pbuf + (uint32_t)p * PIECE_BYTES;
          const int u = U + p;   // TMA form: piece unit u in slot u & 1
          if (TMA) {   // the MMA thread is on the critical path: poll without sleeping
            if (!mbar_wait_spin(bar(B_FULL0 + (u & 1)), (u >> 1) & 1, S.abort_flag)) {
              ok = false;
              break;
            }
            TC_TRACE(1, 2 * u);
            tc_fence_after();
            pa = S.pieces + (uint32_t)(u & 1) * PIECE_BYTES;
          }
          // Descriptors: the base ones once per piece; the K steps only move
          // the start-address field (address >> 4, bits 0-13), which the
          // constant offsets below never carry out of (shared addresses <
          // 256 KB), so the single issuing thread spends two integer adds per
          // MMA instead of rebuilding both descriptors.
          const uint64_t dA = sdesc(pa, 0u, 2048u), dPsi = sdesc(psi_s, 0u, 2048u);
          const uint64_t dAy = sdesc(pa, 1024u, 2048u), dOm = sdesc(om, 0u, 2048u);
          const uint32_t acc0 = (accw >> ct) & 1u;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {   // W^T: K = 16 rows per instruction
            const uint64_t ko = (uint64_t)((kk >> 2) * 64 + (kk & 3) * 2);   // bytes >> 4
            mma_bf16(wtm, dA + ko, dPsi + ko, idesc_w, acc0 | (uint32_t)(p | kk));
          }
          if (wy) {   // without Y the pieces feed the W^T product only
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {   // Y: K = 16 columns per instruction
              const uint64_t ko = (uint64_t)((kk >> 2) * 64 + (kk & 3) * 2);
              mma_bf16(ytm, dAy + (uint64_t)(kk * 256), dOm + ko, IDESC_Y,
                       (uint32_t)(ct | p | kk));
            }
          }
          if (TMA) mma_commit(bar(B_FREE0 + (u & 1)));
          TC_TRACE(1, 2 * u + 1);
        }
        if (!ok) break;
        accw |= 1u << ct;
        if (!TMA) mma_commit(bar(B_FREE0 + b));
        if (drain_due(i, ct)) {   // hand tile ct's partials to the epilogue
          mma_commit(bar(B_WF0 + ct));
          wpar ^= 1u << ct;
          wpend |= 1u << ct;
          accw &= ~(1u << ct);
        }
      }
      if (!ok) break;
      if (wy) mma_commit(bar(B_YF0 + yb));
      mma_commit(bar(B_PSIE0 + pb));
    }
    // every issued MMA has completed before the range ends (the TMEM is
    // released, or the next range overwrites the accumulators)
    mma_commit(bar(B_DONE));
    const long long t0 = clock64();
    while (!mbar_try(bar(B_DONE), rc.done & 1)) {
      if (clock64() - t0 > kWaitCycles) {
        st_volatile_shared(S.abort_flag, 1);
        break;
      }
    }
    rc.done += 1;
    rc.g += nloc;
    rc.t = t;
    rc.u = U;
    rc.wpar = wpar;
    rc.wpend = wpend;
  } else if (TMA && warp == PROD_WARP && lane == 0) {
    // -------------------------------------------------------- TMA producer
    const uint64_t stream_once = policy_evict_first();
    int u = rc.box;
    bool ok = true;
    for (int t = 0; t < ntile && ok; ++t) {
      const int i = t / nct, ct = t - i * nct;
      const int row = (int)((rb_begin + i) * TR);
      for (int j = 0; j < 4; ++j, ++u) {
        const int st = u % NST;
        if (u >= NST && !mbar_wait(bar(B_RE0 + st), ((u / NST) - 1) & 1, S.abort_flag, 32)) {
          ok = false;
          break;
        }
        TC_TRACE(3, u);
        mbar_expect_tx(bar(B_RF0 + st), RAW_BYTES);
        tma_load_2d(S.raw + (uint32_t)st * RAW_BYTES, tm, row, ct * TCOLS + 32 * j,
                    bar(B_RF0 + st), stream_once);
      }
    }
    rc.box = u;
  }
}

// Omega(window, :) as a K-major bf16 B operand of the Y product, resident
// for the row range.
template <bool TMA, bool Q8>
__device__ __forceinline__ void fill_omega(const Smem& S, const SketchArgs& a, int ncols,
                                           int64_t col_base) {
  constexpr int NT_ALL = TMA ? NTHREADS_TMA : NTHREADS;
  for (int e = threadIdx.x; e < kTcMaxTiles * TCOLS * LP; e += NT_ALL) {
    const int s = e % LP, c = e / LP;
    float v = 0.f;
    if (s < a.l && c < ncols) v = a.omega[(col_base + c) * a.l + s];
    if (Q8 && c < ncols) v /= a.colscale[c];   // a power of two: exact (FP8 form)
    st_shared_u16(S.omega + (uint32_t)(c >> 7) * OMEGA_TILE_BYTES + swz(s, c & 127, 2048u),
                  bf16_bits(v));
  }
}

__device__ __forceinline__ void tmem_alloc_all(const Smem& S) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   S.tmem_slot),
               "n"(TMEM_COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free_all(uint32_t tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
               "n"(TMEM_COLS)
               : "memory");
}

// One window of one matrix: CTA b takes the contiguous row blocks
// [nrb b / G, nrb (b + 1) / G) of the G CTAs, its W^T partials into slab b.
template <int NP, bool TMA, bool WY, bool Q8>
__global__ void __launch_bounds__(TMA ? NTHREADS_TMA : NTHREADS, 1)
    sketch_tc_kernel(const __grid_constant__ SketchArgs a, const __grid_constant__ Window w,
                     int drain_blocks, int* __restrict__ status,
                     const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ uint8_t smem_raw[];
  const Smem S = carve<NP, TMA>((smem_u32(smem_raw) + 1023u) & ~1023u);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t nrb = (a.m + TR - 1) / TR;
  const int64_t rb_begin = nrb * blockIdx.x / gridDim.x;
  const int64_t rb_end = nrb * (blockIdx.x + 1) / gridDim.x;
  if (tid == 0) {
    st_volatile_shared(S.abort_flag, 0);
    init_bars<TMA>(S);
  }
  if (WY) fill_omega<TMA, Q8>(S, a, w.ncols, w.col_base);
  if (warp == MMA_WARP) tmem_alloc_all(S);
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(S.tmem_slot) : "memory");
  RoleCounters rc;
  sketch_roles<NP, TMA, WY, Q8>(a, &w, w.ncols, reinterpret_cast<uint64_t>(&tmap), rb_begin,
                            (int)(rb_end - rb_begin),
                            a.wpart + (int64_t)blockIdx.x * (kTcMaxTiles * TCOLS) *
                                          w_width(a.l, a.want_Y != 0),
                            drain_blocks, S, tmem, smem_raw, rc);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == MMA_WARP) tmem_free_all(tmem);
  if (tid == 0 && ld_volatile_shared(S.abort_flag)) atomicOr(status, 1);
}

// Batched form, the last step of one matrix: W = the sum of its items'
// slabs in item order (deterministic, FP32 pairs, read past L1: other SMs
// wrote them), then the pivoted QR of W and the solve for P into the
// batch's outputs, all by this CTA (shared scratch in the free buffers).
__device__ __forceinline__ void finish_job(const BatchJob& jb, const BatchItem* __restrict__ items,
                                           const float* __restrict__ slabs, const QrJob& q,
                                           double tol_factor, uint8_t* scratch) {
  const int l = jb.a.l, n = jb.ncols, lw = w_width(l, false);
  for (int e = threadIdx.x; e < l * n; e += NTHREADS_TMA) {
    const int c = e / l, s = e - c * l;
    float hi = 0.f, lo = 0.f;
    for (int q0 = 0; q0 < jb.nitem; q0 += 8) {
      float x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        x[u] = q0 + u < jb.nitem
                   ? __ldcg(slabs + items[jb.item0 + q0 + u].slab + (int64_t)c * lw + s)
                   : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) df_add(hi, lo, x[u], 0.f);
    }
    jb.Wd[(int64_t)s * n + c] = (double)hi + (double)lo;
  }
  __syncthreads();
  qr::QrShared& sh = *reinterpret_cast<qr::QrShared*>(scratch);
  qr::cta_pivoted_qr<NTHREADS_TMA>(q.M, q.rows, q.n, q.n, q.k, tol_factor, q.R, q.J, q.colpos,
                                   q.kout, sh);
  __syncthreads();
  double* r11 = reinterpret_cast<double*>(scratch + 4096);
  double* rdiag = r11 + kLMaxW * kLMaxW;
  int* Js = reinterpret_cast<int*>(rdiag + kLMaxW);
  const int kk = qr::solve_setup(q.R, q.J, q.kout, q.n, r11, Js, rdiag);
  for (int j = threadIdx.x >> 5; j < q.n; j += NTHREADS_TMA / 32)
    qr::solve_column(j, q.R, q.colpos, q.k, kk, q.n, q.P, r11, rdiag);
  __syncthreads();
}

// Batched form in one persistent launch: a work list of row ranges (items)
// over the sketches (jobs) of many matrices, one CTA per SM.  A CTA takes the
// next item from a global counter (jobs in order of decreasing QR work, each
// job's items in row order), copies the job's arguments to shared memory,
// runs the roles over the item's row blocks into the item's W^T slab, and
// synchronises.  One barrier set serves all items: every role carries its
// running counts (RoleCounters) from item to item, so each wait expects the
// right phase, including the commits of an earlier item that nobody waited
// for inside it.  The CTA that completes a job's last item (counted per job
// after its slab writes are fenced) sums the job's slabs into W and runs its
// pivoted QR and solve, while the other CTAs go on with later items.  The
// TMEM stays allocated throughout.  Every wait stays bounded: a CTA that
// gives up raises its job's problem flag and stops taking items.
__global__ void __launch_bounds__(NTHREADS_TMA, 1)
    sketch_batch_kernel(const BatchJob* __restrict__ jobs, const CUtensorMap* __restrict__ tmaps,
                        const BatchItem* __restrict__ items, const int32_t* __restrict__ order,
                        int nitems, float* __restrict__ slabs, int* __restrict__ counters,
                        const QrJob* __restrict__ qjobs, double tol_factor,
                        int* __restrict__ stat, int drain_blocks) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t sbase = smem_u32(smem_raw);
  const Smem S = carve<1, true>((sbase + 1023u) & ~1023u);
  const uint32_t s_args = (S.abort_flag + 4u + 15u) & ~15u;       // SketchArgs of the job
  const uint32_t s_item = s_args + (uint32_t)sizeof(SketchArgs);   // item index
  const uint32_t s_last = s_item + 4u;                             // the item completed its job
  SketchArgs* args = reinterpret_cast<SketchArgs*>(smem_raw + (s_args - sbase));
  uint8_t* scratch = smem_raw + (S.pieces - sbase);   // free between items
  int* job_done = counters + 1;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    st_volatile_shared(S.abort_flag, 0);
    init_bars<true>(S);   // one barrier set for all ranges: phases follow the counters
  }
  if (warp == MMA_WARP) tmem_alloc_all(S);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(S.tmem_slot) : "memory");
  RoleCounters rc;
  for (;;) {
    if (tid == 0) {
      const int q = atomicAdd(counters, 1);
      st_volatile_shared(s_item, q < nitems ? order[q] : -1);
    }
    __syncthreads();
    {
      const int it = ld_volatile_shared(s_item);
      if (it < 0) break;
      const BatchItem item = items[it];
      const BatchJob& jb = jobs[item.job];
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&jb.a);
      uint32_t* dst = reinterpret_cast<uint32_t*>(args);
      for (int e = tid; e < (int)(sizeof(SketchArgs) / 4); e += NTHREADS_TMA) dst[e] = src[e];
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      const uint64_t tm = reinterpret_cast<uint64_t>(tmaps + item.job);
      if (jb.np == 2)
        sketch_roles<2, true, false>(*args, nullptr, jb.ncols, tm, item.rb0, item.nrb,
                                     slabs + item.slab, drain_blocks, S, tmem, smem_raw, rc);
      else
        sketch_roles<1, true, false>(*args, nullptr, jb.ncols, tm, item.rb0, item.nrb,
                                     slabs + item.slab, drain_blocks, S, tmem, smem_raw, rc);
    }
    if (warp >= NCONV && warp < MMA_WARP) __threadfence();   // the slab writes, GPU-wide
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int it = ld_volatile_shared(s_item);
    const int job = items[it].job;
    if (ld_volatile_shared(S.abort_flag)) {
      if (tid == 0) atomicOr(stat + jobs[job].prob, 1);
      break;
    }
    if (tid == 0) {
      __threadfence();
      const int done = atomicAdd(job_done + job, 1) + 1;
      st_volatile_shared(s_last, done == jobs[job].nitem ? 1 : 0);
    }
    __syncthreads();
    if (ld_volatile_shared(s_last)) {
      __threadfence();
      finish_job(jobs[job], items, slabs, qjobs[job], tol_factor, scratch);
      fence_proxy_async();   // the scratch's generic writes before the next TMA writes
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == MMA_WARP) tmem_free_all(tmem);
}

// W(:, window) = sum over CTAs of their slabs, in CTA order (deterministic),
// as FP32 pairs (about 48 bits; GB300's FP64 pipe is too narrow for 152
// dependent FP64 additions per entry), eight slabs' loads in flight at a
// time.  A CTA whose row range is empty never wrote its slab and is skipped
// (only possible when there are fewer row blocks than CTAs).
__global__ void wpart_reduce_kernel(const float* __restrict__ wpart, int nslab, int l, int lw,
                                    int ncols, int64_t nrb, double* __restrict__ W, int64_t ldw,
                                    int64_t col_base, const float* __restrict__ colscale) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * ncols) return;
  const int c = e / l, s = e - c * l;
  const float* src = wpart + (int64_t)c * lw + s;
  const int64_t slab = (int64_t)kTcMaxTiles * TCOLS * lw;
  const bool all_rows = nrb >= nslab;   // then every CTA owns at least one row block
  float hi = 0.f, lo = 0.f;
  for (int b0 = 0; b0 < nslab; b0 += 8) {
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = b0 + q;
      const bool used = b < nslab && (all_rows || nrb * (b + 1) / nslab != nrb * b / nslab);
      x[q] = used ? src[(int64_t)b * slab] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) df_add(hi, lo, x[q], 0.f);
  }
  double wv = (double)hi + (double)lo;
  if (colscale) wv /= (double)colscale[c];   // FP8 form: a power of two, exact
  W[(int64_t)s * ldw + col_base + c] = wv;
}

// FP8 form: per column of the window, the power of two 2^e with
// max_r |A(r, c)| 2^e <= 448 < max_r |A(r, c)| 2^(e + 1) (e in [-100, 100];
// 1 for a zero column), into scale[c].  One CTA per column.
__global__ void fp8_scale_kernel(const __grid_constant__ Window w, int64_t m,
                                 float* __restrict__ scale) {
  __shared__ float red[32];
  const int c = blockIdx.x;
  const float* col = column_ptr(w, c);
  float mx = 0.f;
  for (int64_t r = threadIdx.x; r < m; r += blockDim.x) mx = fmaxf(mx, fabsf(col[r]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmaxf(mx, red[i]);
    int e = 0;
    if (mx > 0.f) {
      int p = 0;
      const float f = frexpf(mx, &p);   // mx = f 2^p, 0.5 <= f < 1
      e = f <= 0.875f ? 9 - p : 8 - p;
      while (e > -100 && ldexpf(mx, e) > 448.f) --e;
      while (e < 100 && ldexpf(mx, e + 1) <= 448.f) ++e;
      e = max(-100, min(100, e));
    }
    scale[c] = ldexpf(1.f, e);
  }
}

template <int NP, bool TMA>
size_t tc_smem_bytes() {
  return 1024 + (TMA ? 2u : 2u * NP) * PIECE_BYTES + kTcMaxTiles * OMEGA_TILE_BYTES +
         2u * PSI_BYTES + (TMA ? NST * RAW_BYTES : 0u) + NBAR * 8 + 16;
}

// Tensor map of the window's single segment: rows x columns FP32, boxes of
// 128 rows x 32 columns, zero fill outside.  False when it cannot be built.
bool make_tmap(const SketchArgs& a, const Window& w, CUtensorMap* tm) {
  if (w.nseg != 1) return false;
  const char* env = getenv("IDSKETCH_SKETCH_TMA");
  if (env && env[0] == '0') return false;
  return make_tmap_f32_2d(w.seg[0].ptr, a.m, w.seg[0].ncols, w.seg[0].ld, TR, 32, tm);
}

template <int NP, bool TMA, bool WY, bool Q8>
cudaError_t launch_variant(const SketchArgs& a, const Window& w, int grid, int drain_blocks,
                           int* status, const CUtensorMap& tm, cudaStream_t st,
                           KernelTimer* timer) {
  const size_t sm = tc_smem_bytes<NP, TMA>();
  cudaError_t e = cudaFuncSetAttribute(sketch_tc_kernel<NP, TMA, WY, Q8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (timer && (e = timer->mark(st)) != cudaSuccess) return e;
  sketch_tc_kernel<NP, TMA, WY, Q8><<<grid, TMA ? NTHREADS_TMA : NTHREADS, sm, st>>>(
      a, w, drain_blocks, status, tm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (timer) e = timer->mark(st);
  return e;
}

}  // namespace

#ifdef IDSK_TC_TRACE
// Profiling harness only: the clock64 timeline of CTA 0 ([4][8192]): role 0
// converter warp 0 (per tile with first piece unit u: 4u start, 4u+1 first
// piece out, 4u+2 second slot free, 4u+3 second piece out), role 1 MMA (2u
// piece unit u ready, 2u+1 issued), role 2 epilogue (per row block i: 4i
// flushes done, 4i+1 Y ready, 4i+2 Y drained, 4i+3 Psi drawn), role 3
// producer (box u issued).
extern "C" int idsk_tc_trace_read(long long* host) {
  return (int)cudaMemcpyFromSymbol(host, g_tc_trace, sizeof(g_tc_trace));
}
#endif

cudaError_t launch_sketch_tc(const SketchArgs& a0, const Window& w, int npieces, int nsm,
                             int drain_blocks, int* status, cudaStream_t st, KernelTimer* timer) {
  if (w.ncols <= 0) return cudaSuccess;
  if (w.ncols > kTcMaxTiles * TCOLS || a0.l > kLMaxW || a0.s0 % 10 != 0)
    return cudaErrorInvalidValue;
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  const bool tma = make_tmap(a0, w, &tm);
  if (a0.l > LP && a0.want_Y) return cudaErrorInvalidValue;
  if (a0.l > LP && !tma) {
    if (a0.s0 != 0) return cudaErrorInvalidValue;
    // a wide sketch (W only) in the register form: one launch per kPassRows
    // rows of Psi, the coarse rows gathered by the first (the TMA form takes
    // all l <= 96 rows in one pass)
    for (int s0 = 0; s0 < a0.l; s0 += kPassRows) {
      SketchArgs a = a0;
      a.s0 = s0;
      a.l = std::min(kPassRows, a0.l - s0);
      a.W = a0.W + (int64_t)s0 * a0.ldw;
      if (s0 > 0) a.cg.on = 0;
      const cudaError_t e = launch_sketch_tc(a, w, npieces, nsm, drain_blocks, status, st, timer);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const SketchArgs& a = a0;
  const int64_t nrb = (a.m + TR - 1) / TR;
  const int grid = (int)std::min<int64_t>(nrb, nsm);
  cudaError_t e;
  auto go = [&](auto np, auto tmaf, auto wy) {
    return launch_variant<decltype(np)::value, decltype(tmaf)::value, decltype(wy)::value,
                          false>(a, w, grid, drain_blocks, status, tm, st, timer);
  };
  auto go8 = [&](auto tmaf, auto wy) {   // FP8 form: one piece, quantised
    return launch_variant<1, decltype(tmaf)::value, decltype(wy)::value, true>(
        a, w, grid, drain_blocks, status, tm, st, timer);
  };
  using T = std::true_type;
  using F = std::false_type;
  using N1 = std::integral_constant<int, 1>;
  using N2 = std::integral_constant<int, 2>;
  if (a.fp8) {
    if (npieces != 1 || !a.colscale) return cudaErrorInvalidValue;
    if (a.want_Y)
      e = tma ? go8(T(), T()) : go8(F(), T());
    else
      e = tma ? go8(T(), F()) : go8(F(), F());
  } else if (a.want_Y) {
    if (npieces == 1)
      e = tma ? go(N1(), T(), T()) : go(N1(), F(), T());
    else
      e = tma ? go(N2(), T(), T()) : go(N2(), F(), T());
  } else {
    if (npieces == 1)
      e = tma ? go(N1(), T(), F()) : go(N1(), F(), F());
    else
      e = tma ? go(N2(), T(), F()) : go(N2(), F(), F());
  }
  if (e != cudaSuccess) return e;
  const int tot = a.l * w.ncols;
  wpart_reduce_kernel<<<(tot + 255) / 256, 256, 0, st>>>(
      a.wpart, grid, a.l, w_width(a.l, a.want_Y != 0), w.ncols, nrb, a.W, a.ldw, w.col_base,
      a.fp8 ? a.colscale : nullptr);
  count_launches(2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.cg.on) e = launch_coarse_gather(w, a.crow, a.cg.mc, reinterpret_cast<float*>(a.Ac), st);
  return e;
}

namespace {
// The fine row of every coarse-grid row: crow[coarse_index(r)] = r.
__global__ void coarse_rows_kernel(CoarseGeom g, int64_t m, int64_t* __restrict__ crow) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int64_t rc = coarse_index_tc(r, g);
  if (rc >= 0) crow[rc] = r;
}

// A_c(:, window) = A(crow, window) (Algorithm 5 step 3), exact FP32, right
// after the window's sketch while its columns are still the caller's:
// blockIdx.y = column of the window, threads over the coarse rows.
__global__ void coarse_gather_kernel(const __grid_constant__ Window w,
                                     const int64_t* __restrict__ crow, int64_t mc,
                                     float* __restrict__ Ac) {
  const int c = blockIdx.y;
  const int64_t rc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (rc >= mc) return;
  const float* col = column_ptr(w, c);
  Ac[(w.col_base + c) * mc + rc] = col[crow[rc]];
}
}  // namespace

cudaError_t launch_coarse_rows(const CoarseGeom& g, int64_t m, int64_t* crow, cudaStream_t st) {
  coarse_rows_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(g, m, crow);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fp8_scales(const Window& w, int64_t m, float* scale, cudaStream_t st) {
  if (w.ncols <= 0) return cudaSuccess;
  fp8_scale_kernel<<<w.ncols, 256, 0, st>>>(w, m, scale);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_gather(const Window& w, const int64_t* crow, int64_t mc, float* Ac,
                                 cudaStream_t st) {
  if (w.ncols <= 0 || mc <= 0) return cudaSuccess;
  coarse_gather_kernel<<<dim3((unsigned)((mc + 255) / 256), (unsigned)w.ncols), 256, 0, st>>>(
      w, crow, mc, Ac);
  count_launches(1);
  return cudaGetLastError();
}

size_t sketch_batch_smem_bytes() {
  return tc_smem_bytes<1, true>() + 16 + sizeof(SketchArgs) + 16;
}

cudaError_t launch_sketch_batch(const BatchJob* jobs, const CUtensorMap* tmaps,
                                const BatchItem* items, const int32_t* order, int nitems,
                                float* slabs, int* counters, const QrJob* qjobs,
                                double tol_factor, int* stat, int grid, int drain_blocks,
                                cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const size_t sm = sketch_batch_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(sketch_batch_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  sketch_batch_kernel<<<grid, NTHREADS_TMA, sm, st>>>(jobs, tmaps, items, order, nitems, slabs,
                                                      counters, qjobs, tol_factor, stat,
                                                      drain_blocks);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace idsk
