// C ABI of the pass-efficient ID (declared in include/idsketch.h): handle
// lifecycle, column windows, argument checks and host/device outputs.  Every
// arithmetic step runs in the kernels of this directory.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "idsk_internal.h"

using namespace idsk;

namespace idsk {
int coarse_blocks_needed(int64_t mc, int nsm);

std::atomic<int64_t> g_launches{0};
std::atomic<int> g_last_cuda_error{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_table_mu;
float* g_table[kMaxDevices] = {nullptr};

// Device copy of the quantile table, one per device for the process lifetime.
cudaError_t device_table(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_table_mu);
  if (!g_table[dev]) {
    float host[kTableSize];
    gaussian_table_host(host, nullptr);
    float* d = nullptr;
    e = cudaMalloc(&d, sizeof(host));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(d, host, sizeof(host), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return e;
    }
    g_table[dev] = d;
  }
  *out = g_table[dev];
  return cudaSuccess;
}

// Optional allocation cap (bytes) for fault-injection tests.
size_t alloc_cap() {
  const char* s = getenv("IDSKETCH_ALLOC_CAP_BYTES");
  if (!s || !*s) return (size_t)-1;
  return (size_t)strtoull(s, nullptr, 10);
}

struct Allocator {
  size_t used = 0, cap = alloc_cap();
  id_status st = ID_OK;
  template <class T>
  void get(T** p, size_t count) {
    if (st != ID_OK || count == 0) return;
    const size_t bytes = count * sizeof(T);
    if (used + bytes > cap) {
      st = ID_ERR_OOM;
      return;
    }
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      st = ID_ERR_OOM;
      return;
    }
    if (e != cudaSuccess) {
      st = ID_ERR_CUDA;
      return;
    }
    used += bytes;
  }
};

void free_all(id_sketch* h) {
  void* ptrs[] = {h->d_omega, h->d_W, h->d_Y, h->d_Ac, h->d_work, h->d_R, h->d_P, h->d_J,
                  h->d_colpos, h->d_kout, h->d_V, h->d_F, h->d_nu2, h->d_nu20, h->d_gvec, h->d_hvec, h->d_vh, h->d_vl,
                  h->d_upart, h->d_cscal, h->d_cint, h->d_rlist, h->d_Rc, h->d_Pc, h->d_Jc,
                  h->d_colposc, h->d_part, h->d_out3, h->d_Jin, h->d_Pin, h->d_status, h->d_wpart,
                  h->d_axis, h->d_Sc, h->d_cand, h->d_fq, h->d_crow, h->d_colscale};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

id_status validate(const id_config* c) {
  if (!c) return ID_ERR_INVALID_ARG;
  if (c->m <= 0 || c->n_max <= 0 || c->n_max > (int64_t)1 << 30) return ID_ERR_INVALID_ARG;
  if (c->k < 1 || c->l < c->k || c->l > kLMaxW) return ID_ERR_INVALID_ARG;
  // l > 64: FP32 data, W only (the tensor-core sketch in passes; no Y), and
  // no coarse-grid QR above k = 64
  if (c->l > kLMax && (c->dtype != ID_F32 || c->want_Y)) return ID_ERR_UNSUPPORTED;
  if (c->want_coarse && c->k > kLMax) return ID_ERR_UNSUPPORTED;
  if (c->dtype != ID_F32 && c->dtype != ID_F64) return ID_ERR_INVALID_ARG;
  if (c->prec != ID_SKETCH_EXACT && c->prec != ID_SKETCH_BF16 && c->prec != ID_SKETCH_FP8E4M3)
    return ID_ERR_INVALID_ARG;
  if (c->prec != ID_SKETCH_EXACT && c->dtype != ID_F32) return ID_ERR_INVALID_ARG;
  if (c->window_cols < 0) return ID_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (c->reserved[i] != 0) return ID_ERR_INVALID_ARG;
  if (c->want_coarse) {
    if (c->ncomp < 1) return ID_ERR_INVALID_ARG;
    int64_t pts = c->ncomp;
    for (int d = 0; d < 3; ++d) {
      if (c->grid[d] < 1 || c->coarse_stride[d] < 1) return ID_ERR_INVALID_ARG;
      pts *= c->grid[d];
    }
    if (pts != c->m) return ID_ERR_INVALID_ARG;
  }
  if (c->n_max > 32 * 1024) return ID_ERR_INVALID_ARG;   // one-CTA pivoted QR limit
  return ID_OK;
}

#define IDSK_CUDA(h, expr)                 \
  do {                                     \
    cudaError_t e_ = (expr);               \
    if (e_ != cudaSuccess) {               \
      g_last_cuda_error.store((int)e_);    \
      (h)->poisoned = true;                \
      return ID_ERR_CUDA;                  \
    }                                      \
  } while (0)

// Tensor-core sketch: FP32 data whose pending columns all start on 16-byte
// boundaries (128-bit loads); everything else takes the SIMT kernel.
bool use_tc(const id_sketch* h) {
  if (h->cfg.dtype != ID_F32 || h->sketch_kernel == 2 || h->m < 128) return false;
  for (const Seg& s : h->pend)
    if (((uintptr_t)s.ptr & 15u) != 0 || (s.ld & 3) != 0) return false;
  return true;
}

}  // namespace

namespace idsk {

// Orders the side stream's coarse QR (if any is in flight) before the work
// that id_sketch's own stream enqueues next: it reads A_c and writes the
// coarse workspace, which a new sketch or a reset would overwrite.
id_status join_coarse(id_sketch* h) {
  if (!h->cq_pending) return ID_OK;
  IDSK_CUDA(h, cudaStreamWaitEvent(h->st, h->ev_cq, 0));
  h->cq_pending = false;
  return ID_OK;
}

id_status launch_pending(id_sketch* h) {
  if (!h->pend.empty()) {
    const id_status s = join_coarse(h);
    if (s != ID_OK) return s;
    h->coarse_spec = -1;   // new columns: a started coarse QR no longer applies
  }
  while (!h->pend.empty()) {
    Window w;
    memset(&w, 0, sizeof(w));
    w.col_base = h->n_launched;
    const bool tc = use_tc(h);
    if (!tc && h->l > kLMax) return ID_ERR_UNSUPPORTED;   // wide sketches: tensor-core path only
    const bool fp8 = h->cfg.prec == ID_SKETCH_FP8E4M3;
    if (!tc && fp8) return ID_ERR_UNSUPPORTED;             // FP8 form: tensor-core path only
    const int wmax = tc ? kTcMaxTiles * 128 : kSimtWindowMax;
    int taken = 0;
    size_t consumed = 0;
    while (consumed < h->pend.size() && w.nseg < kMaxSegs && taken < wmax) {
      Seg& s = h->pend[consumed];
      const int use = std::min(s.ncols, wmax - taken);
      Seg part = s;
      part.col0 = taken;
      part.ncols = use;
      w.seg[w.nseg++] = part;
      taken += use;
      if (use == s.ncols) {
        ++consumed;
      } else {
        s.ptr = (const char*)s.ptr + (size_t)use * s.ld * h->esz;
        s.ncols -= use;
      }
    }
    h->pend.erase(h->pend.begin(), h->pend.begin() + consumed);
    w.ncols = taken;

    SketchArgs a;
    memset(&a, 0, sizeof(a));
    a.m = h->m;
    a.l = h->l;
    a.lpad = h->lpad;
    a.k0 = h->key0;
    a.k1 = h->key1;
    a.table = h->d_table;
    a.omega = h->d_omega;
    a.W = h->d_W;
    a.ldw = h->n_max;
    a.Y = h->d_Y;
    a.want_Y = h->cfg.want_Y ? 1 : 0;
    a.y_accumulate = h->y_started ? 1 : 0;
    a.Ac = h->d_Ac;
    a.cg = h->cg;
    a.bf16 = h->cfg.prec == ID_SKETCH_BF16 ? 1 : 0;
    a.wpart = h->d_wpart;
    a.crow = h->d_crow;
    a.fp8 = fp8 ? 1 : 0;
    a.colscale = fp8 ? h->d_colscale + w.col_base : nullptr;
    if (fp8) IDSK_CUDA(h, launch_fp8_scales(w, h->m, h->d_colscale + w.col_base, h->st));
    const int nsm_eff = h->grid_cap > 0 ? std::min(h->grid_cap, h->nsm) : h->nsm;
    if (tc) {
      IDSK_CUDA(h, launch_sketch_tc(a, w, (a.bf16 || a.fp8) ? 1 : 2, nsm_eff, h->drain_blocks,
                                    h->d_status,
                                    h->st, h->timer_sketch));
    } else {
      IDSK_CUDA(h, launch_sketch_simt(a, w, h->cfg.dtype, nsm_eff, h->st));
    }
    h->y_started = true;
    h->n_launched += taken;
  }
  h->pend_cols = 0;
  return ID_OK;
}

id_status factor_enqueue(id_sketch* h, bool one_cta) {
  id_status s = launch_pending(h);
  if (s != ID_OK) return s;
  const int64_t n = h->n_seen;
  if (n == 0) return ID_ERR_STATE;
  const int k = h->k, l = h->l;
  IDSK_CUDA(h, cudaMemcpy2DAsync(h->d_work, sizeof(double) * n, h->d_W,
                                 sizeof(double) * h->n_max, sizeof(double) * n, l,
                                 cudaMemcpyDeviceToDevice, h->st));
  IDSK_CUDA(h, launch_cpqr_small(h->d_work, l, (int)n, (int)n, k, ID_RANK_TOL_FACTOR, h->d_R,
                                 h->d_J, h->d_colpos, h->d_kout, h->st, one_cta));
  IDSK_CUDA(h, launch_solve_p(h->d_R, h->d_J, h->d_colpos, h->d_kout, k, (int)n, h->d_P, h->st));
  return ID_OK;
}


}  // namespace idsk

namespace {

id_status copy_out(id_sketch* h, void* dst, const void* src, size_t bytes) {
  if (!dst || bytes == 0) return ID_OK;
  IDSK_CUDA(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->st));
  return ID_OK;
}

}  // namespace

// ------------------------------------------------------- single-pass ID
namespace {

idsk::InterpGeom interp_geom(const id_sketch* h) {
  idsk::InterpGeom g;
  g.ax = h->d_axis;
  g.ay = h->d_axis + h->cg.nx;
  g.az = h->d_axis + h->cg.nx + h->cg.ny;
  g.Sc = h->d_Sc;
  g.nx = h->cg.nx;
  g.ny = h->cg.ny;
  g.nz = h->cg.nz;
  g.cx = h->cg.cx;
  g.cy = h->cg.cy;
  g.cz = h->cg.cz;
  return g;
}

// Common checks of the single-pass calls; copies J_c (host or device) to the
// device and compacts the coarse skeleton A_c(:, J_c) into d_Sc.
id_status stage_coarse_skeleton(id_sketch* h, const int32_t* Jc, int32_t kc) {
  if (!h->cfg.want_coarse || !h->mesh_set) return ID_ERR_STATE;
  id_status s = launch_pending(h);
  if (s != ID_OK) return s;
  if (h->n_seen == 0) return ID_ERR_STATE;
  int32_t jh[kRecKMax];
  IDSK_CUDA(h, cudaMemcpyAsync(jh, Jc, sizeof(int32_t) * kc, cudaMemcpyDefault, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  for (int u = 0; u < kc; ++u)
    if (jh[u] < 0 || jh[u] >= h->n_seen) return ID_ERR_INVALID_ARG;
  IDSK_CUDA(h, cudaMemcpyAsync(h->d_Jin, jh, sizeof(int32_t) * kc, cudaMemcpyHostToDevice, h->st));
  IDSK_CUDA(h, launch_skeleton_compact(h->d_Ac, h->mc, h->cfg.dtype, h->d_Jin, kc, h->d_Sc, h->st));
  return ID_OK;
}

}  // namespace

extern "C" {

const char* id_status_str(id_status s) {
  switch (s) {
    case ID_OK: return "ok";
    case ID_ERR_INVALID_ARG: return "invalid argument";
    case ID_ERR_STATE: return "call out of order";
    case ID_ERR_OOM: return "out of device memory";
    case ID_ERR_CUDA: return "CUDA error";
    case ID_ERR_RANK_DEFICIENT: return "rank deficient: fewer than k pivots";
    case ID_ERR_TIMEOUT: return "device wait timed out";
    case ID_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

int32_t id_version(void) { return 100; }

int64_t id_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* id_last_cuda_error(void) {
  return cudaGetErrorString((cudaError_t)g_last_cuda_error.load());
}

id_status id_gaussian_table(uint16_t out[4096]) {
  if (!out) return ID_ERR_INVALID_ARG;
  gaussian_table_host(nullptr, out);
  return ID_OK;
}

id_status id_gaussian_fill(int32_t which, uint64_t seed, int64_t first, int64_t count,
                           int32_t width, float* d_out, void* cuda_stream) {
  if ((which != (int32_t)kStreamPsi && which != (int32_t)kStreamOmega) || first < 0 ||
      count < 0 || width < 1 || (count > 0 && !d_out))
    return ID_ERR_INVALID_ARG;
  if (count == 0) return ID_OK;
  float* tab = nullptr;
  if (device_table(&tab) != cudaSuccess) return ID_ERR_CUDA;
  cudaError_t e = launch_gaussian_fill((uint32_t)which, (uint32_t)seed, (uint32_t)(seed >> 32),
                                       first, count, width, tab, d_out,
                                       (cudaStream_t)cuda_stream);
  return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

id_status id_sketch_create(const id_config* cfg, void* cuda_stream, id_sketch** out) {
  if (!out) return ID_ERR_INVALID_ARG;
  *out = nullptr;
  id_status v = validate(cfg);
  if (v != ID_OK) return v;
  id_sketch* h = new (std::nothrow) id_sketch();
  if (!h) return ID_ERR_OOM;
  h->cfg = *cfg;
  h->st = (cudaStream_t)cuda_stream;
  h->m = cfg->m;
  h->n_max = cfg->n_max;
  h->k = cfg->k;
  h->l = cfg->l;
  h->lpad = ((cfg->l + 15) / 16) * 16;
  h->esz = cfg->dtype == ID_F64 ? 8 : 4;
  h->key0 = (uint32_t)cfg->seed;
  h->key1 = (uint32_t)(cfg->seed >> 32);
  if (cudaGetDevice(&h->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return ID_ERR_CUDA;
  }
  if (cfg->want_coarse) {
    CoarseGeom& g = h->cg;
    g.on = 1;
    g.nx = cfg->grid[0];
    g.ny = cfg->grid[1];
    g.nz = cfg->grid[2];
    g.sx = cfg->coarse_stride[0];
    g.sy = cfg->coarse_stride[1];
    g.sz = cfg->coarse_stride[2];
    g.cx = (g.nx + g.sx - 1) / g.sx;
    g.cy = (g.ny + g.sy - 1) / g.sy;
    g.cz = (g.nz + g.sz - 1) / g.sz;
    g.mc = (int64_t)cfg->ncomp * g.cx * g.cy * g.cz;
    h->mc = g.mc;
  }
  if (device_table(&h->d_table) != cudaSuccess) {
    delete h;
    return ID_ERR_CUDA;
  }
  if (const char* e = getenv("IDSKETCH_SKETCH")) {
    if (!strcmp(e, "tc")) h->sketch_kernel = 1;
    if (!strcmp(e, "simt")) h->sketch_kernel = 2;
  }
  if (const char* e = getenv("IDSKETCH_DRAIN_BLOCKS")) h->drain_blocks = std::max(1, atoi(e));
  const int64_t nm = h->n_max;
  const int k = h->k, l = h->l;
  Allocator al;
  al.get(&h->d_status, 1);
  if (cfg->dtype == ID_F32)
    al.get(&h->d_wpart,
           (size_t)h->nsm * w_width(cfg->l, cfg->want_Y != 0) * kTcMaxTiles * 128);
  al.get(&h->d_omega, (size_t)nm * l);
  al.get(&h->d_W, (size_t)l * nm);
  if (cfg->want_Y) al.get((char**)&h->d_Y, (size_t)h->m * l * h->esz);
  if (cfg->want_coarse) al.get((char**)&h->d_Ac, (size_t)h->mc * nm * h->esz);
  if (cfg->want_coarse && cfg->dtype == ID_F32) al.get(&h->d_crow, (size_t)h->mc);
  if (cfg->prec == ID_SKETCH_FP8E4M3) al.get(&h->d_colscale, (size_t)nm);
  al.get(&h->d_work, (size_t)l * nm);
  al.get(&h->d_R, (size_t)k * nm);
  al.get(&h->d_P, (size_t)k * nm);
  al.get(&h->d_J, (size_t)k);
  al.get(&h->d_colpos, (size_t)nm);
  al.get(&h->d_kout, 1);
  al.get(&h->d_cand, (size_t)nm);
  al.get(&h->d_fq, (size_t)l * k + k + (size_t)k * k);
  h->rec_blocks = 8 * h->nsm;
  al.get(&h->d_part, (size_t)3 * h->rec_blocks);
  al.get(&h->d_out3, 3);
  al.get(&h->d_Jin, (size_t)kRecKMax);
  if (cfg->want_coarse) {
    h->coarse_blocks = coarse_blocks_needed(h->mc, h->nsm);
    al.get(&h->d_V, (size_t)h->mc * k);
    al.get(&h->d_F, (size_t)nm * k);
    al.get(&h->d_nu2, (size_t)nm);
    al.get(&h->d_nu20, (size_t)nm);
    al.get(&h->d_gvec, (size_t)h->coarse_blocks * nm);            // row-range partials of A_c^T u
    al.get(&h->d_hvec, (size_t)kLMax);                             // V_s^T v_s
    al.get(&h->d_vh, (size_t)h->mc + 8);                           // u below row s, FP32 pair
    al.get(&h->d_vl, (size_t)h->mc + 8);
    al.get(&h->d_upart, (size_t)h->coarse_blocks * (kLMax + 1));   // V_s^T u, ||u||^2 partials
    al.get(&h->d_cscal, 8);
    al.get(&h->d_cint, 8);
    al.get(&h->d_rlist, (size_t)nm);
    al.get(&h->d_Rc, (size_t)k * nm);
    al.get(&h->d_Pc, (size_t)k * nm);
    al.get(&h->d_Jc, (size_t)k);
    al.get(&h->d_colposc, (size_t)nm);
  }
  if (al.st != ID_OK) {
    free_all(h);
    delete h;
    return al.st;
  }
  cudaError_t e = launch_gaussian_fill(kStreamOmega, h->key0, h->key1, 0, nm, l, h->d_table,
                                       h->d_omega, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_W, 0, sizeof(double) * l * nm, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st);
  if (e == cudaSuccess && h->d_crow) e = launch_coarse_rows(h->cg, h->m, h->d_crow, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e == cudaSuccess && cfg->want_coarse && cfg->dtype == ID_F32 &&
      !getenv("IDSKETCH_NO_SIDE_STREAM")) {
    e = cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_sk, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_cq, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    if (h->st2) cudaStreamDestroy(h->st2);
    if (h->ev_sk) cudaEventDestroy(h->ev_sk);
    if (h->ev_cq) cudaEventDestroy(h->ev_cq);
    free_all(h);
    delete h;
    return ID_ERR_CUDA;
  }
  *out = h;
  return ID_OK;
}

id_status id_sketch_stream_columns(id_sketch* h, const void* d_cols, int64_t ld, int64_t ncols) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  if (ncols < 0 || (ncols > 0 && (!d_cols || ld < h->m))) return ID_ERR_INVALID_ARG;
  if (h->n_seen + ncols > h->n_max) return ID_ERR_INVALID_ARG;
  if (ncols == 0) return ID_OK;
  Seg s;
  s.ptr = d_cols;
  s.ld = ld;
  s.col0 = 0;
  s.ncols = (int32_t)ncols;
  if (!h->pend.empty()) {
    Seg& b = h->pend.back();
    const char* end = (const char*)b.ptr + (size_t)b.ncols * b.ld * h->esz;
    if (b.ld == ld && end == (const char*)d_cols) {
      b.ncols += (int32_t)ncols;
    } else {
      h->pend.push_back(s);
    }
  } else {
    h->pend.push_back(s);
  }
  h->n_seen += ncols;
  h->pend_cols += ncols;
  if (h->cfg.window_cols == 0 || h->pend_cols >= h->cfg.window_cols) return launch_pending(h);
  return ID_OK;
}

id_status id_sketch_flush(id_sketch* h) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  return launch_pending(h);
}

id_status id_sketch_reset(id_sketch* h) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  const id_status js = join_coarse(h);
  if (js != ID_OK) return js;
  h->coarse_spec = -1;
  h->pend.clear();
  h->pend_cols = 0;
  h->n_seen = 0;
  h->n_launched = 0;
  h->y_started = false;
  IDSK_CUDA(h, cudaMemsetAsync(h->d_W, 0, sizeof(double) * h->l * h->n_max, h->st));
  return ID_OK;
}

id_status id_factor(id_sketch* h, int32_t* J, double* P, int32_t* k_out) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  id_status s = launch_pending(h);
  if (s != ID_OK) return s;
  if (h->n_seen == 0) return ID_ERR_STATE;
  // With want_coarse, the coarse QR of these columns (Algorithm 5) starts now
  // on the side stream, on all SMs but one, and the QR of W runs beside it in
  // one CTA; id_coarse_factor then only waits for it.
  const bool spec = h->st2 && h->coarse_spec != h->n_seen &&
                    coarse_coop_ok_ctas(h, h->nsm - 1);
  if (spec) IDSK_CUDA(h, cudaEventRecord(h->ev_sk, h->st));
  s = factor_enqueue(h, spec);
  if (s != ID_OK) return s;
  if (spec) {
    const id_status js = join_coarse(h);   // an earlier coarse QR, if any
    if (js != ID_OK) return js;
    IDSK_CUDA(h, cudaStreamWaitEvent(h->st2, h->ev_sk, 0));
    IDSK_CUDA(h, launch_coarse_coop(h, h->n_seen, h->st2, h->nsm - 1));
    IDSK_CUDA(h, cudaEventRecord(h->ev_cq, h->st2));
    h->coarse_spec = h->n_seen;
    h->cq_pending = true;
  }
  const int64_t n = h->n_seen;
  const int k = h->k;
  if ((s = copy_out(h, J, h->d_J, sizeof(int32_t) * k)) != ID_OK) return s;
  if ((s = copy_out(h, P, h->d_P, sizeof(double) * k * n)) != ID_OK) return s;
  int32_t kk = 0, dst = 0;
  IDSK_CUDA(h, cudaMemcpyAsync(&kk, h->d_kout, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaMemcpyAsync(&dst, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  if (dst) {
    h->poisoned = true;
    return ID_ERR_TIMEOUT;
  }
  if (k_out) *k_out = kk;
  return kk < k ? ID_ERR_RANK_DEFICIENT : ID_OK;
}

id_status id_factor_restricted(id_sketch* h, const int32_t* cand, int32_t ncand, int32_t* J,
                               double* P, int32_t* k_out) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  if (!cand || ncand < 1) return ID_ERR_INVALID_ARG;
  id_status s = launch_pending(h);
  if (s != ID_OK) return s;
  const int64_t n = h->n_seen;
  if (n == 0) return ID_ERR_STATE;
  if (ncand > n) return ID_ERR_INVALID_ARG;
  std::vector<int32_t> hc((size_t)ncand);
  IDSK_CUDA(h, cudaMemcpyAsync(hc.data(), cand, sizeof(int32_t) * ncand, cudaMemcpyDefault,
                               h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  {
    std::vector<int32_t> sorted(hc);
    std::sort(sorted.begin(), sorted.end());
    for (int32_t q = 0; q < ncand; ++q)
      if (sorted[q] < 0 || sorted[q] >= n || (q > 0 && sorted[q] == sorted[q - 1]))
        return ID_ERR_INVALID_ARG;   // outside the streamed columns, or repeated
  }
  const int k = h->k, l = h->l;
  IDSK_CUDA(h, cudaMemcpyAsync(h->d_cand, hc.data(), sizeof(int32_t) * ncand,
                               cudaMemcpyHostToDevice, h->st));
  IDSK_CUDA(h, launch_gather_cols(h->d_W, h->n_max, l, h->d_cand, ncand, h->d_work, h->st));
  IDSK_CUDA(h, launch_cpqr_small(h->d_work, l, ncand, ncand, k, ID_RANK_TOL_FACTOR, h->d_R,
                                 h->d_J, h->d_colpos, h->d_kout, h->st));
  IDSK_CUDA(h, launch_map_pivots(h->d_J, h->d_cand, h->d_kout, k, h->d_Jin, h->st));
  IDSK_CUDA(h, launch_fixed_solve(h->d_W, h->n_max, l, (int)n, h->d_Jin, h->d_kout, k, h->d_fq,
                                  h->d_P, h->st));
  if ((s = copy_out(h, J, h->d_Jin, sizeof(int32_t) * k)) != ID_OK) return s;
  if ((s = copy_out(h, P, h->d_P, sizeof(double) * k * n)) != ID_OK) return s;
  int32_t kk = 0, dst = 0;
  IDSK_CUDA(h, cudaMemcpyAsync(&kk, h->d_kout, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaMemcpyAsync(&dst, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  if (dst) {
    h->poisoned = true;
    return ID_ERR_TIMEOUT;
  }
  if (k_out) *k_out = kk;
  return kk < k ? ID_ERR_RANK_DEFICIENT : ID_OK;
}

id_status id_coarse_factor(id_sketch* h, int32_t* Jc, double* Pc, int32_t* k_out) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  if (!h->cfg.want_coarse) return ID_ERR_STATE;
  id_status s = launch_pending(h);
  if (s != ID_OK) return s;
  const int64_t n = h->n_seen;
  if (n == 0) return ID_ERR_STATE;
  const int k = h->k;
  if (h->coarse_spec == n) {   // started by id_factor on the side stream
    if ((s = join_coarse(h)) != ID_OK) return s;
  } else {
    if ((s = join_coarse(h)) != ID_OK) return s;
    IDSK_CUDA(h, launch_coarse_cpqr(h, n, h->st));
    h->coarse_spec = -1;
  }
  if ((s = copy_out(h, Jc, h->d_Jc, sizeof(int32_t) * k)) != ID_OK) return s;
  if ((s = copy_out(h, Pc, h->d_Pc, sizeof(double) * k * n)) != ID_OK) return s;
  int32_t kk = 0, dst = 0;
  IDSK_CUDA(h, cudaMemcpyAsync(&kk, h->d_cint + 3, sizeof(int32_t), cudaMemcpyDeviceToHost,
                               h->st));
  IDSK_CUDA(h, cudaMemcpyAsync(&dst, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  if (dst) {
    h->poisoned = true;
    return ID_ERR_TIMEOUT;
  }
  if (k_out) *k_out = kk;
  return kk < k ? ID_ERR_RANK_DEFICIENT : ID_OK;
}

id_status id_reconstruct_error(id_sketch* h, const void* d_A, int64_t lda, int64_t n,
                               const int32_t* J, const double* P, int32_t k, double* rel_fro,
                               double* rel_max) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  if (!d_A || !J || !P || lda < h->m || n < 1 || k < 1 || k > kRecKMax)
    return ID_ERR_INVALID_ARG;
  int32_t jh[kRecKMax];
  IDSK_CUDA(h, cudaMemcpyAsync(jh, J, sizeof(int32_t) * k, cudaMemcpyDefault, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  for (int u = 0; u < k; ++u)
    if (jh[u] < 0 || jh[u] >= n) return ID_ERR_INVALID_ARG;
  if ((int64_t)k * n > h->pin_cap) {
    if (h->d_Pin) cudaFree(h->d_Pin);
    h->d_Pin = nullptr;
    h->pin_cap = 0;
    Allocator al;
    al.get(&h->d_Pin, (size_t)k * n);
    if (al.st != ID_OK) return al.st;
    h->pin_cap = (int64_t)k * n;
  }
  IDSK_CUDA(h, cudaMemcpyAsync(h->d_Jin, jh, sizeof(int32_t) * k, cudaMemcpyHostToDevice, h->st));
  IDSK_CUDA(h, cudaMemcpyAsync(h->d_Pin, P, sizeof(double) * k * n, cudaMemcpyDefault, h->st));
  IDSK_CUDA(h, launch_recon_error(d_A, lda, h->m, n, h->cfg.dtype, h->d_Jin, h->d_Pin, k,
                                  h->d_part, h->rec_blocks, h->d_out3, h->d_status, h->st,
                                  h->timer_recon));
  double o[3];
  int32_t dst = 0;
  IDSK_CUDA(h, cudaMemcpyAsync(o, h->d_out3, sizeof(o), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaMemcpyAsync(&dst, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  if (dst) {
    h->poisoned = true;
    return ID_ERR_TIMEOUT;
  }
  if (rel_fro) *rel_fro = o[1] > 0.0 ? sqrt(o[0] / o[1]) : 0.0;
  if (rel_max) *rel_max = o[2];
  return ID_OK;
}

id_status id_set_mesh(id_sketch* h, const double* x, const double* y, const double* z,
                      const double period[3]) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  if (!h->cfg.want_coarse) return ID_ERR_STATE;
  if (!x || !y || !z || !period) return ID_ERR_INVALID_ARG;
  const double* c[3] = {x, y, z};
  const int n[3] = {h->cg.nx, h->cg.ny, h->cg.nz};
  const int sd[3] = {h->cg.sx, h->cg.sy, h->cg.sz};
  std::vector<idsk::AxisW> tab;
  for (int d = 0; d < 3; ++d) {
    if (!(period[d] >= 0.0) || !std::isfinite(period[d])) return ID_ERR_INVALID_ARG;
    for (int i = 0; i < n[d]; ++i) {
      if (!std::isfinite(c[d][i])) return ID_ERR_INVALID_ARG;
      if (i > 0 && !(c[d][i] > c[d][i - 1])) return ID_ERR_INVALID_ARG;   // increasing
    }
    if (period[d] > 0.0 && !(c[d][0] + period[d] > c[d][n[d] - 1])) return ID_ERR_INVALID_ARG;
    const size_t off = tab.size();
    tab.resize(off + n[d]);
    idsk::build_axis_weights(c[d], n[d], sd[d], period[d], tab.data() + off);
  }
  if (!h->d_axis) {
    Allocator al;
    al.get(&h->d_axis, tab.size());
    al.get((char**)&h->d_Sc, (size_t)h->mc * idsk::kSkelLd * h->esz);
    if (al.st != ID_OK) {
      if (h->d_axis) cudaFree(h->d_axis);
      if (h->d_Sc) cudaFree(h->d_Sc);
      h->d_axis = nullptr;
      h->d_Sc = nullptr;
      return al.st;
    }
  }
  IDSK_CUDA(h, cudaMemcpyAsync(h->d_axis, tab.data(), sizeof(idsk::AxisW) * tab.size(),
                               cudaMemcpyHostToDevice, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  h->mesh_set = true;
  return ID_OK;
}

id_status id_single_pass_lift(id_sketch* h, const int32_t* Jc, int32_t kc, void* d_S) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  if (!Jc || !d_S || kc < 1 || kc > kRecKMax) return ID_ERR_INVALID_ARG;
  id_status s = stage_coarse_skeleton(h, Jc, kc);
  if (s != ID_OK) return s;
  IDSK_CUDA(h, launch_single_pass_lift(interp_geom(h), h->m, h->cfg.dtype, kc, d_S, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  return ID_OK;
}

id_status id_single_pass_error(id_sketch* h, const void* d_A, int64_t lda, int64_t n,
                               const int32_t* Jc, const double* Pc, int32_t kc, double* rel_fro,
                               double* rel_max) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  if (!d_A || !Jc || !Pc || lda < h->m || n < 1 || kc < 1 || kc > kRecKMax)
    return ID_ERR_INVALID_ARG;
  id_status s = stage_coarse_skeleton(h, Jc, kc);
  if (s != ID_OK) return s;
  if ((int64_t)kc * n > h->pin_cap) {
    if (h->d_Pin) cudaFree(h->d_Pin);
    h->d_Pin = nullptr;
    h->pin_cap = 0;
    Allocator al;
    al.get(&h->d_Pin, (size_t)kc * n);
    if (al.st != ID_OK) return al.st;
    h->pin_cap = (int64_t)kc * n;
  }
  IDSK_CUDA(h, cudaMemcpyAsync(h->d_Pin, Pc, sizeof(double) * kc * n, cudaMemcpyDefault, h->st));
  const idsk::InterpGeom g = interp_geom(h);
  IDSK_CUDA(h, launch_recon_error(d_A, lda, h->m, n, h->cfg.dtype, h->d_Jin, h->d_Pin, kc,
                                  h->d_part, h->rec_blocks, h->d_out3, h->d_status, h->st,
                                  nullptr, &g));
  double o[3];
  int32_t dst = 0;
  IDSK_CUDA(h, cudaMemcpyAsync(o, h->d_out3, sizeof(o), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaMemcpyAsync(&dst, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
  IDSK_CUDA(h, cudaStreamSynchronize(h->st));
  if (dst) {
    h->poisoned = true;
    return ID_ERR_TIMEOUT;
  }
  if (rel_fro) *rel_fro = o[1] > 0.0 ? sqrt(o[0] / o[1]) : 0.0;
  if (rel_max) *rel_max = o[2];
  return ID_OK;
}

id_status id_sketch_get(id_sketch* h, const double** d_W, const void** d_Y, const void** d_Ac,
                        int64_t* n_seen, int64_t* m_c) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (h->poisoned) return ID_ERR_CUDA;
  id_status s = launch_pending(h);
  if (s != ID_OK) return s;
  if (d_W) *d_W = h->d_W;
  if (d_Y) *d_Y = h->d_Y;
  if (d_Ac) *d_Ac = h->d_Ac;
  if (n_seen) *n_seen = h->n_seen;
  if (m_c) *m_c = h->mc;
  return ID_OK;
}

id_status id_timing_enable(id_sketch* h, int32_t on) {
  if (!h) return ID_ERR_INVALID_ARG;
  if (on) {
    if (!h->timer_sketch) h->timer_sketch = new idsk::KernelTimer();
    if (!h->timer_recon) h->timer_recon = new idsk::KernelTimer();
  } else {
    cudaStreamSynchronize(h->st);
    delete h->timer_sketch;
    delete h->timer_recon;
    h->timer_sketch = h->timer_recon = nullptr;
  }
  return ID_OK;
}

id_status id_timing_read(id_sketch* h, int32_t which, double* total_ms, int64_t* launches) {
  if (!h || (which != 0 && which != 1) || !total_ms || !launches) return ID_ERR_INVALID_ARG;
  idsk::KernelTimer* t = which == 0 ? h->timer_sketch : h->timer_recon;
  if (!t) return ID_ERR_STATE;
  IDSK_CUDA(h, t->read(total_ms, launches));
  return ID_OK;
}

id_status id_check_wait(int32_t device, int32_t mode) {
  if (mode < 0 || mode > 3) return ID_ERR_INVALID_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    g_last_cuda_error.store((int)cudaGetLastError());
    return ID_ERR_CUDA;
  }
  cudaStream_t st = nullptr;
  int gave_up = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = idsk::run_wait_check(mode, st, &gave_up);
  if (st) cudaStreamDestroy(st);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    g_last_cuda_error.store((int)e);
    return ID_ERR_CUDA;
  }
  return gave_up ? ID_ERR_TIMEOUT : ID_OK;
}

void id_sketch_destroy(id_sketch* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  if (h->st2) {
    cudaStreamSynchronize(h->st2);
    cudaStreamDestroy(h->st2);
  }
  if (h->ev_sk) cudaEventDestroy(h->ev_sk);
  if (h->ev_cq) cudaEventDestroy(h->ev_cq);
  free_all(h);
  delete h->timer_sketch;
  delete h->timer_recon;
  delete h;
}

}  // extern "C"
