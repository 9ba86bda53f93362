// Batched form of the randomized ID (Algorithm 4, Sec. 2.4): many independent
// snapshot matrices of uneven size (the column blocks of Sec. 3.3, or several
// variables and windows side by side) in one CUDA-graph launch.
//
// Each problem keeps its own sketch state (W, Omega, QR work space), created
// once.  The per-problem work -- zero W, the fused sketch of all n columns,
// the pivoted QR of W and the solve for P, the copies into the packed
// outputs -- is captured once into a graph whose parallel branches are a pool
// of worker streams; problems are dealt to the branches largest first so that
// each branch carries about the same bytes.  Later runs replay the graph: one
// launch for the whole batch, and no host round trip between problems.  Every
// device wait inside the kernels is bounded and raises the problem's status
// flag; id_batch_wait gathers those flags (copied into one array by the
// graph) with a single read.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <numeric>
#include <vector>

#include "idsk_internal.h"

using namespace idsk;

namespace idsk {
extern std::atomic<int64_t> g_launches;
extern std::atomic<int> g_last_cuda_error;
}

struct id_batch {
  std::vector<id_batch_problem> prob;
  std::vector<id_sketch*> h;
  std::vector<int> lane;              // worker stream of each problem
  std::vector<cudaStream_t> aux;      // worker streams (graph branches)
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t st = nullptr;          // the caller's stream
  cudaStream_t origin = nullptr;      // private stream the graph is captured and launched on
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;   // st -> origin -> st ordering
  std::vector<int64_t> joff, poff;    // offsets of each problem in J and P
  int* d_stat = nullptr;              // per-problem status flags, gathered by the graph
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;          // kernels per graph launch
  int32_t* cap_J = nullptr;           // output pointers the graph was captured with
  double* cap_P = nullptr;
  int32_t* cap_k = nullptr;
  bool ran = false;
  bool poisoned = false;
  int rows_per_cta = 0;               // autotuned work split of the sketches (0: one CTA per SM)
};

namespace {

constexpr int kBatchLanes = 8;

id_status fail_cuda(id_batch* b, cudaError_t e) {
  g_last_cuda_error.store((int)e);
  b->poisoned = true;
  return ID_ERR_CUDA;
}

id_status check_problem(const id_batch_problem& p) {
  if (!p.d_A || p.m < 1 || p.lda < p.m || p.n < 1 || p.n > ID_BATCH_MAX_COLS)
    return ID_ERR_INVALID_ARG;
  if (p.k < 1 || p.l < p.k || p.l > kLMaxW || p.k > p.n) return ID_ERR_INVALID_ARG;
  if (p.l > kLMax && p.dtype != ID_F32) return ID_ERR_INVALID_ARG;
  if (p.dtype != ID_F32 && p.dtype != ID_F64) return ID_ERR_INVALID_ARG;
  if (p.prec != ID_SKETCH_EXACT && p.prec != ID_SKETCH_BF16) return ID_ERR_INVALID_ARG;
  if (p.prec == ID_SKETCH_BF16 && p.dtype != ID_F32) return ID_ERR_INVALID_ARG;
  if (p.reserved != 0) return ID_ERR_INVALID_ARG;
  return ID_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void release(id_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (id_sketch* h : b->h)
    if (h) id_sketch_destroy(h);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaStream_t s : b->aux)
    if (s) cudaStreamDestroy(s);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->d_stat) cudaFree(b->d_stat);
}

// Enqueue problem i on its worker stream (called while capturing).
id_status enqueue_problem(id_batch* b, int i, int32_t* J, double* P, int32_t* kout) {
  const id_batch_problem& p = b->prob[i];
  id_sketch* h = b->h[i];
  id_status s = id_sketch_reset(h);
  if (s == ID_OK) s = id_sketch_stream_columns(h, p.d_A, p.lda, p.n);
  if (s == ID_OK) s = factor_enqueue(h);
  if (s != ID_OK) return s;
  cudaError_t e = cudaMemcpyAsync(J + b->joff[i], h->d_J, sizeof(int32_t) * p.k,
                                  cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P + b->poff[i], h->d_P, sizeof(double) * p.k * p.n,
                        cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(kout + i, h->d_kout, sizeof(int32_t), cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_stat + i, h->d_status, sizeof(int), cudaMemcpyDeviceToDevice, h->st);
  if (e != cudaSuccess) {
    g_last_cuda_error.store((int)e);
    return ID_ERR_CUDA;
  }
  return ID_OK;
}

// Capture the whole batch into b->exec.  The capture is always ended (and
// every worker stream joined back) so that the streams stay usable after an
// error.
id_status capture(id_batch* b, int32_t* J, double* P, int32_t* kout) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  const int64_t l0 = g_launches.load();
  cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail_cuda(b, e);
  id_status s = ID_OK;
  e = cudaEventRecord(b->fork, b->origin);
  for (size_t q = 0; q < b->aux.size() && e == cudaSuccess; ++q)
    e = cudaStreamWaitEvent(b->aux[q], b->fork, 0);
  if (e != cudaSuccess) s = ID_ERR_CUDA;
  for (size_t i = 0; i < b->prob.size() && s == ID_OK; ++i)
    s = enqueue_problem(b, (int)i, J, P, kout);
  for (size_t q = 0; q < b->aux.size(); ++q) {
    cudaEventRecord(b->join[q], b->aux[q]);
    cudaStreamWaitEvent(b->origin, b->join[q], 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(b->origin, &graph);
  const int64_t kernels = g_launches.load() - l0;
  count_launches(-kernels);   // counted again per graph launch
  if (s == ID_OK && ee != cudaSuccess) {
    s = ID_ERR_CUDA;
    e = ee;
  }
  if (s == ID_OK) {
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (e != cudaSuccess) s = ID_ERR_CUDA;
  }
  if (graph) cudaGraphDestroy(graph);
  if (s != ID_OK) {
    cudaGetLastError();
    if (e != cudaSuccess) g_last_cuda_error.store((int)e);
    b->poisoned = true;
    return s;
  }
  b->graph_kernels = kernels;
  b->cap_J = J;
  b->cap_P = P;
  b->cap_k = kout;
  return ID_OK;
}

// The sketch of problem i runs on at most ceil(row blocks / rows_per_cta)
// CTAs (rows_per_cta = 0: one per SM, the persistent grid of a single
// problem); smaller grids let the sketches of several small problems share
// the GPU instead of each spreading a few row blocks over every SM.
void apply_split(id_batch* b, int rows_per_cta) {
  for (size_t i = 0; i < b->prob.size(); ++i) {
    const int64_t nrb = (b->prob[i].m + 127) / 128;
    b->h[i]->grid_cap =
        rows_per_cta > 0 ? (int)std::max<int64_t>(1, (nrb + rows_per_cta - 1) / rows_per_cta) : 0;
  }
  b->rows_per_cta = rows_per_cta;
}

}  // namespace

extern "C" {

id_status id_batch_create(const id_batch_problem* problems, int32_t count, void* cuda_stream,
                          id_batch** out) {
  if (!out) return ID_ERR_INVALID_ARG;
  *out = nullptr;
  if (!problems || count < 1 || count > ID_BATCH_MAX_PROBLEMS) return ID_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (check_problem(problems[i]) != ID_OK) return ID_ERR_INVALID_ARG;
  id_batch* b = new (std::nothrow) id_batch();
  if (!b) return ID_ERR_OOM;
  b->prob.assign(problems, problems + count);
  b->st = (cudaStream_t)cuda_stream;
  b->joff.resize(count);
  b->poff.resize(count);
  int64_t jo = 0, po = 0;
  for (int i = 0; i < count; ++i) {
    b->joff[i] = jo;
    b->poff[i] = po;
    jo += problems[i].k;
    po += (int64_t)problems[i].k * problems[i].n;
  }
  // largest problems first, each to the least loaded worker stream
  const int lanes = std::min(count, kBatchLanes);
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  auto bytes = [&](int i) {
    return (double)problems[i].m * problems[i].n * (problems[i].dtype == ID_F64 ? 8.0 : 4.0);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return bytes(a) > bytes(c); });
  std::vector<double> load(lanes, 0.0);
  b->lane.assign(count, 0);
  for (int i : order) {
    const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lane[i] = q;
    load[q] += bytes(i);
  }
  cudaError_t e = cudaSuccess;
  b->aux.assign(lanes, nullptr);
  b->join.assign(lanes, nullptr);
  for (int q = 0; q < lanes && e == cudaSuccess; ++q) {
    e = cudaStreamCreateWithFlags(&b->aux[q], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[q], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_stat, sizeof(int) * count);
  if (e == cudaSuccess) e = cudaMemset(b->d_stat, 0, sizeof(int) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g_last_cuda_error.store((int)e);
    release(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? ID_ERR_OOM : ID_ERR_CUDA;
  }
  b->h.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    const id_batch_problem& p = problems[i];
    id_config c;
    memset(&c, 0, sizeof(c));
    c.m = p.m;
    c.n_max = p.n;
    c.k = p.k;
    c.l = p.l;
    c.seed = p.seed;
    c.dtype = p.dtype;
    c.prec = p.prec;
    const id_status s = id_sketch_create(&c, b->aux[b->lane[i]], &b->h[i]);
    if (s != ID_OK) {
      release(b);
      delete b;
      return s;
    }
  }
  *out = b;
  return ID_OK;
}

id_status id_batch_run(id_batch* b, int32_t* J, double* P, int32_t* kout) {
  if (!b) return ID_ERR_INVALID_ARG;
  if (b->poisoned) return ID_ERR_CUDA;
  if (!J || !P || !kout) return ID_ERR_INVALID_ARG;
  if (J != b->cap_J || P != b->cap_P || kout != b->cap_k || !b->exec) {
    if (!is_device_ptr(J) || !is_device_ptr(P) || !is_device_ptr(kout)) return ID_ERR_INVALID_ARG;
    const id_status s = capture(b, J, P, kout);
    if (s != ID_OK) return s;
  }
  // in stream order with the caller's stream: st -> graph on origin -> st
  cudaError_t e = cudaEventRecord(b->ev_in, b->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev_in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->origin);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->origin);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->ev_out, 0);
  if (e != cudaSuccess) return fail_cuda(b, e);
  count_launches(b->graph_kernels);
  b->ran = true;
  return ID_OK;
}

id_status id_batch_wait(id_batch* b, int32_t* kout_host) {
  if (!b) return ID_ERR_INVALID_ARG;
  if (b->poisoned) return ID_ERR_CUDA;
  if (!b->ran) return ID_ERR_STATE;
  const int count = (int)b->prob.size();
  std::vector<int> st(count), ko(count);
  cudaError_t e = cudaMemcpyAsync(st.data(), b->d_stat, sizeof(int) * count,
                                  cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ko.data(), b->cap_k, sizeof(int) * count, cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return fail_cuda(b, e);
  for (int i = 0; i < count; ++i)
    if (st[i]) {
      b->poisoned = true;
      return ID_ERR_TIMEOUT;
    }
  if (kout_host) std::copy(ko.begin(), ko.end(), kout_host);
  for (int i = 0; i < count; ++i)
    if (ko[i] < b->prob[i].k) return ID_ERR_RANK_DEFICIENT;
  return ID_OK;
}

id_status id_batch_tune(id_batch* b, int32_t* J, double* P, int32_t* kout,
                         int32_t* rows_per_cta, float* ms) {
  if (!b) return ID_ERR_INVALID_ARG;
  if (b->poisoned) return ID_ERR_CUDA;
  if (!J || !P || !kout || !is_device_ptr(J) || !is_device_ptr(P) || !is_device_ptr(kout))
    return ID_ERR_INVALID_ARG;
  static const int kCand[] = {0, 64, 32, 16, 8};
  constexpr int kNC = (int)(sizeof(kCand) / sizeof(kCand[0]));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail_cuda(b, e);
  }
  int best = 0;
  float best_ms = 0.f;
  id_status s = ID_OK;
  for (int c = 0; c < kNC && s == ID_OK; ++c) {
    apply_split(b, kCand[c]);
    s = capture(b, J, P, kout);   // the grid sizes are part of the graph
    if (s != ID_OK) break;
    // one replay to warm up, then three timed replays on the graph's stream
    e = cudaGraphLaunch(b->exec, b->origin);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->origin);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->exec, b->origin);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->origin);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) {
      s = fail_cuda(b, e);
      break;
    }
    t /= 3.f;
    if (ms) ms[c] = t;
    if (c == 0 || t < best_ms) {
      best_ms = t;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != ID_OK) return s;
  apply_split(b, kCand[best]);
  s = capture(b, J, P, kout);
  if (s != ID_OK) return s;
  if (rows_per_cta) *rows_per_cta = kCand[best];
  return ID_OK;
}

void id_batch_destroy(id_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  if (b->origin) cudaStreamSynchronize(b->origin);
  release(b);
  delete b;
}

}  // extern "C"
