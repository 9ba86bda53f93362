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
  // Work-list form: FP32 problems whose columns start on 16-byte boundaries
  // (all of them in the usual case) share one persistent sketch launch, one
  // slab-sum launch, the batched QRs and the batched solve; the others keep
  // their own graph branch.
  std::vector<int> pers;              // problems in the work-list form
  std::vector<char> in_pers;          // per problem
  std::vector<BatchJob> jobs;         // one per sketch pass of a work-list problem
  std::vector<CUtensorMap> tmaps;     // one per job
  BatchJob* d_jobs = nullptr;
  CUtensorMap* d_tmaps = nullptr;
  BatchItem* d_items = nullptr;
  int32_t* d_order = nullptr;
  int nitems = 0;
  int items_cap = 0;
  float* d_slabs = nullptr;
  size_t slab_cap = 0;                // floats
  int* d_counter = nullptr;           // [0] the item counter, [1 + j] job j's completed items
  QrJob* d_qr = nullptr;
  int item_mb = 0;                    // autotuned work-item size (0: automatic)
  int nsm = 0;
};

namespace {

constexpr int kBatchLanes = 8;
constexpr int kBatchDrainBlocks = 8;   // row blocks between W^T flushes (work-list form)

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
  void* ptrs[] = {b->d_jobs, b->d_tmaps, b->d_items, b->d_order, b->d_slabs, b->d_counter,
                  b->d_qr};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

// ------------------------------------------------------------ work list

// A problem joins the work-list form when the tensor-core sketch takes it:
// FP32 data, at least one row block, 16-byte aligned columns.
bool work_list_ok(const id_batch_problem& p) {
  return p.dtype == ID_F32 && p.m >= 128 && ((uintptr_t)p.d_A & 15u) == 0 && (p.lda & 3) == 0;
}

// The jobs of the work-list problems (one per problem: without Y the
// tensor-core sketch takes l <= 96 in one pass), with their tensor maps; a
// problem whose tensor map cannot be built leaves the work list.
void build_jobs(id_batch* b) {
  b->pers.clear();
  b->jobs.clear();
  b->tmaps.clear();
  b->in_pers.assign(b->prob.size(), 0);
  for (size_t i = 0; i < b->prob.size(); ++i) {
    const id_batch_problem& p = b->prob[i];
    if (!work_list_ok(p)) continue;
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    if (!make_tmap_f32_2d(p.d_A, p.m, p.n, p.lda, 128, 32, &tm)) continue;
    const id_sketch* h = b->h[i];
    b->pers.push_back((int)i);
    b->in_pers[i] = 1;
    {   // all l <= 96 sketch rows in one pass (no Y)
      const int s0 = 0;
      BatchJob j;
      memset(&j, 0, sizeof(j));
      j.a.m = p.m;
      j.a.l = p.l;
      j.a.lpad = h->lpad;
      j.a.k0 = h->key0;
      j.a.k1 = h->key1;
      j.a.table = h->d_table;
      j.a.omega = h->d_omega;
      j.a.ldw = p.n;
      j.a.bf16 = p.prec == ID_SKETCH_BF16 ? 1 : 0;
      j.a.s0 = s0;
      j.ncols = p.n;
      j.np = j.a.bf16 ? 1 : 2;
      j.prob = (int)i;
      j.Wd = h->d_work + (int64_t)s0 * p.n;
      b->jobs.push_back(j);
      b->tmaps.push_back(tm);
    }
  }
}

// Work items of item_mb MB of A each (0: the work-list bytes over 16 items
// per SM, between 4 and 64 MB), whole row blocks, ordered largest first; the
// job table (with each job's item range), the items, the order and the
// slabs are uploaded.  The batch's stream must be idle (no run in flight).
id_status build_items(id_batch* b, int item_mb) {
  double tot = 0.0;
  for (const BatchJob& j : b->jobs) tot += 4.0 * (double)j.a.m * j.ncols;
  double target = (double)item_mb * (1 << 20);
  if (item_mb <= 0)
    target = std::min(64.0 * (1 << 20), std::max(4.0 * (1 << 20), tot / (16.0 * b->nsm)));
  std::vector<BatchItem> items;
  size_t slab = 0;
  for (size_t q = 0; q < b->jobs.size(); ++q) {
    BatchJob& j = b->jobs[q];
    const int64_t nrb = (j.a.m + 127) / 128;
    const double rb_bytes = 128.0 * 4.0 * j.ncols;
    const int64_t per = std::max<int64_t>(1, (int64_t)(target / rb_bytes + 0.5));
    const int64_t nct = (j.ncols + 127) / 128;
    const int64_t lw = w_width(j.a.l, false);
    j.item0 = (int32_t)items.size();
    for (int64_t r0 = 0; r0 < nrb; r0 += per) {
      BatchItem it;
      it.rb0 = r0;
      it.nrb = (int32_t)std::min(per, nrb - r0);
      it.job = (int32_t)q;
      it.slab = (int64_t)slab;
      slab += (size_t)(nct * 128 * lw);
      items.push_back(it);
    }
    j.nitem = (int32_t)items.size() - j.item0;
  }
  // jobs in order of decreasing QR work (k n l), so that the QRs which the
  // CTAs run as matrices complete overlap later items and the last matrices
  // to complete have the cheapest ones; each job's items in row order
  std::vector<int> jorder(b->jobs.size());
  std::iota(jorder.begin(), jorder.end(), 0);
  auto qr_work = [&](int q) {
    const BatchJob& j = b->jobs[q];
    return (double)b->prob[j.prob].k * j.ncols * j.a.l;
  };
  std::stable_sort(jorder.begin(), jorder.end(),
                   [&](int x, int y) { return qr_work(x) > qr_work(y); });
  std::vector<int32_t> order;
  order.reserve(items.size());
  for (int q : jorder)
    for (int32_t it = b->jobs[q].item0; it < b->jobs[q].item0 + b->jobs[q].nitem; ++it)
      order.push_back(it);
  cudaError_t e = cudaSuccess;
  if ((int)items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_order) cudaFree(b->d_order);
    b->d_items = nullptr;
    b->d_order = nullptr;
    b->items_cap = 0;
    e = cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int32_t) * items.size());
    if (e == cudaSuccess) b->items_cap = (int)items.size();
  }
  if (e == cudaSuccess && slab > b->slab_cap) {
    if (b->d_slabs) cudaFree(b->d_slabs);
    b->d_slabs = nullptr;
    b->slab_cap = 0;
    e = cudaMalloc(&b->d_slabs, sizeof(float) * slab);
    if (e == cudaSuccess) b->slab_cap = slab;
  }
  if (e == cudaSuccess && !b->d_jobs) {
    e = cudaMalloc(&b->d_jobs, sizeof(BatchJob) * b->jobs.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tmaps, sizeof(CUtensorMap) * b->tmaps.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int) * (1 + b->jobs.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_qr, sizeof(QrJob) * b->jobs.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_tmaps, b->tmaps.data(), sizeof(CUtensorMap) * b->tmaps.size(),
                     cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_jobs, b->jobs.data(), sizeof(BatchJob) * b->jobs.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_order, order.data(), sizeof(int32_t) * order.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g_last_cuda_error.store((int)e);
    b->poisoned = true;
    return e == cudaErrorMemoryAllocation ? ID_ERR_OOM : ID_ERR_CUDA;
  }
  b->nitems = (int)items.size();
  b->item_mb = item_mb;
  return ID_OK;
}

// The QR jobs of the work-list problems for these output pointers, one per
// job (in job order).
id_status upload_qr_jobs(id_batch* b, int32_t* J, double* P, int32_t* kout) {
  std::vector<QrJob> q;
  for (const BatchJob& jb : b->jobs) {
    const int i = jb.prob;
    const id_batch_problem& p = b->prob[i];
    const id_sketch* h = b->h[i];
    QrJob j;
    memset(&j, 0, sizeof(j));
    j.M = h->d_work;
    j.R = h->d_R;
    j.J = J + b->joff[i];
    j.colpos = h->d_colpos;
    j.kout = kout + i;
    j.P = P + b->poff[i];
    j.rows = p.l;
    j.n = p.n;
    j.k = p.k;
    q.push_back(j);
  }
  if (q.empty()) return ID_OK;
  const cudaError_t e = cudaMemcpy(b->d_qr, q.data(), sizeof(QrJob) * q.size(),
                                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail_cuda(b, e);
  return ID_OK;
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
  if (!b->pers.empty()) {
    // the job tables are read by the graph: no run may be in flight
    cudaError_t e = cudaStreamSynchronize(b->origin);
    if (e != cudaSuccess) return fail_cuda(b, e);
    const id_status s = upload_qr_jobs(b, J, P, kout);
    if (s != ID_OK) return s;
  }
  const int64_t l0 = g_launches.load();
  cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail_cuda(b, e);
  id_status s = ID_OK;
  e = cudaMemsetAsync(b->d_stat, 0, sizeof(int) * b->prob.size(), b->origin);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->origin);
  for (size_t q = 0; q < b->aux.size() && e == cudaSuccess; ++q)
    e = cudaStreamWaitEvent(b->aux[q], b->fork, 0);
  if (e != cudaSuccess) s = ID_ERR_CUDA;
  // the work list on the origin stream, the other problems on their branches
  if (s == ID_OK && !b->pers.empty()) {
    e = cudaMemsetAsync(b->d_counter, 0, sizeof(int) * (1 + b->jobs.size()), b->origin);
    if (e == cudaSuccess)
      e = launch_sketch_batch(b->d_jobs, b->d_tmaps, b->d_items, b->d_order, b->nitems,
                              b->d_slabs, b->d_counter, b->d_qr, ID_RANK_TOL_FACTOR, b->d_stat,
                              std::min(b->nsm, b->nitems), kBatchDrainBlocks, b->origin);
    if (e != cudaSuccess) s = ID_ERR_CUDA;
  }
  for (size_t i = 0; i < b->prob.size() && s == ID_OK; ++i)
    if (!b->in_pers[i]) s = enqueue_problem(b, (int)i, J, P, kout);
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

// A tuning candidate c: with a work list, work items of c MB of A (0:
// automatic) and one CTA per SM for the branch problems; without one, the
// branch problems' sketches on at most ceil(row blocks / c) CTAs.
id_status apply_choice(id_batch* b, int c) {
  if (b->pers.empty()) {
    apply_split(b, c);
    return ID_OK;
  }
  apply_split(b, 0);
  const cudaError_t e = cudaStreamSynchronize(b->origin);
  if (e != cudaSuccess) return fail_cuda(b, e);
  return build_items(b, c);
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
  // largest problems first, each to the least loaded worker stream (the
  // problems of the work list run on the graph's own stream)
  int nbranch = 0;
  for (int i = 0; i < count; ++i) nbranch += work_list_ok(problems[i]) ? 0 : 1;
  const int lanes = std::max(1, std::min(nbranch, kBatchLanes));
  std::vector<int> order;
  for (int i = 0; i < count; ++i)
    if (!work_list_ok(problems[i])) order.push_back(i);
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
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();   // every Omega drawn
  if (e != cudaSuccess) {
    g_last_cuda_error.store((int)e);
    release(b);
    delete b;
    return ID_ERR_CUDA;
  }
  build_jobs(b);
  if (!b->pers.empty()) {
    const id_status s = build_items(b, 0);
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

id_status id_batch_tune(id_batch* b, int32_t* J, double* P, int32_t* kout, int32_t* choice,
                        float* ms) {
  if (!b) return ID_ERR_INVALID_ARG;
  if (b->poisoned) return ID_ERR_CUDA;
  if (!J || !P || !kout || !is_device_ptr(J) || !is_device_ptr(P) || !is_device_ptr(kout))
    return ID_ERR_INVALID_ARG;
  static const int kCand[] = {0, 32, 16, 8, 4};
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
    s = apply_choice(b, kCand[c]);
    if (s == ID_OK) s = capture(b, J, P, kout);   // the work split is part of the graph
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
    // a candidate whose device waits gave up is an error, not a timing
    std::vector<int> flags(b->prob.size());
    e = cudaMemcpy(flags.data(), b->d_stat, sizeof(int) * flags.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      s = fail_cuda(b, e);
      break;
    }
    if (std::any_of(flags.begin(), flags.end(), [](int f) { return f != 0; })) {
      b->poisoned = true;
      s = ID_ERR_TIMEOUT;
      break;
    }
    if (ms) ms[c] = t;
    if (c == 0 || t < best_ms) {
      best_ms = t;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != ID_OK) return s;
  s = apply_choice(b, kCand[best]);
  if (s == ID_OK) s = capture(b, J, P, kout);
  if (s != ID_OK) return s;
  if (choice) *choice = kCand[best];
  b->ran = true;   // the outputs hold the last candidate's result
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
