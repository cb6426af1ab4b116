// ots_batch.cu -- host side of the batch API (ots_batch_* in include/ots.h).
//
// A batch owns one device pool, a table of slots (BatchInst + BatchCtl on the device), the
// list of work items of the resident instances, and one captured CUDA graph of
// ticks_per_launch tick kernels followed by a copy of the slot states to pinned host
// memory.  Host work between launches: admit instances (build the state graph on the host,
// carve its memory from the pool, upload; all on the batch stream, so it is ordered after
// every launch that could still touch the reused memory), notice finished instances from
// the copied slot states, and rebuild the item list when the set of running instances
// changed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ots.h"
#include "ots_batch.cuh"
#include "ots_internal.h"

namespace ots {
cudaError_t batch_tick_grid(int *grid);
cudaError_t launch_batch_tick(const TickArgs &ta, int grid, cudaStream_t s);
}  // namespace ots

using namespace ots;
using namespace ots_host;

namespace ots_host {

// First-fit sub-allocator over one device range (256-byte granules), thread-safe.
struct Pool {
  char *base = nullptr;
  size_t size = 0;
  size_t used = 0;
  std::map<size_t, size_t> free_;   // offset -> bytes
  std::map<size_t, size_t> live_;   // offset -> bytes
  std::mutex mu;

  void init(void *b, size_t n) {
    base = (char *)b;
    size = n;
    free_.clear();
    live_.clear();
    used = 0;
    if (n) free_[0] = n;
  }
  void *alloc(size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 1), 256);
    std::lock_guard<std::mutex> lock(mu);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      live_[off] = bytes;
      used += bytes;
      return base + off;
    }
    return nullptr;
  }
  void release(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(mu);
    const size_t off = (size_t)((char *)p - base);
    auto it = live_.find(off);
    if (it == live_.end()) return;
    size_t o = off, len = it->second;
    live_.erase(it);
    used -= len;
    auto nx = free_.lower_bound(o);
    if (nx != free_.end() && o + len == nx->first) { len += nx->second; free_.erase(nx); }
    auto pv = free_.lower_bound(o);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second == o) { o = pv->first; len += pv->second; free_.erase(pv); }
    }
    free_[o] = len;
  }
  size_t largest_free() {
    std::lock_guard<std::mutex> lock(mu);
    size_t m = 0;
    for (auto &kv : free_) m = std::max(m, kv.second);
    return m;
  }
};

void *pool_alloc_cb(size_t bytes, void *ctx) { return ((Pool *)ctx)->alloc(bytes); }
void pool_free_cb(void *p, void *ctx) { ((Pool *)ctx)->release(p); }

}  // namespace ots_host

namespace {

enum class SlotState { Free, Running, Final };

struct Slot {
  SlotState state = SlotState::Free;
  ots_problem *p = nullptr;
  int32_t id = -1;
  int n_items = 0;
  double tol = 1e-6;
  double timeout_ms = 0.0;
  bool stop_sent = false;
  std::chrono::steady_clock::time_point t_add, t_done;
  BatchCtl final_ctl{};
};

ots_status status_of_slot(int s) {
  switch (s) {
    case kSlotConverged: return OTS_OK;
    case kSlotNotConverged: return OTS_ERR_NOT_CONVERGED;
    case kSlotInfeasible: return OTS_ERR_INFEASIBLE;
    case kSlotNumeric: return OTS_ERR_NUMERIC;
    case kSlotStopped: return OTS_ERR_TIMEOUT;
    default: return OTS_PENDING;
  }
}

bool is_final(int s) { return s >= kSlotConverged; }

int pow2_at_least(int q) {
  int g = 1;
  while (g < q) g <<= 1;
  return g;
}

// Class of a commodity count: 0 for L <= 4, 1 for L <= 8, ..., 6 for L <= 256.
int l_class(int L) {
  int c = 0, cap = 4;
  while (cap < L) { cap <<= 1; ++c; }
  return c;
}
constexpr int kLClasses = 7;

// Default mapping: C = 1 while one warp covers the row, then 2 chunks per thread.
void default_mapping(int L, int &G, int &C) {
  const int q = (L + 3) / 4;
  if (q <= 32) { G = pow2_at_least(q); C = 1; }
  else { G = 32; C = 2; }
}

}  // namespace

struct ots_batch {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ots_alloc_fn alloc = nullptr;
  ots_free_fn free_fn = nullptr;
  void *actx = nullptr;
  void *pool_mem = nullptr;
  Pool pool;

  int max_slots = 0, max_items = 0, ticks_per_launch = 32, grid = 0;
  BatchInst *d_inst = nullptr;
  BatchCtl *d_ctl = nullptr;
  int2 *d_items = nullptr;
  int *d_n_items = nullptr;
  BatchInst *h_inst = nullptr;       // pinned staging, one per slot
  BatchCtl *h_ctl_init = nullptr;    // pinned staging, one per slot
  BatchCtl *h_ctl = nullptr;         // pinned copy of d_ctl after every launch
  int2 *h_items = nullptr;           // pinned staging of the item list
  int *h_n_items = nullptr;
  int *h_stop = nullptr;             // pinned constant kSlotStopped
  cudaGraphExec_t exec = nullptr;

  std::vector<Slot> slots;
  std::map<int32_t, int> id_slot;
  int32_t next_id = 0;
  bool items_dirty = true;
  int n_items_list = 0;
  int map_G[kLClasses], map_C[kLClasses];
  bool tuned = false;
  long long launches = 0, ticks = 0, h2d = 0, d2h = 0;
};

namespace {

void release_device(ots_batch *b) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  for (auto &s : b->slots)
    if (s.p) { ots_destroy_problem(s.p); s.p = nullptr; }
  void *dev_ptrs[] = {b->d_inst, b->d_ctl, b->d_items, b->d_n_items};
  for (void *p : dev_ptrs)
    if (p) cudaFree(p);
  void *host_ptrs[] = {b->h_inst, b->h_ctl_init, b->h_ctl, b->h_items, b->h_n_items, b->h_stop};
  for (void *p : host_ptrs)
    if (p) cudaFreeHost(p);
  if (b->pool_mem) {
    if (b->free_fn) b->free_fn(b->pool_mem, b->actx);
    else cudaFree(b->pool_mem);
  }
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

ots_status capture_graph(ots_batch *b) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  TickArgs ta{};
  ta.inst = b->d_inst;
  ta.ctl = b->d_ctl;
  ta.items = b->d_items;
  ta.n_items = b->d_n_items;
  cudaGraph_t g = nullptr;
  OTS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < b->ticks_per_launch && e == cudaSuccess; ++k) e = launch_batch_tick(ta, b->grid, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl) * b->max_slots, cudaMemcpyDeviceToHost, b->stream);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(OTS_ERR_CUDA, "tick graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { b->exec = nullptr; return fail(OTS_ERR_CUDA, "tick graph instantiate: %s", cudaGetErrorString(e)); }
  return OTS_OK;
}

// Rounds per item for the current load: items of one round while the running instances
// have few node rows in total (keeps every SM busy in the tail of a batch), up to 8 rounds
// when they have many (fewer, longer items).
int choose_rounds(const ots_batch *b) {
  long long rows = 0;
  for (int s = 0; s < b->max_slots; ++s) {
    const Slot &sl = b->slots[s];
    if (sl.state != SlotState::Running) continue;
    const BatchInst &I = b->h_inst[s];
    rows += (I.V + I.npb - 1) / I.npb;
  }
  const long long r = rows / (4LL * std::max(b->grid, 1));
  return (int)std::max(1LL, std::min(8LL, r));
}

// Rebuild and upload the item list of the running instances (slot order, items in order),
// after re-deriving the items of every running instance for the current rounds per item.
ots_status upload_items(ots_batch *b) {
  const int R = choose_rounds(b);
  for (int s = 0; s < b->max_slots; ++s) {
    Slot &sl = b->slots[s];
    if (sl.state != SlotState::Running) continue;
    BatchInst &I = b->h_inst[s];
    if (I.rounds == R) continue;
    I.rounds = R;
    I.npi = R * I.npb;
    I.n_items = (I.V + I.npi - 1) / I.npi;
    sl.n_items = I.n_items;
    OTS_CUDA(cudaMemcpyAsync(b->d_inst + s, &I, sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
    b->h2d += (long long)sizeof(BatchInst);
  }
  int n = 0;
  for (int s = 0; s < b->max_slots; ++s) {
    const Slot &sl = b->slots[s];
    if (sl.state != SlotState::Running) continue;
    if (n + sl.n_items > b->max_items) return fail(OTS_ERR_OOM, "item list full (%d items)", b->max_items);
    for (int k = 0; k < sl.n_items; ++k) b->h_items[n++] = make_int2(s, k);
  }
  *b->h_n_items = n;
  if (n) OTS_CUDA(cudaMemcpyAsync(b->d_items, b->h_items, sizeof(int2) * n, cudaMemcpyHostToDevice, b->stream));
  OTS_CUDA(cudaMemcpyAsync(b->d_n_items, b->h_n_items, sizeof(int), cudaMemcpyHostToDevice, b->stream));
  b->h2d += (long long)(sizeof(int2) * n + sizeof(int));
  b->n_items_list = n;
  b->items_dirty = false;
  return OTS_OK;
}

Slot *find_slot(ots_batch *b, int32_t id) {
  auto it = b->id_slot.find(id);
  if (it == b->id_slot.end()) return nullptr;
  return &b->slots[it->second];
}

BndSide side_of(const Boundary &bd) {
  BndSide s{};
  s.n_seg = bd.n_seg;
  s.n_tri = bd.n;
  s.seg_ptr = bd.d_seg_ptr; s.seg_node = bd.d_seg_node; s.seg_l = bd.d_seg_l;
  s.tri_other = bd.d_tri_other; s.tri_l = bd.d_tri_l;
  s.tri_R = bd.d_tri_R; s.tri_logR = bd.d_tri_logR;
  s.tri_logU = bd.d_tri_logU; s.tri_flow = bd.d_flow;
  return s;
}

}  // namespace

extern "C" {

ots_status ots_default_batch_desc(ots_batch_desc *d) {
  if (!d) return fail(OTS_ERR_INVALID_ARG, "desc is NULL");
  std::memset(d, 0, sizeof(*d));
  d->pool_bytes = (int64_t)4 << 30;
  d->max_instances = 256;
  d->max_items = 1 << 20;
  d->ticks_per_launch = 32;
  return OTS_OK;
}

ots_status ots_batch_create(const ots_batch_desc *d, ots_batch **out) {
  clear_error();
  if (!d || !out) return fail(OTS_ERR_INVALID_ARG, "desc or out is NULL");
  *out = nullptr;
  if (d->pool_bytes <= 0 || d->max_instances < 1 || d->max_items < 0 || d->ticks_per_launch < 0)
    return fail(OTS_ERR_INVALID_ARG, "bad batch sizes");
  if ((d->alloc == nullptr) != (d->free_fn == nullptr)) return fail(OTS_ERR_INVALID_ARG, "alloc and free_fn go together");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(OTS_ERR_CUDA, "no CUDA device");
  if (d->device < 0 || d->device >= ndev) return fail(OTS_ERR_INVALID_ARG, "device %d out of range", d->device);
  ots_batch *b = new (std::nothrow) ots_batch();
  if (!b) return fail(OTS_ERR_OOM, "host allocation failed");
  DeviceGuard guard(d->device);
  auto bail = [&](ots_status s) { release_device(b); delete b; return s; };
  b->dev = d->device;
  b->alloc = d->alloc;
  b->free_fn = d->free_fn;
  b->actx = d->alloc_ctx;
  b->max_slots = d->max_instances;
  b->max_items = d->max_items ? d->max_items : (1 << 20);
  b->ticks_per_launch = d->ticks_per_launch ? d->ticks_per_launch : 32;
  b->slots.resize(b->max_slots);
  for (int c = 0; c < kLClasses; ++c) default_mapping(4 << c, b->map_G[c], b->map_C[c]);
  if (d->stream) {
    b->stream = (cudaStream_t)d->stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(OTS_ERR_CUDA, "stream creation failed"));
    b->own_stream = true;
  }
  const size_t pool_bytes = (size_t)d->pool_bytes;
  b->pool_mem = b->alloc ? b->alloc(pool_bytes, b->actx) : nullptr;
  if (!b->alloc && cudaMalloc(&b->pool_mem, pool_bytes) != cudaSuccess) b->pool_mem = nullptr;
  if (!b->pool_mem) return bail(fail(OTS_ERR_OOM, "device pool of %zu bytes", pool_bytes));
  b->pool.init(b->pool_mem, pool_bytes);
  const size_t ns = b->max_slots, ni = b->max_items;
  if (cudaMalloc(&b->d_inst, sizeof(BatchInst) * ns) != cudaSuccess ||
      cudaMalloc(&b->d_ctl, sizeof(BatchCtl) * ns) != cudaSuccess ||
      cudaMalloc(&b->d_items, sizeof(int2) * ni) != cudaSuccess ||
      cudaMalloc(&b->d_n_items, sizeof(int)) != cudaSuccess)
    return bail(fail(OTS_ERR_OOM, "batch tables"));
  if (cudaMallocHost(&b->h_inst, sizeof(BatchInst) * ns) != cudaSuccess ||
      cudaMallocHost(&b->h_ctl_init, sizeof(BatchCtl) * ns) != cudaSuccess ||
      cudaMallocHost(&b->h_ctl, sizeof(BatchCtl) * ns) != cudaSuccess ||
      cudaMallocHost(&b->h_items, sizeof(int2) * ni) != cudaSuccess ||
      cudaMallocHost(&b->h_n_items, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&b->h_stop, sizeof(int)) != cudaSuccess)
    return bail(fail(OTS_ERR_OOM, "pinned batch tables"));
  *b->h_stop = kSlotStopped;
  *b->h_n_items = 0;
  std::memset(b->h_ctl, 0, sizeof(BatchCtl) * ns);
  if (cudaMemsetAsync(b->d_ctl, 0, sizeof(BatchCtl) * ns, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_inst, 0, sizeof(BatchInst) * ns, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_n_items, 0, sizeof(int), b->stream) != cudaSuccess)
    return bail(fail(OTS_ERR_CUDA, "batch table init"));
  if (batch_tick_grid(&b->grid) != cudaSuccess) return bail(fail(OTS_ERR_CUDA, "tick kernel occupancy"));
  ots_status st = capture_graph(b);
  if (st) return bail(st);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bail(fail(OTS_ERR_CUDA, "batch init sync"));
  *out = b;
  return OTS_OK;
}

void ots_batch_destroy(ots_batch *b) {
  if (!b) return;
  DeviceGuard guard(b->dev);
  if (b->stream) cudaStreamSynchronize(b->stream);
  release_device(b);
  delete b;
}

ots_status ots_batch_mapping(const ots_batch *b, int32_t L, int32_t *G, int32_t *C) {
  if (!b || !G || !C) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  if (L < 1 || L > 256) return fail(OTS_ERR_INVALID_ARG, "batched instances take 1 <= L <= 256");
  const int c = l_class(L);
  *G = b->map_G[c];
  *C = b->map_C[c];
  return OTS_OK;
}

ots_status ots_batch_add(ots_batch *b, const ots_problem_desc *desc, const ots_solve_opts *opts, int32_t *id) {
  clear_error();
  if (!b || !desc || !id) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  *id = -1;
  if (batch_free_slots(b) == 0) return fail(OTS_ERR_OOM, "no free slot (%d resident)", b->max_slots);
  DeviceGuard guard(b->dev);
  ots_problem *p = nullptr;
  ots_status st = batch_prepare(b, desc, b->stream, &p);
  if (st) return st;
  st = batch_admit(b, p, opts, id);
  if (st) ots_destroy_problem(p);
  return st;
}

}  // extern "C"

// Host build and upload of a batch member (its mapping from the batch's table, its memory
// from the pool, uploads on `upload_stream`).  Touches no batch table, so builder threads may
// call it while the driver thread runs the batch; the caller synchronises upload_stream
// before batch_admit when it is not the batch stream.
ots_status ots_host::batch_prepare(ots_batch *b, const ots_problem_desc *desc, cudaStream_t upload_stream,
                                   ots_problem **out) {
  *out = nullptr;
  if (desc->L < 1 || desc->L > 256) return fail(OTS_ERR_INVALID_ARG, "batched instances take 1 <= L <= 256");
  if (desc->commodity_cost || desc->commodity_capacity)
    return fail(OTS_ERR_INVALID_ARG, "batched instances take commodity-independent costs and capacities");
  int G = 0, C = 0;
  ots_batch_mapping(b, desc->L, &G, &C);
  ots_problem_desc d = *desc;
  d.device = b->dev;
  d.stream = upload_stream;
  d.alloc = pool_alloc_cb;
  d.free_fn = pool_free_cb;
  d.alloc_ctx = &b->pool;
  CreateOpts co;
  co.member = true;
  co.G = G;
  co.C = C;
  ots_problem *p = nullptr;
  ots_status st = create_problem_impl(&d, co, &p);
  if (st) return st;
  p->stream = b->stream;                       // all later work of the member is on the batch stream
  *out = p;
  return OTS_OK;
}

Pool *ots_host::batch_pool(ots_batch *b) { return &b->pool; }

int ots_host::batch_free_slots(const ots_batch *b) {
  int n = 0;
  for (auto &s : b->slots) n += s.state == SlotState::Free;
  return n;
}

// Put a prepared member into a free slot (driver thread only); the batch owns p afterwards.
ots_status ots_host::batch_admit(ots_batch *b, ots_problem *p, const ots_solve_opts *opts, int32_t *id) {
  ots_solve_opts o;
  ots_default_solve_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iters < 1) return fail(OTS_ERR_INVALID_ARG, "bad solve options");
  int s = -1;
  for (int k = 0; k < b->max_slots; ++k)
    if (b->slots[k].state == SlotState::Free) { s = k; break; }
  if (s < 0) return fail(OTS_ERR_OOM, "no free slot (%d resident)", b->max_slots);
  const int G = p->G, C = p->C;
  const int npb = kTickBlock / G;
  // one round per item to start with; upload_items re-derives the rounds for the load
  const int rounds = 1;
  const int npi = npb;
  const int n_items = (p->V + npi - 1) / npi;
  if (b->n_items_list + n_items > b->max_items) return fail(OTS_ERR_OOM, "item list full (%d items)", b->max_items);
  DeviceGuard guard(b->dev);

  BatchInst &I = b->h_inst[s];
  std::memset(&I, 0, sizeof(I));
  I.V = p->V; I.S = p->S; I.T = p->T; I.Lp = p->Lp; I.G = G; I.C = C;
  I.n_items = n_items; I.npb = npb; I.rounds = rounds; I.npi = npi;
  I.qs = p->qs;
  I.mass = p->mass; I.eps = p->eps; I.tol = o.tol;
  I.stage_tol = o.eps_stage_tol > 0.0 ? o.eps_stage_tol : 1e-4;
  I.max_passes = o.max_iters;
  I.kl_stride = p->tv ? p->S : 0;
  I.cap_stride = p->cv ? p->S : 0;
  I.in_ptr = p->d_in_ptr; I.in_state = p->d_in_state; I.in_nbr = p->d_in_nbr;
  I.out_ptr = p->d_out_ptr; I.out_state = p->d_out_state; I.out_nbr = p->d_out_nbr;
  I.kl_hi = p->d_kl_hi; I.kl_lo = p->d_kl_lo; I.logd_hi = p->d_logd_hi; I.logd_lo = p->d_logd_lo;
  I.cap = p->d_cap;
  I.lu = p->d_logu; I.w_hi = p->d_w_hi; I.w_lo = p->d_w_lo; I.flow = p->d_flow;
  I.a0_hi = p->d_a_hi[0]; I.a1_hi = p->d_a_hi[1]; I.a2_hi = p->d_a_hi[2];
  I.a0_lo = p->d_a_lo[0]; I.a1_lo = p->d_a_lo[1]; I.a2_lo = p->d_a_lo[2];
  I.b_hi = p->d_b_hi; I.b_lo = p->d_b_lo;
  I.src = side_of(p->src);
  I.snk = side_of(p->snk);
  I.partials = p->d_partials;
  BatchCtl &c = b->h_ctl_init[s];
  std::memset(&c, 0, sizeof(c));
  c.status = kSlotRunning;
  // epsilon continuation in the batch: stages at eps 2^k, ..., 2 eps, eps (k from eps_start / eps)
  if (o.eps_start > p->eps && std::isfinite(o.eps_start))
    c.shift = std::min(16, std::max(1, (int)std::lround(std::log2(o.eps_start / p->eps))));
  OTS_CUDA(cudaMemcpyAsync(b->d_inst + s, &I, sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
  OTS_CUDA(cudaMemcpyAsync(b->d_ctl + s, &c, sizeof(BatchCtl), cudaMemcpyHostToDevice, b->stream));
  b->h2d += (long long)(sizeof(BatchInst) + sizeof(BatchCtl)) + p->h2d_bytes;
  Slot &sl = b->slots[s];
  sl = Slot{};
  sl.state = SlotState::Running;
  sl.p = p;
  sl.id = b->next_id++;
  sl.n_items = n_items;
  sl.tol = o.tol;
  sl.timeout_ms = o.timeout_ms;
  sl.t_add = std::chrono::steady_clock::now();
  b->h_ctl[s] = c;
  b->id_slot[sl.id] = s;
  b->n_items_list += n_items;
  b->items_dirty = true;
  *id = sl.id;
  return OTS_OK;
}

extern "C" {

ots_status ots_batch_run(ots_batch *b, int32_t max_launches, int32_t *n_running) {
  clear_error();
  if (!b || max_launches < 0) return fail(OTS_ERR_INVALID_ARG, "bad arguments");
  DeviceGuard guard(b->dev);
  auto count_running = [&]() {
    int n = 0;
    for (auto &s : b->slots) n += s.state == SlotState::Running;
    return n;
  };
  int running = count_running();
  for (int k = 0; k < max_launches && running > 0; ++k) {
    if (b->items_dirty) {
      ots_status st = upload_items(b);
      if (st) return st;
    }
    OTS_CUDA(cudaGraphLaunch(b->exec, b->stream));
    OTS_CUDA(cudaStreamSynchronize(b->stream));
    b->launches += 1;
    b->ticks += b->ticks_per_launch;
    b->d2h += (long long)sizeof(BatchCtl) * b->max_slots;
    const auto now = std::chrono::steady_clock::now();
    for (int s = 0; s < b->max_slots; ++s) {
      Slot &sl = b->slots[s];
      if (sl.state != SlotState::Running) continue;
      const BatchCtl &c = b->h_ctl[s];
      if (is_final(c.status)) {
        sl.state = SlotState::Final;
        sl.t_done = now;
        sl.final_ctl = c;
        b->n_items_list -= sl.n_items;
        b->items_dirty = true;
        continue;
      }
      if (sl.timeout_ms > 0 && !sl.stop_sent &&
          std::chrono::duration<double, std::milli>(now - sl.t_add).count() > sl.timeout_ms) {
        // stream-ordered after every launch so far: the next tick sees a final status
        OTS_CUDA(cudaMemcpyAsync(&b->d_ctl[s].status, b->h_stop, sizeof(int), cudaMemcpyHostToDevice, b->stream));
        sl.stop_sent = true;
      }
    }
    running = count_running();
  }
  if (n_running) *n_running = running;
  return OTS_OK;
}

ots_status ots_batch_status(ots_batch *b, int32_t id, ots_solve_report *rep) {
  if (!b) return fail(OTS_ERR_INVALID_ARG, "batch is NULL");
  Slot *sl = find_slot(b, id);
  if (!sl) return fail(OTS_ERR_INVALID_ARG, "unknown batch instance %d", id);
  if (sl->state != SlotState::Final) {
    if (rep) {
      std::memset(rep, 0, sizeof(*rep));
      rep->status = OTS_PENDING;
    }
    return OTS_PENDING;
  }
  const BatchCtl &c = sl->final_ctl;
  const ots_status st = status_of_slot(c.status);
  if (rep) {
    rep->iterations = c.passes;
    rep->src_residual = c.report.src_resid_rel;
    rep->cap_violation = c.report.cap_viol_rel;
    rep->dual_objective = c.report.dual_objective;
    rep->seconds = std::chrono::duration<double>(sl->t_done - sl->t_add).count();
    rep->status = st;
  }
  return st;
}

ots_status ots_batch_get_flows(ots_batch *b, int32_t id, int32_t t_begin, int32_t t_end, double *out) {
  clear_error();
  if (!b || !out) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  Slot *sl = find_slot(b, id);
  if (!sl) return fail(OTS_ERR_INVALID_ARG, "unknown batch instance %d", id);
  if (sl->state != SlotState::Final) return OTS_PENDING;
  const int fs = sl->final_ctl.status;
  if (fs != kSlotConverged && fs != kSlotNotConverged)
    return fail(status_of_slot(fs), "instance finished without flows (%s)", ots_status_string(status_of_slot(fs)));
  ots_problem *p = sl->p;
  if (t_begin < 1 || t_end > p->T + 1 || t_begin >= t_end) return fail(OTS_ERR_INVALID_ARG, "bad t range");
  DeviceGuard guard(b->dev);
  const size_t S = p->S;
  std::vector<double> sf(p->src.n), zf(p->snk.n);
  const int t0 = std::max(t_begin, 2), t1 = std::min(t_end, p->T);   // interior rows, one copy
  if (t0 < t1) {
    OTS_CUDA(cudaMemcpyAsync(out + (size_t)(t0 - t_begin) * S, p->d_flow + (size_t)t0 * S,
                             sizeof(double) * S * (t1 - t0), cudaMemcpyDeviceToHost, b->stream));
    b->d2h += (long long)(sizeof(double) * S * (t1 - t0));
  }
  if (p->src.n) OTS_CUDA(cudaMemcpyAsync(sf.data(), p->src.d_flow, sizeof(double) * p->src.n, cudaMemcpyDeviceToHost, b->stream));
  if (p->snk.n) OTS_CUDA(cudaMemcpyAsync(zf.data(), p->snk.d_flow, sizeof(double) * p->snk.n, cudaMemcpyDeviceToHost, b->stream));
  b->d2h += (long long)(sizeof(double) * (p->src.n + p->snk.n));
  OTS_CUDA(cudaStreamSynchronize(b->stream));
  for (int t = t_begin; t < t_end; ++t) {
    if (t != 1 && t != p->T) continue;
    double *row = out + (size_t)(t - t_begin) * S;
    std::fill(row, row + S, 0.0);
    const Boundary &bd = t == 1 ? p->src : p->snk;
    const std::vector<double> &f = t == 1 ? sf : zf;
    for (int q = 0; q < bd.n; ++q) row[bd.tri_state[q]] += f[q];
  }
  return OTS_OK;
}

ots_status ots_batch_get_duals(ots_batch *b, int32_t id, double *log_u, double *log_U01, double *log_U0T) {
  clear_error();
  if (!b) return fail(OTS_ERR_INVALID_ARG, "batch is NULL");
  Slot *sl = find_slot(b, id);
  if (!sl) return fail(OTS_ERR_INVALID_ARG, "unknown batch instance %d", id);
  return ots_get_duals(sl->p, log_u, log_U01, log_U0T);   // copies only, on the batch stream
}

ots_status ots_batch_remove(ots_batch *b, int32_t id) {
  clear_error();
  if (!b) return fail(OTS_ERR_INVALID_ARG, "batch is NULL");
  auto it = b->id_slot.find(id);
  if (it == b->id_slot.end()) return fail(OTS_ERR_INVALID_ARG, "unknown batch instance %d", id);
  Slot &sl = b->slots[it->second];
  DeviceGuard guard(b->dev);
  if (sl.state == SlotState::Running) {
    OTS_CUDA(cudaMemcpyAsync(&b->d_ctl[it->second].status, b->h_stop, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    b->n_items_list -= sl.n_items;
    b->items_dirty = true;
  }
  // every launch that could touch the instance's memory precedes the copies issued for the
  // next instance placed there (same stream)
  ots_destroy_problem(sl.p);
  sl = Slot{};
  b->id_slot.erase(it);
  return OTS_OK;
}

ots_status ots_batch_info(const ots_batch *b, ots_batch_stats *o) {
  if (!b || !o) return fail(OTS_ERR_INVALID_ARG, "NULL argument");
  std::memset(o, 0, sizeof(*o));
  for (auto &s : b->slots) {
    o->resident += s.state != SlotState::Free;
    o->running += s.state == SlotState::Running;
  }
  o->pool_bytes = (int64_t)b->pool.size;
  o->pool_used = (int64_t)b->pool.used;
  o->launches = b->launches;
  o->ticks = b->ticks;
  o->items = b->n_items_list;
  o->h2d_bytes = b->h2d;
  o->d2h_bytes = b->d2h;
  return OTS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Autotuner of the thread mapping (G threads per node row, C = 1 or 2 chunks of 4
// commodities per thread) per class of commodity counts.  Candidates of a class with at most Lc commodities
// are the mappings with panel width 4 G C = Lc and G <= 32; each is timed on copies of a
// synthetic 128 x 128 grid instance (T = 8, L = Lc, one source and one sink per commodity,
// no capacities) that never converge (tol = 0), over 4 launches after 2 warm-up launches.
// ---------------------------------------------------------------------------------------
namespace {

struct SynthGrid {
  int n = 0;
  std::vector<int32_t> src, dst, sc, ss, zc, zs;
  std::vector<double> cost, wait, sm, zm;
  ots_problem_desc desc{};
};

void make_grid(SynthGrid &g, int side, int L, int T) {
  const int V = side * side;
  g.n = V;
  for (int y = 0; y < side; ++y)
    for (int x = 0; x < side; ++x) {
      const int v = y * side + x;
      const int nb[4][2] = {{x + 1, y}, {x - 1, y}, {x, y + 1}, {x, y - 1}};
      for (auto &q : nb) {
        if (q[0] < 0 || q[0] >= side || q[1] < 0 || q[1] >= side) continue;
        g.src.push_back(v);
        g.dst.push_back(q[1] * side + q[0]);
        g.cost.push_back(1.0 + 0.25 * ((v * 7 + q[0] * 3 + q[1]) % 5));
      }
    }
  g.wait.assign(V, 0.1);
  const int E = (int)g.src.size();
  for (int l = 0; l < L; ++l) {
    // endpoints within T - 2 hops: a node and one a few steps along the diagonal
    const int x0 = (l * 37) % (side - 3), y0 = (l * 91) % (side - 3);
    const int a = y0 * side + x0, z = (y0 + 1) * side + x0 + 2;
    g.sc.push_back(l); g.ss.push_back(E + a); g.sm.push_back(1.0);
    g.zc.push_back(l); g.zs.push_back(E + z); g.zm.push_back(1.0);
  }
  ots_problem_desc &d = g.desc;
  std::memset(&d, 0, sizeof(d));
  d.n_nodes = V;
  d.n_edges = E;
  d.edge_src = g.src.data();
  d.edge_dst = g.dst.data();
  d.edge_cost = g.cost.data();
  d.add_wait_loops = 1;
  d.wait_cost = g.wait.data();
  d.T = T;
  d.L = L;
  d.eps = 0.05;
  d.n_sources = L;
  d.src_commodity = g.sc.data(); d.src_state = g.ss.data(); d.src_mass = g.sm.data();
  d.n_sinks = L;
  d.snk_commodity = g.zc.data(); d.snk_state = g.zs.data(); d.snk_mass = g.zm.data();
}

bool read_tune_file(const char *path, const std::string &device, int *G, int *C) {
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
  std::fclose(f);
  if (txt.find("\"device\": \"" + device + "\"") == std::string::npos) return false;
  int got = 0;
  size_t pos = 0;
  while ((pos = txt.find("{\"L_max\":", pos)) != std::string::npos) {
    int lmax = 0, g = 0, c = 0;
    if (std::sscanf(txt.c_str() + pos, "{\"L_max\": %d, \"G\": %d, \"C\": %d", &lmax, &g, &c) == 3) {
      const int cls = l_class(lmax);
      if (cls < kLClasses && (4 << cls) == lmax && g >= 1 && g <= 32 && (g & (g - 1)) == 0 &&
          (c == 1 || c == 2) && 4 * g * c >= lmax) {
        G[cls] = g;
        C[cls] = c;
        ++got;
      }
    }
    ++pos;
  }
  return got == kLClasses;
}

}  // namespace

extern "C" ots_status ots_batch_autotune(ots_batch *b, const char *cache_path) {
  clear_error();
  if (!b) return fail(OTS_ERR_INVALID_ARG, "batch is NULL");
  for (auto &s : b->slots)
    if (s.state != SlotState::Free) return fail(OTS_ERR_INVALID_ARG, "autotune needs an empty batch");
  DeviceGuard guard(b->dev);
  cudaDeviceProp prop{};
  OTS_CUDA(cudaGetDeviceProperties(&prop, b->dev));
  const std::string device = prop.name;
  int G[kLClasses], C[kLClasses];
  if (cache_path && read_tune_file(cache_path, device, G, C)) {
    std::memcpy(b->map_G, G, sizeof(G));
    std::memcpy(b->map_C, C, sizeof(C));
    b->tuned = true;
    return OTS_OK;
  }
  const int side = 128, T = 8;
  double best_us[kLClasses];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  OTS_CUDA(cudaEventCreate(&e0));
  OTS_CUDA(cudaEventCreate(&e1));
  ots_status rc = OTS_OK;
  for (int cls = 0; cls < kLClasses && rc == OTS_OK; ++cls) {
    const int Lc = 4 << cls;
    SynthGrid g;
    make_grid(g, side, Lc, T);
    ots_solve_opts o;
    ots_default_solve_opts(&o);
    o.tol = 1e-300;
    o.max_iters = 1 << 30;
    best_us[cls] = INFINITY;
    G[cls] = b->map_G[cls];
    C[cls] = b->map_C[cls];
    for (int cc : {1, 2}) {
      const int q = Lc / (4 * cc);
      if (q < 1 || q > 32) continue;
      b->map_G[cls] = q;
      b->map_C[cls] = cc;
      const int copies = std::max(1, std::min(b->max_slots, (1 << 22) / (g.n * Lc)));
      std::vector<int32_t> ids;
      for (int k = 0; k < copies; ++k) {
        int32_t id = -1;
        ots_status st = ots_batch_add(b, &g.desc, &o, &id);
        if (st == OTS_ERR_OOM && !ids.empty()) break;   // as many copies as fit
        if (st) { rc = st; break; }
        ids.push_back(id);
      }
      if (rc == OTS_OK) rc = ots_batch_run(b, 2, nullptr);
      float ms = 0.f;
      if (rc == OTS_OK) {
        if (cudaEventRecord(e0, b->stream) != cudaSuccess) rc = fail(OTS_ERR_CUDA, "event record");
        for (int k = 0; k < 4 && rc == OTS_OK; ++k)
          if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) rc = fail(OTS_ERR_CUDA, "graph launch");
        if (rc == OTS_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          rc = fail(OTS_ERR_CUDA, "event timing");
        b->launches += 4;
        b->ticks += 4LL * b->ticks_per_launch;
      }
      for (int32_t id : ids) ots_batch_remove(b, id);
      if (rc) break;
      // time per tick and per (node x commodity) of the resident copies
      const double us = 1000.0 * ms / (4.0 * b->ticks_per_launch) / ((double)ids.size());
      if (us < best_us[cls]) { best_us[cls] = us; G[cls] = q; C[cls] = cc; }
    }
    b->map_G[cls] = G[cls];
    b->map_C[cls] = C[cls];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->tuned = true;
  if (cache_path) {
    FILE *f = std::fopen(cache_path, "w");
    if (!f) return fail(OTS_ERR_INVALID_ARG, "cannot write %s", cache_path);
    std::fprintf(f, "{\"device\": \"%s\", \"grid_side\": %d, \"T\": %d, \"classes\": [\n", device.c_str(), side, T);
    for (int cls = 0; cls < kLClasses; ++cls)
      std::fprintf(f, "  {\"L_max\": %d, \"G\": %d, \"C\": %d, \"us_per_tick\": %.3f}%s\n", 4 << cls, G[cls], C[cls],
                   best_us[cls], cls + 1 < kLClasses ? "," : "");
    std::fprintf(f, "]}\n");
    std::fclose(f);
  }
  return OTS_OK;
}
