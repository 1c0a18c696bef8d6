// Serving loop: continuous admission of circuit energy+gradient requests.
//
// Requests (an op list, parameters and a Pauli sum, as in tc_expect_grad) are
// queued by tc_submit and planned at once on a few planner threads (plan
// compilation and the Pauli-sum plan, host only), off the scheduler thread.
// The scheduler admits them in arrival order as soon as a stream slot and
// enough of the memory budget are free.  Requests whose plans differ only in
// the column words of packed diagonal groups and in the Pauli sum's diagonal
// records (QAOA instances of one width and depth on different graphs, for
// example) are admitted together, up to max_group_rows of them, as the rows
// of one evaluation: one launch per pass for the whole group, with a per-row
// copy of those entries.  Each admitted group gets one stream-ordered block
// from the server's own memory pool holding its plan, the per-row entries,
// its parameters, its workspace (two states per row) and its outputs, and
// runs on its own CUDA stream, so groups overlap on the device.  Completion
// is detected with an event query; the block is returned to the pool in
// stream order and the next request is admitted.  A row's arithmetic is
// exactly tc_expect_grad's on that request alone, so a result does not
// depend on what it was grouped or overlapped with.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "engine.h"

using namespace tcb;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// TC_SERVER_TRACE=1: one line per planning, admission, launch step and
// completion on stderr (request ids, slot, rows, status)
bool trace_on() {
  static const bool on = [] {
    const char* v = std::getenv("TC_SERVER_TRACE");
    return v && v[0] == '1';
  }();
  return on;
}
#define TC_TRACE(...)                                    \
  do {                                                   \
    if (trace_on()) {                                    \
      std::fprintf(stderr, "[tc_server %.6f] ", now_s()); \
      std::fprintf(stderr, __VA_ARGS__);                 \
      std::fprintf(stderr, "\n");                        \
    }                                                    \
  } while (0)

enum : int { RS_PENDING = 0, RS_RUNNING = 1, RS_DONE = 2 };
enum : int { PL_QUEUED = 0, PL_READY = 1, PL_FAILED = 2 };

struct Req {
  uint64_t id = 0;
  int n = 0, init = 0, n_params = 0, n_pool = 0, T = 0;
  std::vector<tc_op> ops;
  std::vector<double> pool, theta, weights;
  std::vector<uint8_t> structures;
  double t_submit = 0, t_start = 0, t_done = 0;
  int state = RS_PENDING;
  tc_status status = TC_OK;
  std::string error;
  // planned on a planner thread
  int planned = PL_QUEUED;
  tc_circuit* circ = nullptr;
  HamPlan H;
  std::string shape;  // the plan's bytes that all rows of one launch share
  uint64_t key = 0;   // hash of `shape`
  // result
  double energy = 0;
  std::vector<double> grad;
};

// Requests evaluated as the rows of one launch sequence on one slot.
struct Group {
  std::vector<std::shared_ptr<Req>> reqs;
  int slot = -1;
  size_t bytes = 0;
  tc_status status = TC_OK;
  std::string error;
};

// Everything of a plan except the diagonal entries' values and the Pauli
// sum's diagonal records: requests with equal shapes can share one launch.
std::string plan_shape(const tc_circuit* c, const HamPlan& H) {
  std::string s;
  auto put = [&](const void* p, size_t n) { s.append((const char*)p, n); };
  auto vec = [&](const auto& v) {
    const uint64_t n = v.size();
    put(&n, sizeof n);
    if (n) put(v.data(), v.size() * sizeof(v[0]));
  };
  auto sched = [&](const Schedule& q) {
    const int f[] = {q.first_pass, q.n_passes, q.k, q.n_gslots, q.n_stages, q.first_mat, q.n_mats, q.table_total};
    put(f, sizeof f);
    vec(q.slot_param);
  };
  const int hdr[] = {c->n, c->N, (int)c->init, (int)c->dtype, c->n_params, c->n_noise, c->k_fwd, c->k_bwd, c->k_ham};
  put(hdr, sizeof hdr);
  sched(c->fwd);
  sched(c->bwd);
  vec(c->A.passes);
  vec(c->A.stages);
  vec(c->A.instrs);
  vec(c->A.mats);
  vec(c->A.diags);
  const uint64_t nd = c->A.dents.size(), nh = H.hdiag.size();
  put(&nd, sizeof nd);
  vec(c->pool);
  vec(c->csr_off);
  vec(c->csr_slots);
  vec(H.passes);
  vec(H.hterms);
  vec(H.hflips);
  put(&nh, sizeof nh);
  return s;
}

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char ch : s) h = (h ^ ch) * 1099511628211ull;
  return h;
}

// Host-only planning of one request (planner thread, no lock held: it reads
// only the request's inputs, which never change after tc_submit).
struct Planned {
  int planned = PL_FAILED;
  tc_status status = TC_OK;
  std::string error;
  tc_circuit* circ = nullptr;
  HamPlan H;
  std::string shape;
  uint64_t key = 0;
};

Planned plan_request(const Req& r) {
  Planned o;
  tc_circuit* c = nullptr;
  tc_status st = tc_circuit_create(r.n, TC_C64, (tc_init)r.init, r.ops.data(), (int)r.ops.size(), r.n_params,
                                   r.pool.empty() ? nullptr : r.pool.data(), r.n_pool, nullptr, &c);
  if (st != TC_OK) {
    o.status = st;
    o.error = tc_last_error();
    return o;
  }
  std::string err;
  if (!build_hamiltonian(c->n, c->N, c->k_ham, r.structures.data(), r.weights.data(), r.T, o.H, err)) {
    tc_circuit_destroy(c);
    o.status = TC_E_INVALID;
    o.error = err;
    return o;
  }
  // the circuit carries its Pauli sum from here on: the workspace size of an
  // energy+gradient evaluation (grad_ws_bytes) depends on its passes
  c->H = o.H;
  o.circ = c;
  o.shape = plan_shape(c, o.H);
  o.key = fnv1a(o.shape);
  o.planned = PL_READY;
  return o;
}

void release_plan(Req& r) {
  if (r.circ) tc_circuit_destroy(r.circ);
  r.circ = nullptr;
}

}  // namespace

struct tc_server {
  tc_server_options opt{};
  int device = -1;
  int max_rows = 1;  // requests a group may hold
  std::mutex mu;
  std::condition_variable cv;       // scheduler wake-ups
  std::condition_variable plan_cv;  // planner wake-ups
  std::deque<std::shared_ptr<Req>> pending;  // arrival order, planned or not
  std::deque<std::shared_ptr<Req>> to_plan;
  std::vector<std::shared_ptr<Group>> inflight;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> table;  // every request not yet collected by tc_poll
  uint64_t next_id = 1;
  std::atomic<bool> stop{false};
  std::atomic<bool> paused{false};
  std::thread th;
  std::vector<std::thread> planners;
  bool gpu_ready = false;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<double*> h_out;  // pinned, per slot: max_rows x [energy, grad...]
  std::vector<char> slot_busy;
  int n_high = 0;  // slots [0, n_high) use high-priority streams (small requests)
  cudaMemPool_t pool = nullptr;
  int64_t used = 0;
  tc_server_stats stats{};
  std::string fatal;
};

namespace {

constexpr int kMaxParams = 256;
constexpr int kSmallQubits = 20;     // two states of at most 2^20 amplitudes: "small"
constexpr int kGroupMaxQubits = 20;  // wider requests fill the GPU alone: not grouped
constexpr int kGroupScan = 512;      // pending requests examined for one group

size_t out_doubles(int rows) { return (size_t)rows * (1 + kMaxParams); }

tc_status gpu_init(tc_server* s) {
  if (s->gpu_ready) return TC_OK;
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  if ((e = cudaMemPoolCreate(&s->pool, &props)) != cudaSuccess) return cuda_fail(e, "cudaMemPoolCreate");
  uint64_t keep = (uint64_t)s->opt.mem_budget_bytes;  // keep freed blocks for reuse up to the budget
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  const int slots = s->opt.max_inflight;
  s->streams.resize(slots);
  s->events.resize(slots);
  s->h_out.resize(slots);
  s->slot_busy.assign(slots, 0);
  // the first half of the slots run on high-priority streams: small requests
  // placed there are not held back by the thread blocks of large ones
  int lo_prio = 0, hi_prio = 0;
  cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
  s->n_high = slots / 2;
  for (int i = 0; i < slots; ++i) {
    if ((e = cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking, i < s->n_high ? hi_prio : lo_prio)) !=
        cudaSuccess)
      return cuda_fail(e, "stream");
    if ((e = cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "event");
    if ((e = cudaMallocHost((void**)&s->h_out[i], sizeof(double) * out_doubles(s->max_rows))) != cudaSuccess)
      return cuda_fail(e, "pinned result buffer");
  }
  s->gpu_ready = true;
  return TC_OK;
}

void finish(tc_server* s, const std::shared_ptr<Req>& r, tc_status st, const std::string& msg) {
  r->status = st;
  r->error = msg;
  r->state = RS_DONE;
  r->t_done = now_s();
  release_plan(*r);
  if (st == TC_OK) s->stats.completed++;
  else if (st == TC_E_CANCELLED) s->stats.cancelled++;
  else if (st == TC_E_TIMEOUT) s->stats.timed_out++;
  else s->stats.failed++;
}

void planner(tc_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->plan_cv.wait(lk, [&] { return s->stop || !s->to_plan.empty(); });
    if (s->to_plan.empty()) {
      if (s->stop) break;
      continue;
    }
    std::shared_ptr<Req> r = s->to_plan.front();
    s->to_plan.pop_front();
    if (r->state != RS_PENDING) continue;  // cancelled or expired meanwhile
    lk.unlock();
    Planned o = plan_request(*r);
    lk.lock();
    if (r->state != RS_PENDING) {  // finished while it was planned
      if (o.circ) tc_circuit_destroy(o.circ);
      continue;
    }
    r->planned = o.planned;
    r->circ = o.circ;
    r->H = std::move(o.H);
    r->shape = std::move(o.shape);
    r->key = o.key;
    if (o.planned == PL_FAILED) r->status = o.status, r->error = o.error;
    TC_TRACE("planned id %llu n %d ok %d key %016llx", (unsigned long long)r->id, r->n, o.planned == PL_READY,
             (unsigned long long)o.key);
    s->cv.notify_one();
  }
}

// Bytes of one group's block: plan and Pauli sum once, per-row diagonal
// copies, workspace, parameters and outputs.
size_t group_bytes(const tc_circuit* c, const HamPlan& H, int rows) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t np = (size_t)std::max(c->n_params, 1);
  return al(plan_dev_bytes(c) + ham_dev_bytes(H)) + al(rows * c->A.dents.size() * sizeof(DevDiagEnt)) +
         al(rows * H.hdiag.size() * sizeof(DevHDiag)) + al(grad_ws_bytes(c, rows)) + al(8 * np * rows) +
         al(8 * (size_t)rows) + al(8 * np * rows) + 256;
}

// Admit the request at the head of the queue, with the later queued requests
// of the same plan shape as further rows (lock held by the caller; released
// around the GPU work).  Returns false if nothing can be admitted right now.
bool try_admit(tc_server* s, std::unique_lock<std::mutex>& lk) {
  if (s->pending.empty()) return false;
  std::shared_ptr<Req> r = s->pending.front();
  if (r->planned == PL_QUEUED) return false;  // its plan is on the way; arrival order is kept
  if (r->planned == PL_FAILED) {
    s->pending.pop_front();
    finish(s, r, r->status, r->error);
    return true;
  }
  // small requests (two states of at most 2^20 amplitudes) prefer the
  // high-priority slots and may use any; large ones use the others
  const bool small = r->n <= kSmallQubits;
  int slot = -1;
  for (int i = small ? 0 : s->n_high; i < (int)s->slot_busy.size(); ++i)
    if (!s->slot_busy[i]) {
      slot = i;
      break;
    }
  if (slot < 0) return false;
  std::vector<std::shared_ptr<Req>> mem{r};
  if (r->n <= kGroupMaxQubits && s->max_rows > 1) {
    const size_t scan = std::min(s->pending.size(), (size_t)kGroupScan);
    for (size_t i = 1; i < scan && (int)mem.size() < s->max_rows; ++i) {
      const auto& q = s->pending[i];
      if (q->planned == PL_READY && q->key == r->key && q->shape == r->shape) mem.push_back(q);
    }
  }
  tc_circuit* c = r->circ;
  size_t need = group_bytes(c, r->H, (int)mem.size());
  while (mem.size() > 1 && s->used + (int64_t)need > s->opt.mem_budget_bytes) {
    mem.pop_back();
    need = group_bytes(c, r->H, (int)mem.size());
  }
  if (mem.size() == 1 && (int64_t)need > s->opt.mem_budget_bytes) {
    s->pending.pop_front();
    finish(s, r, TC_E_NOMEM, "request needs more device memory than the server's whole budget");
    return true;
  }
  if (s->used + (int64_t)need > s->opt.mem_budget_bytes) return false;  // wait for memory to free up
  // take the members out of the queue
  {
    std::deque<std::shared_ptr<Req>> rest;
    size_t m = 0;
    for (auto& q : s->pending) {
      if (m < mem.size() && q == mem[m]) ++m;
      else rest.push_back(q);
    }
    s->pending.swap(rest);
  }
  auto g = std::make_shared<Group>();
  g->reqs = mem;
  g->slot = slot;
  g->bytes = need;
  s->slot_busy[slot] = 1;
  s->used += (int64_t)need;
  s->stats.peak_bytes = std::max<int64_t>(s->stats.peak_bytes, s->used);
  const double t = now_s();
  for (auto& q : mem) q->state = RS_RUNNING, q->t_start = t;
  s->inflight.push_back(g);
  int32_t rows_in_flight = 0;
  for (auto& f : s->inflight) rows_in_flight += (int32_t)f->reqs.size();
  s->stats.peak_inflight = std::max<int32_t>(s->stats.peak_inflight, rows_in_flight);
  s->stats.groups++;
  if (mem.size() > 1) s->stats.grouped_requests += (int64_t)mem.size();
  // host copies of the per-row data (the inputs never change after tc_submit)
  const int B = (int)mem.size();
  const int P = r->n_params;
  const size_t nd = c->A.dents.size(), nh = r->H.hdiag.size();
  std::vector<DevDiagEnt> h_dents(B * nd);
  std::vector<DevHDiag> h_hdiag(B * nh);
  std::vector<double> h_theta((size_t)B * std::max(P, 1));
  for (int i = 0; i < B; ++i) {
    std::copy(mem[i]->circ->A.dents.begin(), mem[i]->circ->A.dents.end(), h_dents.begin() + i * nd);
    std::copy(mem[i]->H.hdiag.begin(), mem[i]->H.hdiag.end(), h_hdiag.begin() + i * nh);
    std::copy(mem[i]->theta.begin(), mem[i]->theta.end(), h_theta.begin() + (size_t)i * P);
  }
  const HamPlan H = r->H;
  TC_TRACE("admit id %llu rows %d slot %d bytes %zu", (unsigned long long)r->id, B, slot, need);
  lk.unlock();
  // ---- device work, in stream order on this slot's stream ----
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  cudaStream_t str = s->streams[slot];
  char* block = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync((void**)&block, need, s->pool, str);
  tc_status rs = TC_OK;
  std::string msg;
  if (e != cudaSuccess) {
    rs = TC_E_NOMEM;
    msg = std::string("pool allocation: ") + cudaGetErrorString(e);
    cudaGetLastError();
  } else {
    char* p_plan = block;
    char* p_dents = p_plan + al(plan_dev_bytes(c) + ham_dev_bytes(H));
    char* p_hdiag = p_dents + al(B * nd * sizeof(DevDiagEnt));
    char* p_ws = p_hdiag + al(B * nh * sizeof(DevHDiag));
    double* d_theta = (double*)(p_ws + al(grad_ws_bytes(c, B)));
    double* d_e = d_theta + al(8 * (size_t)std::max(P, 1) * B) / 8;
    double* d_g = d_e + al(8 * (size_t)B) / 8;
    TC_TRACE("slot %d block allocated", slot);
    // the layout must end inside the block (its size is group_bytes')
    if ((char*)(d_g + (size_t)B * P) > block + need) rs = fail(TC_E_INVALID, "internal: group layout exceeds its block");
    const size_t ws_room = (size_t)((char*)d_theta - p_ws);
    if (rs == TC_OK) rs = place_plan_and_ham(c, H, p_plan, str);
    // the evaluation's own workspace size, now that the circuit holds its
    // Pauli sum, must fit the room the layout gave it
    if (rs == TC_OK && grad_ws_bytes(c, B) > ws_room) rs = fail(TC_E_INVALID, "internal: workspace exceeds its room");
    auto up = [&](void* dst, const void* src, size_t bytes, const char* what) {
      if (rs != TC_OK || bytes == 0) return;
      const cudaError_t ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, str);
      if (ce != cudaSuccess) rs = cuda_fail(ce, what);
    };
    up(p_dents, h_dents.data(), h_dents.size() * sizeof(DevDiagEnt), "diagonal entries copy");
    up(p_hdiag, h_hdiag.data(), h_hdiag.size() * sizeof(DevHDiag), "Pauli-sum diagonal copy");
    up(d_theta, h_theta.data(), (size_t)B * P * 8, "parameter copy");
    const RowDiag rd{(const DevDiagEnt*)p_dents, (int)nd, (const DevHDiag*)p_hdiag, (int)nh};
    TC_TRACE("slot %d inputs copied (status %d)", slot, (int)rs);
    if (rs == TC_OK) rs = expect_grad_run(c, d_theta, B, 0, d_e, d_g, B, p_ws, str, &rd);
    TC_TRACE("slot %d launched (status %d)", slot, (int)rs);
    if (rs == TC_OK) {
      e = cudaMemcpyAsync(s->h_out[slot], d_e, 8 * (size_t)B, cudaMemcpyDeviceToHost, str);
      if (e == cudaSuccess && P > 0)
        e = cudaMemcpyAsync(s->h_out[slot] + B, d_g, 8 * (size_t)B * P, cudaMemcpyDeviceToHost, str);
      if (e != cudaSuccess) rs = cuda_fail(e, "result copy");
    }
    if (rs != TC_OK) msg = tc_last_error();
    cudaFreeAsync(block, str);
  }
  cudaEventRecord(s->events[slot], str);
  lk.lock();
  if (rs != TC_OK) g->status = rs, g->error = msg;  // reported when the event completes
  return true;
}

void reap(tc_server* s) {
  for (size_t i = 0; i < s->inflight.size();) {
    auto g = s->inflight[i];
    const cudaError_t q = cudaEventQuery(s->events[g->slot]);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    const int B = (int)g->reqs.size();
    TC_TRACE("slot %d done: event %d group status %d", g->slot, (int)q, (int)g->status);
    if (q == cudaSuccess && g->status == TC_OK) {
      const double* o = s->h_out[g->slot];
      for (int k = 0; k < B; ++k) {
        const auto& r = g->reqs[k];
        r->energy = o[k];
        r->grad.assign(o + B + (size_t)k * r->n_params, o + B + (size_t)(k + 1) * r->n_params);
        finish(s, r, TC_OK, "");
      }
    } else {
      for (auto& r : g->reqs)
        finish(s, r, g->status != TC_OK ? g->status : TC_E_CUDA,
               g->error.empty() ? std::string(cudaGetErrorString(q)) : g->error);
    }
    s->slot_busy[g->slot] = 0;
    s->used -= (int64_t)g->bytes;
    s->inflight.erase(s->inflight.begin() + i);
  }
}

void expire(tc_server* s) {
  if (s->opt.timeout_ms <= 0) return;
  const double t = now_s();
  for (size_t i = 0; i < s->pending.size();) {
    auto r = s->pending[i];
    if ((t - r->t_submit) * 1e3 > s->opt.timeout_ms) {
      finish(s, r, TC_E_TIMEOUT, "waited longer than the server timeout before admission");
      s->pending.erase(s->pending.begin() + i);
    } else {
      ++i;
    }
  }
}

void scheduler(tc_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    expire(s);
    if (!s->paused) {
      if (!s->gpu_ready) {
        lk.unlock();
        tc_status st = gpu_init(s);
        lk.lock();
        if (st != TC_OK) {
          s->fatal = tc_last_error();
          for (auto& r : s->pending) finish(s, r, st, s->fatal);
          s->pending.clear();
          s->paused = true;
        }
      }
      if (s->gpu_ready) {
        reap(s);
        while (try_admit(s, lk)) {
        }
      }
    }
    if (s->stop && s->inflight.empty() && (s->pending.empty() || s->paused)) break;
    // short waits keep admission latency low while work is in flight
    s->cv.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 1000 : 20));
  }
}

}  // namespace

extern "C" {

tc_status tc_server_create(const tc_server_options* opt, tc_server** out) {
  if (!out) return fail(TC_E_INVALID, "out is NULL");
  *out = nullptr;
  auto* s = new tc_server();
  if (opt) s->opt = *opt;
  if (s->opt.max_inflight <= 0) s->opt.max_inflight = 16;
  if (s->opt.max_inflight > 256) s->opt.max_inflight = 256;
  if (s->opt.mem_budget_bytes <= 0) s->opt.mem_budget_bytes = (int64_t)8 << 30;
  s->max_rows = s->opt.max_group_rows <= 0 ? 32 : std::min(s->opt.max_group_rows, 1024);
  const int nplan = s->opt.planner_threads <= 0 ? 2 : std::min(s->opt.planner_threads, 16);
  s->paused = s->opt.start_paused != 0;
  cudaGetDevice(&s->device);
  for (int i = 0; i < nplan; ++i) s->planners.emplace_back(planner, s);
  s->th = std::thread(scheduler, s);
  *out = s;
  return TC_OK;
}

tc_status tc_submit(tc_server* s, const tc_request* q, uint64_t* id_out) {
  if (!s || !q || !id_out) return fail(TC_E_INVALID, "NULL argument");
  if (q->n_qubits < 1 || q->n_qubits > kMaxQubits) return fail(TC_E_INVALID, "n_qubits must be in 1..30");
  if (q->n_ops < 0 || (q->n_ops > 0 && !q->ops)) return fail(TC_E_INVALID, "ops is NULL");
  if (q->n_params < 0 || q->n_params > kMaxParams) return fail(TC_E_INVALID, "n_params must be in 0..256");
  if (q->n_params > 0 && !q->theta) return fail(TC_E_INVALID, "theta is NULL");
  if (q->T < 0 || (q->T > 0 && (!q->structures || !q->weights))) return fail(TC_E_INVALID, "Pauli sum is NULL");
  if (q->n_pool < 0 || (q->n_pool > 0 && !q->pool)) return fail(TC_E_INVALID, "pool is NULL");
  // validate the op list now so a malformed request is refused at the door
  {
    std::vector<HGate> g;
    std::string err;
    const int N = q->n_qubits < kMinQubits ? kMinQubits : q->n_qubits;
    if (!normalise_ops(q->n_qubits, N, q->ops, q->n_ops, q->n_params, q->n_pool, g, err))
      return fail(TC_E_INVALID, err);
    for (int t = 0; t < q->T * q->n_qubits; ++t)
      if (q->structures[t] > 3) return fail(TC_E_INVALID, "structure entry outside {0,1,2,3}");
  }
  auto r = std::make_shared<Req>();
  r->n = q->n_qubits;
  r->init = q->init;
  r->n_params = q->n_params;
  r->n_pool = q->n_pool;
  r->T = q->T;
  r->ops.assign(q->ops, q->ops + q->n_ops);
  r->pool.assign(q->pool, q->pool + 2 * (size_t)q->n_pool);
  r->theta.assign(q->theta, q->theta + q->n_params);
  r->structures.assign(q->structures, q->structures + (size_t)q->T * q->n_qubits);
  r->weights.assign(q->weights, q->weights + q->T);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(TC_E_CANCELLED, "server is shutting down");
    if (s->opt.max_queue > 0 && (int)s->pending.size() >= s->opt.max_queue) {
      s->stats.rejected++;
      return fail(TC_E_BUSY, "queue full");
    }
    r->id = s->next_id++;
    r->t_submit = now_s();
    s->pending.push_back(r);
    s->to_plan.push_back(r);
    s->table[r->id] = r;
    s->stats.submitted++;
  }
  s->plan_cv.notify_one();
  *id_out = r->id;
  return TC_OK;
}

tc_status tc_poll(tc_server* s, uint64_t id, tc_result* out, double* grad_out, int max_params) {
  if (!s || !out) return fail(TC_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->table.find(id);
  if (it == s->table.end()) return fail(TC_E_INVALID, "unknown request id");
  auto r = it->second;
  if (r->state != RS_DONE) return TC_E_BUSY;
  memset(out, 0, sizeof(*out));
  out->id = r->id;
  out->status = r->status;
  out->n_params = r->n_params;
  out->energy = r->energy;
  out->t_submit = r->t_submit;
  out->t_start = r->t_start;
  out->t_done = r->t_done;
  if (grad_out)
    for (int k = 0; k < r->n_params && k < max_params; ++k) grad_out[k] = r->grad.size() > (size_t)k ? r->grad[k] : 0;
  if (r->status != TC_OK) set_error(r->error);
  s->table.erase(it);
  return TC_OK;
}

tc_status tc_cancel(tc_server* s, uint64_t id) {
  if (!s) return fail(TC_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->table.find(id);
  if (it == s->table.end()) return fail(TC_E_INVALID, "unknown request id");
  auto r = it->second;
  if (r->state != RS_PENDING) return fail(TC_E_BUSY, "request already admitted");
  for (size_t i = 0; i < s->pending.size(); ++i)
    if (s->pending[i] == r) {
      s->pending.erase(s->pending.begin() + i);
      break;
    }
  finish(s, r, TC_E_CANCELLED, "cancelled");
  return TC_OK;
}

tc_status tc_server_resume(tc_server* s) {
  if (!s) return fail(TC_E_INVALID, "NULL argument");
  s->paused = false;
  s->cv.notify_one();
  return TC_OK;
}

tc_status tc_server_get_stats(tc_server* s, tc_server_stats* out) {
  if (!s || !out) return fail(TC_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->pending = (int32_t)s->pending.size();
  int32_t rows = 0;
  for (auto& g : s->inflight) rows += (int32_t)g->reqs.size();
  out->inflight = rows;
  int32_t planned = 0;
  for (auto& r : s->pending) planned += r->planned == PL_READY ? 1 : 0;
  out->planned = planned;
  out->bytes_in_use = s->used;
  return TC_OK;
}

tc_status tc_server_destroy(tc_server* s) {
  if (!s) return TC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // requests never admitted are cancelled; admitted ones finish on the GPU
    for (auto& r : s->pending) finish(s, r, TC_E_CANCELLED, "server destroyed");
    s->pending.clear();
  }
  s->cv.notify_one();
  s->plan_cv.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto& t : s->planners)
    if (t.joinable()) t.join();
  if (s->gpu_ready) {
    for (size_t i = 0; i < s->streams.size(); ++i) {
      cudaStreamSynchronize(s->streams[i]);
      cudaStreamDestroy(s->streams[i]);
      cudaEventDestroy(s->events[i]);
      cudaFreeHost(s->h_out[i]);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
  }
  delete s;
  return TC_OK;
}

}  // extern "C"
