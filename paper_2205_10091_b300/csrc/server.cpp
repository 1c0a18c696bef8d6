// Serving loop: continuous admission of circuit energy+gradient requests.
//
// Requests (an op list, parameters and a Pauli sum, as in tc_expect_grad) are
// queued by tc_submit.  A scheduler thread admits them in arrival order as
// soon as a stream slot and enough of the memory budget are free: each
// admitted request gets one stream-ordered block from the server's own memory
// pool holding its plan, its compiled Pauli sum, its parameters, its
// workspace (two states) and its outputs, and runs on its own CUDA stream, so
// the work of requests that arrive while others run overlaps on the device.
// Completion is detected with an event query; the block is returned to the
// pool in stream order and the next request is admitted.  The per-request
// arithmetic is exactly tc_expect_grad's, so a result does not depend on what
// else is in flight.
#include <atomic>
#include <chrono>
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

enum : int { RS_PENDING = 0, RS_RUNNING = 1, RS_DONE = 2 };

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
  // in flight
  tc_circuit* circ = nullptr;
  int slot = -1;
  size_t bytes = 0;
  // result
  double energy = 0;
  std::vector<double> grad;
};

}  // namespace

struct tc_server {
  tc_server_options opt{};
  int device = -1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Req>> pending;
  std::vector<std::shared_ptr<Req>> inflight;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> table;  // every request not yet collected by tc_poll
  uint64_t next_id = 1;
  std::atomic<bool> stop{false};
  std::atomic<bool> paused{false};
  std::thread th;
  bool gpu_ready = false;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<double*> h_out;  // pinned, per slot: [energy, grad...]
  std::vector<char> slot_busy;
  int n_high = 0;  // slots [0, n_high) use high-priority streams (small requests)
  cudaMemPool_t pool = nullptr;
  int64_t used = 0;
  tc_server_stats stats{};
  std::string fatal;
};

namespace {

constexpr int kMaxParams = 256;
constexpr int kSmallQubits = 20;

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
    if ((e = cudaMallocHost((void**)&s->h_out[i], sizeof(double) * (1 + kMaxParams))) != cudaSuccess)
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
  if (st == TC_OK) s->stats.completed++;
  else if (st == TC_E_CANCELLED) s->stats.cancelled++;
  else if (st == TC_E_TIMEOUT) s->stats.timed_out++;
  else s->stats.failed++;
}

// Admit one request (lock held by the caller is released around GPU work).
// Returns false if it does not fit right now.
bool try_admit(tc_server* s, std::unique_lock<std::mutex>& lk) {
  if (s->pending.empty()) return false;
  std::shared_ptr<Req> r = s->pending.front();
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
  // plan on the host (no device memory yet)
  tc_circuit* c = nullptr;
  tc_status st = tc_circuit_create(r->n, TC_C64, (tc_init)r->init, r->ops.data(), (int)r->ops.size(), r->n_params,
                                   r->pool.empty() ? nullptr : r->pool.data(), r->n_pool, nullptr, &c);
  if (st != TC_OK) {
    s->pending.pop_front();
    finish(s, r, st, tc_last_error());
    return true;
  }
  HamPlan H;
  std::string err;
  if (!build_hamiltonian(c->n, c->N, c->k_ham, r->structures.data(), r->weights.data(), r->T, H, err)) {
    tc_circuit_destroy(c);
    s->pending.pop_front();
    finish(s, r, TC_E_INVALID, err);
    return true;
  }
  c->H = H;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t b_plan = plan_dev_bytes(c) + ham_dev_bytes(H);
  const size_t b_ws = grad_ws_bytes(c, 1);
  const size_t b_io = al(8 * (size_t)std::max(r->n_params, 1)) * 2 + 256;
  const size_t need = al(b_plan) + al(b_ws) + b_io;
  if ((int64_t)need > s->opt.mem_budget_bytes) {
    tc_circuit_destroy(c);
    s->pending.pop_front();
    finish(s, r, TC_E_NOMEM, "request needs more device memory than the server's whole budget");
    return true;
  }
  if (s->used + (int64_t)need > s->opt.mem_budget_bytes) {
    tc_circuit_destroy(c);
    return false;  // wait for memory to free up (arrival order is kept)
  }
  s->pending.pop_front();
  s->slot_busy[slot] = 1;
  s->used += (int64_t)need;
  s->stats.peak_bytes = std::max<int64_t>(s->stats.peak_bytes, s->used);
  r->circ = c;
  r->slot = slot;
  r->bytes = need;
  r->state = RS_RUNNING;
  r->t_start = now_s();
  s->inflight.push_back(r);
  s->stats.peak_inflight = std::max<int32_t>(s->stats.peak_inflight, (int32_t)s->inflight.size());
  lk.unlock();
  // ---- device work, in stream order on this slot's stream ----
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
    char* p_ws = block + al(b_plan);
    double* d_theta = (double*)(p_ws + al(b_ws));
    double* d_e = d_theta + al(8 * (size_t)std::max(r->n_params, 1)) / 8;
    double* d_g = d_e + 4;
    rs = place_plan_and_ham(c, H, p_plan, str);
    if (rs == TC_OK && r->n_params > 0) {
      e = cudaMemcpyAsync(d_theta, r->theta.data(), 8 * (size_t)r->n_params, cudaMemcpyHostToDevice, str);
      if (e != cudaSuccess) rs = cuda_fail(e, "parameter copy");
    }
    if (rs == TC_OK) rs = expect_grad_run(c, d_theta, 1, 0, d_e, d_g, 1, p_ws, str);
    if (rs == TC_OK) {
      e = cudaMemcpyAsync(s->h_out[slot], d_e, 8, cudaMemcpyDeviceToHost, str);
      if (e == cudaSuccess && r->n_params > 0)
        e = cudaMemcpyAsync(s->h_out[slot] + 1, d_g, 8 * (size_t)r->n_params, cudaMemcpyDeviceToHost, str);
      if (e != cudaSuccess) rs = cuda_fail(e, "result copy");
    }
    if (rs != TC_OK) msg = tc_last_error();
    cudaFreeAsync(block, str);
  }
  cudaEventRecord(s->events[slot], str);
  lk.lock();
  if (rs != TC_OK) r->status = rs, r->error = msg;  // reported when the event completes
  return true;
}

void reap(tc_server* s) {
  for (size_t i = 0; i < s->inflight.size();) {
    auto r = s->inflight[i];
    const cudaError_t q = cudaEventQuery(s->events[r->slot]);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    if (q == cudaSuccess && r->status == TC_OK) {
      const double* o = s->h_out[r->slot];
      r->energy = o[0];
      r->grad.assign(o + 1, o + 1 + r->n_params);
      finish(s, r, TC_OK, "");
    } else {
      finish(s, r, r->status != TC_OK ? r->status : TC_E_CUDA,
             r->error.empty() ? std::string(cudaGetErrorString(q)) : r->error);
    }
    s->slot_busy[r->slot] = 0;
    s->used -= (int64_t)r->bytes;
    tc_circuit_destroy(r->circ);
    r->circ = nullptr;
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
  s->paused = s->opt.start_paused != 0;
  cudaGetDevice(&s->device);
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
    s->table[r->id] = r;
    s->stats.submitted++;
  }
  s->cv.notify_one();
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
  out->inflight = (int32_t)s->inflight.size();
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
  if (s->th.joinable()) s->th.join();
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
