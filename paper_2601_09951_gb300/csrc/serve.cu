// serve.cu -- continuous-batching request loop (sv_server_*), host code.
//
// Requests are independent VQE optimisations (Sec. 4.1, Eq. 7).  A scheduler thread:
//   * admits queued requests in arrival order while their device footprint fits the budget
//     (a request that cannot fit yet is skipped unless it has waited long enough to block the
//     ones behind it, so large requests are not starved of memory; one that only waits for a
//     slot of its kind is skipped);
//   * runs at most max_active_heavy requests of heavy_qubits or more at once: each fills the
//     GPU by itself, so more of them would only compete for it, while their slots serve
//     mid-size requests whose short launches overlap them;
//   * keeps small requests (n <= SV_BATCH_MAX_QUBITS) resident in one device arena and advances
//     all of them by up to steps_per_tick gradient steps per launch of the persistent batched
//     kernel (per-instance step counts, steps and trajectory offsets);
//   * runs large requests on their own context and stream, concurrently with those launches
//     (batched launches and mid-size requests on the device's greatest stream priority, heavy
//     requests on its least, so that the block scheduler starts short work first);
//   * detects completion with events, copies results back and frees the request's memory.
// A finished large request's context (state buffers, stream, Hamiltonian buffers, completion
// event and pinned result buffer) is kept idle for the next request of the same qubit count:
// device and pinned allocations and frees synchronise the whole GPU, so a request that
// allocated on admission or freed on completion would stall every request in flight.  Idle
// contexts count against the budget and are freed, oldest first, only when an admission needs
// their room.
// The arena is managed by a first-fit allocator with coalescing over 768-byte units (a
// multiple of every record size the batched kernel indexes, so byte offsets convert exactly
// to element offsets).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/svqe.h"
#include "api_internal.h"
#include "host_compile.h"
#include "launch.h"
#include "svqe_types.h"

namespace svqe {
namespace {

constexpr int64_t kUnit = 768;                 // lcm of 48, 32, 24, 16, 8, 4 bytes
constexpr int64_t kCkptAmpsPerCta = 36 * 4096;  // checkpoint capacity of one CTA
constexpr double kStarveSeconds = 0.25;         // a queued request blocks later ones after this

int64_t round_up(int64_t v, int64_t u) { return (v + u - 1) / u * u; }

// First-fit allocator over [0, size) bytes in kUnit granules, free blocks coalesced.
class Arena {
 public:
  void reset(int64_t size) {
    free_.clear();
    used_.clear();
    if (size > 0) free_[0] = size;
  }
  int64_t alloc(int64_t bytes) {
    bytes = round_up(std::max<int64_t>(bytes, kUnit), kUnit);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const int64_t off = it->first, left = it->second - bytes;
        free_.erase(it);
        if (left > 0) free_[off + bytes] = left;
        used_[off] = bytes;
        return off;
      }
    }
    return -1;
  }
  void release(int64_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return;
    int64_t start = off, size = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + size) {
      size += next->second;
      free_.erase(next);
    }
    auto prev = free_.lower_bound(start);
    if (prev != free_.begin()) {
      --prev;
      if (prev->first + prev->second == start) {
        start = prev->first;
        size += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = size;
  }

 private:
  std::map<int64_t, int64_t> free_, used_;
};

enum { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3, Q_CANCELLED = 4 };

struct Req {
  uint64_t id = 0;
  int n = 0, steps = 0;
  double lr = 0.0;
  uint64_t ref = 0;
  bool small = false;
  HostCircuit hc;
  HostHam hh;
  std::vector<sv_gate> gates;
  std::vector<uint64_t> hx, hz;
  std::vector<double> hcoef;
  std::vector<Seg> segs;
  int n_ckpt = 0;
  double cost = 0.0;
  std::vector<double> theta, etraj;
  uint64_t footprint = 0;
  int state = Q_QUEUED;
  sv_status status = SV_EBUSY;
  std::string err;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int done_steps = 0;
  // small: one arena block and the instance record (offsets in element units)
  int64_t block = -1;
  BInst rec{};
  int64_t theta_elem = 0, etraj_elem = 0;
  // large: context, Hamiltonian, completion event and pinned results
  sv_ctx* ctx = nullptr;
  sv_ham* ham = nullptr;
  cudaEvent_t ev = nullptr;
  double* pin = nullptr;
  size_t pin_cap = 0;
  cudaStream_t stream = nullptr;  // the context's stream (the server creates and destroys it)
  bool heavy = false;             // n >= heavy_qubits
};

// The device resources of a finished large request, kept for the next request of width n.
struct Idle {
  int n = 0;
  uint64_t bytes = 0;  // charged against the budget while idle
  sv_ctx* ctx = nullptr;
  sv_ham* ham = nullptr;
  cudaEvent_t ev = nullptr;
  double* pin = nullptr;
  size_t pin_cap = 0;
  cudaStream_t stream = nullptr;
};

// Byte layout of a small request's arena block.
struct Layout {
  int64_t ops, coef, contrib, groups, tables, segs, pptr, pops, theta, grad, etraj, total;
};

Layout small_layout(const Req& r, int64_t n_pops) {
  Layout L{};
  int64_t o = 0;
  auto take = [&](int64_t bytes) {
    const int64_t at = o;
    o += round_up(std::max<int64_t>(bytes, 1), kUnit);
    return at;
  };
  const int64_t n_ops = (int64_t)r.hc.ops.size(), P = r.hc.n_params;
  L.ops = take(n_ops * (int64_t)sizeof(DOp));
  L.coef = take(n_ops * (int64_t)sizeof(Rot));
  L.contrib = take(n_ops * 8);
  L.groups = take((int64_t)r.hh.groups.size() * (int64_t)sizeof(DGroup));
  L.tables = take((int64_t)r.hh.tables.size() * (int64_t)sizeof(double2));
  L.segs = take((int64_t)r.segs.size() * (int64_t)sizeof(Seg));
  L.pptr = take((P + 1) * 4);
  L.pops = take(n_pops * 4);
  L.theta = take(P * 8);
  L.grad = take(P * 8);
  L.etraj = take((int64_t)r.steps * 8);
  L.total = o;
  return L;
}

double now_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace svqe

using namespace svqe;

struct sv_server {
  sv_server_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  std::map<uint64_t, std::shared_ptr<Req>> reqs;
  std::deque<uint64_t> queue;
  sv_server_stats stats{};
  // device resources of the batched path
  unsigned char* arena = nullptr;
  int64_t arena_bytes = 0;
  Arena alloc;
  BInst* d_inst = nullptr;
  BItem* d_items = nullptr;
  double* d_energy = nullptr;
  int* d_counter = nullptr;
  double2* d_ckpt = nullptr;
  BInst* h_inst = nullptr;   // pinned staging
  BItem* h_items = nullptr;
  int grid = 0;
  cudaStream_t bstream = nullptr;  // batched launches
  cudaStream_t ustream = nullptr;  // request uploads (never waits for a launch in flight)
  cudaEvent_t bev = nullptr;
  uint64_t used = 0;
  std::deque<Idle> idle;     // oldest first
  uint64_t idle_bytes = 0;
  int prio_hi = 0, prio_lo = 0;  // greatest and least stream priorities of the device
};

namespace {

sv_status fail_cuda(const char* what, cudaError_t e) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return SV_ECUDA;
}

// Upload a small request into its arena block and fill its instance record.
sv_status place_small(sv_server* s, Req& r) {
  std::vector<int32_t> pptr, pops;
  std::vector<std::vector<int32_t>> uses(r.hc.n_params);
  for (int l = 0; l < (int)r.hc.ops.size(); ++l)
    if (r.hc.ops[l].param >= 0) uses[r.hc.ops[l].param].push_back(l);
  int64_t n_pops = 0;
  for (auto& u : uses) n_pops += (int64_t)u.size();
  const Layout L = small_layout(r, n_pops);
  const int64_t blk = r.block;
  const int64_t base = blk;  // byte offset of the block in the arena
  const int64_t pops_elem = (base + L.pops) / 4;
  for (int p = 0; p < r.hc.n_params; ++p) {
    pptr.push_back((int32_t)(pops_elem + (int64_t)pops.size()));
    pops.insert(pops.end(), uses[p].begin(), uses[p].end());
  }
  pptr.push_back((int32_t)(pops_elem + (int64_t)pops.size()));
  std::vector<DGroup> groups = r.hh.groups;
  const int64_t tables_elem = (base + L.tables) / (int64_t)sizeof(double2);
  for (DGroup& g : groups) g.toff += tables_elem;
  auto up = [&](int64_t off, const void* src, size_t bytes) -> cudaError_t {
    if (!bytes) return cudaSuccess;
    return cudaMemcpyAsync(s->arena + base + off, src, bytes, cudaMemcpyHostToDevice, s->ustream);
  };
  cudaError_t e;
  if ((e = up(L.ops, r.hc.ops.data(), r.hc.ops.size() * sizeof(DOp))) != cudaSuccess ||
      (e = up(L.groups, groups.data(), groups.size() * sizeof(DGroup))) != cudaSuccess ||
      (e = up(L.tables, r.hh.tables.data(), r.hh.tables.size() * sizeof(double2))) != cudaSuccess ||
      (e = up(L.segs, r.segs.data(), r.segs.size() * sizeof(Seg))) != cudaSuccess ||
      (e = up(L.pptr, pptr.data(), pptr.size() * 4)) != cudaSuccess ||
      (e = up(L.pops, pops.data(), pops.size() * 4)) != cudaSuccess ||
      (e = up(L.theta, r.theta.data(), r.theta.size() * 8)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s->ustream)) != cudaSuccess)
    return fail_cuda("request upload", e);
  BInst B{};
  B.n = r.n;
  B.n_ops = (int)r.hc.ops.size();
  B.n_groups = (int)groups.size();
  B.n_params = r.hc.n_params;
  B.n_segs = (int)r.segs.size();
  B.n_ckpt = r.n_ckpt;
  B.ref = r.ref;
  B.op_off = (base + L.ops) / (int64_t)sizeof(DOp);
  B.coef_off = (base + L.coef) / (int64_t)sizeof(Rot);
  B.contrib_off = (base + L.contrib) / 8;
  B.grp_off = (base + L.groups) / (int64_t)sizeof(DGroup);
  B.seg_off = (base + L.segs) / (int64_t)sizeof(Seg);
  B.pp_off = (base + L.pptr) / 4;
  B.theta_off = (base + L.theta) / 8;
  B.grad_off = (base + L.grad) / 8;
  B.tab_off = tables_elem;
  B.tab_n = (int32_t)r.hh.tables.size();
  B.lr = r.lr;
  r.theta_elem = B.theta_off;
  r.etraj_elem = (base + L.etraj) / 8;
  r.rec = B;
  return SV_OK;
}

uint64_t small_footprint(const Req& r) {
  int64_t n_pops = 0;
  for (const DOp& op : r.hc.ops) n_pops += op.param >= 0;
  return (uint64_t)small_layout(r, n_pops).total;
}

uint64_t large_footprint(const Req& r) {
  const uint64_t n_ops = r.hc.ops.size();
  return sv_ctx_device_bytes(r.n) + (uint64_t)r.hh.groups.size() * sizeof(DGroup) +
         (uint64_t)r.hh.tables.size() * sizeof(double2) +
         n_ops * (sizeof(DOp) + sizeof(Rot) + 8 + (uint64_t)kRedBlocks * 8 + 2 * sizeof(FItem)) +
         (uint64_t)r.hc.n_params * 16 + (uint64_t)r.steps * 8 + 4096;
}

void finish(sv_server* s, Req& r, int state, sv_status st, const char* msg) {
  r.state = state;
  r.status = st;
  if (msg) r.err = msg;
  r.t_done = now_since(s->t0);
  if (state == Q_DONE) ++s->stats.completed;
  else if (state == Q_FAILED) ++s->stats.failed;
  else if (state == Q_CANCELLED) ++s->stats.cancelled;
}

void free_idle(Idle& d) {
  if (d.ham) sv_ham_free(d.ham);
  if (d.ctx) sv_destroy(d.ctx);
  if (d.stream) cudaStreamDestroy(d.stream);
  if (d.ev) cudaEventDestroy(d.ev);
  if (d.pin) cudaFreeHost(d.pin);
  d = Idle{};
}

// Free idle contexts of widths other than keep_n, oldest first, while `need` more bytes would
// not fit the budget.
void evict_idle(sv_server* s, uint64_t need, int keep_n) {
  for (auto it = s->idle.begin();
       it != s->idle.end() && s->used + s->idle_bytes + need > s->cfg.hbm_budget_bytes;) {
    if (it->n == keep_n) {
      ++it;
      continue;
    }
    s->idle_bytes -= it->bytes;
    free_idle(*it);
    it = s->idle.erase(it);
  }
}

void release(sv_server* s, Req& r) {
  if (r.block >= 0) {
    s->alloc.release(r.block);
    r.block = -1;
  }
  if (r.ctx && r.ham && r.ev && r.pin && !ctx_sticky(r.ctx)) {
    // keep the resources for the next request of this width
    Idle d;
    d.n = r.n;
    d.bytes = r.footprint;
    d.ctx = r.ctx;
    d.ham = r.ham;
    d.ev = r.ev;
    d.pin = r.pin;
    d.pin_cap = r.pin_cap;
    d.stream = r.stream;
    s->idle.push_back(d);
    s->idle_bytes += d.bytes;
    r.ctx = nullptr;
    r.ham = nullptr;
    r.ev = nullptr;
    r.pin = nullptr;
    r.stream = nullptr;
  }
  if (r.ham) { sv_ham_free(r.ham); r.ham = nullptr; }
  if (r.ctx) { sv_destroy(r.ctx); r.ctx = nullptr; }
  if (r.stream) { cudaStreamDestroy(r.stream); r.stream = nullptr; }
  if (r.ev) { cudaEventDestroy(r.ev); r.ev = nullptr; }
  if (r.pin) { cudaFreeHost(r.pin); r.pin = nullptr; }
  if (r.state != Q_QUEUED) s->used -= r.footprint;
  s->stats.bytes_in_use = s->used;
  // at most max_active_large idle contexts
  while ((int)s->idle.size() > s->cfg.max_active_large) {
    s->idle_bytes -= s->idle.front().bytes;
    free_idle(s->idle.front());
    s->idle.pop_front();
  }
}

// Start a large request: context, Hamiltonian, all its steps enqueued on its own stream.  An
// idle context of the same width is reused when there is one (no allocation then).
sv_status start_large(sv_server* s, Req& r) {
  for (auto it = s->idle.begin(); it != s->idle.end(); ++it) {
    if (it->n != r.n) continue;
    r.ctx = it->ctx;
    r.ham = it->ham;
    r.ev = it->ev;
    r.pin = it->pin;
    r.pin_cap = it->pin_cap;
    r.stream = it->stream;
    s->idle_bytes -= it->bytes;
    s->idle.erase(it);
    break;
  }
  sv_status st;
  cudaError_t e;
  if (!r.ctx) {
    // heavy requests on the least stream priority, mid-size ones on the greatest
    if ((e = cudaStreamCreateWithPriority(&r.stream, cudaStreamNonBlocking,
                                          r.heavy ? s->prio_lo : s->prio_hi)) != cudaSuccess)
      return fail_cuda("request stream", e);
    if ((st = sv_create(&r.ctx, r.n, r.stream)) != SV_OK) return st;
  }
  if ((st = sv_init_reference(r.ctx, r.ref)) != SV_OK) return st;
  sv_paulisum ps{r.n, (int32_t)r.hcoef.size(), r.hx.data(), r.hz.data(), r.hcoef.data()};
  if ((st = r.ham ? ham_reload(r.ctx, r.ham, &ps) : sv_ham_upload(r.ctx, &ps, &r.ham)) != SV_OK)
    return st;
  const size_t pin_n = (size_t)r.hc.n_params + (size_t)std::max(1, r.steps);
  if (r.pin_cap < pin_n) {
    if (r.pin) cudaFreeHost(r.pin);
    r.pin = nullptr;
    r.pin_cap = 0;
    if ((e = cudaMallocHost((void**)&r.pin, pin_n * sizeof(double))) != cudaSuccess)
      return fail_cuda("pinned result buffer", e);
    r.pin_cap = pin_n;
  }
  if (!r.ev && (e = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming)) != cudaSuccess)
    return fail_cuda("event", e);
  if ((st = vqe_enqueue(r.ctx, r.hc, r.ham, r.theta.data(), r.lr, r.steps, r.pin,
                        r.pin + r.hc.n_params)) != SV_OK)
    return st;
  if ((e = cudaEventRecord(r.ev, ctx_stream(r.ctx))) != cudaSuccess) return fail_cuda("record", e);
  return SV_OK;
}

// Admit queued requests that fit (lock held).
void admit(sv_server* s) {
  int running_small = 0, running_large = 0, running_heavy = 0;
  for (auto& kv : s->reqs) {
    if (kv.second->state != Q_RUNNING) continue;
    (kv.second->small ? running_small : running_large)++;
    running_heavy += kv.second->heavy;
  }
  const double t = now_since(s->t0);
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    auto rp = s->reqs[*it];
    Req& r = *rp;
    if (s->cfg.serial && running_small + running_large > 0) break;
    const bool slot = r.small ? running_small < s->cfg.max_active_small
                              : running_large < s->cfg.max_active_large &&
                                    (!r.heavy || running_heavy < s->cfg.max_active_heavy);
    // A request waiting for a slot of its own kind holds back no other kind: only requests of
    // that kind could take the slot, and they come after it in this loop anyway.
    if (!slot) {
      ++it;
      continue;
    }
    // an idle context of this width is taken over with the bytes it already holds
    uint64_t mine = 0;
    if (!r.small)
      for (const Idle& d : s->idle)
        if (d.n == r.n) {
          mine = d.bytes;
          break;
        }
    const uint64_t need = r.footprint > mine ? r.footprint - mine : 0;
    evict_idle(s, need, r.small ? -1 : r.n);
    bool fits = s->used + s->idle_bytes + need <= s->cfg.hbm_budget_bytes;
    if (fits && r.small) {
      r.block = s->alloc.alloc((int64_t)r.footprint);
      fits = r.block >= 0;
    }
    if (!fits) {
      // the budget is shared: a request that has waited long enough for room stops later
      // requests from taking it first
      if (t - r.t_submit > kStarveSeconds) break;
      ++it;
      continue;
    }
    if (!r.small) r.footprint = std::max(r.footprint, mine);
    s->used += r.footprint;
    s->stats.bytes_in_use = s->used;
    s->stats.peak_bytes_in_use = std::max(s->stats.peak_bytes_in_use, (uint64_t)s->used);
    r.state = Q_RUNNING;
    r.t_admit = t;
    it = s->queue.erase(it);
    sv_status st = r.small ? place_small(s, r) : start_large(s, r);
    if (st != SV_OK) {
      finish(s, r, Q_FAILED, st, last_error());
      release(s, r);
      s->cv_done.notify_all();
      continue;
    }
    (r.small ? running_small : running_large)++;
    running_heavy += r.heavy;
  }
}

void worker_loop(sv_server* s) {
  cudaSetDevice(s->device);
  bool tick = false;
  std::vector<std::shared_ptr<Req>> tick_reqs;
  std::vector<int> tick_steps;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    if (s->stop) {
      bool busy = tick;
      for (auto& kv : s->reqs) busy |= kv.second->state == Q_RUNNING;
      if (!busy) break;
    }
    if (!s->stop) admit(s);
    // large requests: completion by event
    for (auto& kv : s->reqs) {
      Req& r = *kv.second;
      if (r.state != Q_RUNNING || r.small) continue;
      const cudaError_t q = cudaEventQuery(r.ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        finish(s, r, Q_FAILED, SV_ECUDA, cudaGetErrorString(q));
      } else {
        std::memcpy(r.theta.data(), r.pin, r.theta.size() * sizeof(double));
        std::memcpy(r.etraj.data(), r.pin + r.hc.n_params, r.etraj.size() * sizeof(double));
        finish(s, r, Q_DONE, SV_OK, nullptr);
      }
      release(s, r);
      s->cv_done.notify_all();
    }
    // small requests: one batched launch in flight at a time
    if (tick) {
      const cudaError_t q = cudaEventQuery(s->bev);
      if (q != cudaErrorNotReady) {
        tick = false;
        for (size_t i = 0; i < tick_reqs.size(); ++i) {
          Req& r = *tick_reqs[i];
          if (q != cudaSuccess) {
            finish(s, r, Q_FAILED, SV_ECUDA, cudaGetErrorString(q));
            release(s, r);
            continue;
          }
          r.done_steps += tick_steps[i];
          if (r.done_steps >= r.steps) {
            cudaError_t e1 = cudaMemcpy(r.theta.data(), s->arena + r.theta_elem * 8,
                                        r.theta.size() * 8, cudaMemcpyDeviceToHost);
            cudaError_t e2 = cudaMemcpy(r.etraj.data(), s->arena + r.etraj_elem * 8,
                                        r.etraj.size() * 8, cudaMemcpyDeviceToHost);
            if (e1 != cudaSuccess || e2 != cudaSuccess)
              finish(s, r, Q_FAILED, SV_ECUDA, "result copy failed");
            else
              finish(s, r, Q_DONE, SV_OK, nullptr);
            release(s, r);
          }
        }
        tick_reqs.clear();
        tick_steps.clear();
        s->cv_done.notify_all();
        if (!s->stop) admit(s);
      }
    }
    if (!tick) {
      for (auto& kv : s->reqs) {
        Req& r = *kv.second;
        if (r.state == Q_RUNNING && r.small && r.done_steps < r.steps) {
          tick_reqs.push_back(kv.second);
          if ((int)tick_reqs.size() >= s->cfg.max_active_small) break;
        }
      }
      if (!tick_reqs.empty()) {
        std::vector<BInst> bi;
        std::vector<double> cost;
        for (auto& rp : tick_reqs) {
          Req& r = *rp;
          const int k = std::min(s->cfg.steps_per_tick, r.steps - r.done_steps);
          tick_steps.push_back(k);
          BInst B = r.rec;
          B.steps = k;
          B.etraj_off = r.etraj_elem + r.done_steps;
          bi.push_back(B);
          cost.push_back(r.cost * k);
        }
        const std::vector<BItem> items = batch_items(bi, cost);
        std::memcpy(s->h_inst, bi.data(), bi.size() * sizeof(BInst));
        std::memcpy(s->h_items, items.data(), items.size() * sizeof(BItem));
        BatchArgs a{};
        a.inst = s->d_inst;
        a.n_inst = (int)bi.size();
        a.items = s->d_items;
        a.n_items = (int)items.size();
        a.ops = (const DOp*)s->arena;
        a.groups = (const DGroup*)s->arena;
        a.tables = (const double2*)s->arena;
        a.segs = (const Seg*)s->arena;
        a.pptr = (const int32_t*)s->arena;
        a.pops = (const int32_t*)s->arena;
        a.theta = (double*)s->arena;
        a.energy = s->d_energy;
        a.grad = (double*)s->arena;
        a.coef = (Rot*)s->arena;
        a.contrib = (double*)s->arena;
        a.ckpt = s->d_ckpt;
        a.ckpt_slot = kCkptAmpsPerCta;
        a.smem_amps = kBatchSmemAmps;
        a.counter = s->d_counter;
        a.n_steps = -1;
        a.lr = 0.0;
        a.lr_inst = nullptr;
        a.etraj = (double*)s->arena;
        a.opt = 0;
        a.adam_m = a.adam_v = nullptr;
        a.adam_t0 = 0;
        a.beta1 = 0.9;
        a.beta2 = 0.999;
        a.eps = 1e-8;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(s->d_inst, s->h_inst, bi.size() * sizeof(BInst),
                                 cudaMemcpyHostToDevice, s->bstream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(s->d_items, s->h_items, items.size() * sizeof(BItem),
                                 cudaMemcpyHostToDevice, s->bstream)) != cudaSuccess ||
            (e = cudaMemsetAsync(s->d_counter, 0, sizeof(int), s->bstream)) != cudaSuccess ||
            (e = launch_batch(a, std::min(s->grid, (int)items.size()), batch_smem_bytes(12),
                              s->bstream)) != cudaSuccess ||
            (e = cudaEventRecord(s->bev, s->bstream)) != cudaSuccess) {
          for (auto& rp : tick_reqs) {
            finish(s, *rp, Q_FAILED, SV_ECUDA, cudaGetErrorString(e));
            release(s, *rp);
          }
          tick_reqs.clear();
          tick_steps.clear();
          s->cv_done.notify_all();
        } else {
          tick = true;
          ++s->stats.launches;
        }
      }
    }
    int running = 0;
    for (auto& kv : s->reqs) running += kv.second->state == Q_RUNNING;
    s->stats.running = running;
    s->stats.queued = (int32_t)s->queue.size();
    if (running == 0 && s->queue.empty() && !s->stop) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

}  // namespace

sv_status sv_server_create(const sv_server_config* cfg, sv_server** out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return SV_EINVAL; }
  *out = nullptr;
  sv_server* s = new (std::nothrow) sv_server();
  if (!s) { set_error("host allocation failed"); return SV_ENOMEM; }
  if (cfg) s->cfg = *cfg;
  if (!s->cfg.hbm_budget_bytes) s->cfg.hbm_budget_bytes = 4ull << 30;
  if (s->cfg.max_active_small <= 0) s->cfg.max_active_small = 4096;
  if (s->cfg.steps_per_tick <= 0) s->cfg.steps_per_tick = 1;
  if (s->cfg.max_active_large <= 0) s->cfg.max_active_large = 8;
  if (s->cfg.max_active_heavy <= 0) s->cfg.max_active_heavy = 2;
  if (s->cfg.heavy_qubits <= 0) s->cfg.heavy_qubits = 20;
  if (s->cfg.serial) {
    s->cfg.max_active_small = 1;
    s->cfg.max_active_large = 1;
    s->cfg.max_active_heavy = 1;
  }
  s->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&s->device);
  // The arena holds every resident small request (its int32 offsets cap it at 6 GiB).  Large
  // requests allocate their own buffers; admitted footprints together never exceed the budget.
  s->arena_bytes = round_up(std::min<int64_t>((int64_t)s->cfg.hbm_budget_bytes, 6ll << 30), kUnit);
  const int cap = s->cfg.max_active_small;
  cudaError_t e;
  int grid = 0;
  if ((e = batch_prepare(12, &grid)) != cudaSuccess) { delete s; return fail_cuda("batch setup", e); }
  s->grid = grid;
  if ((e = cudaDeviceGetStreamPriorityRange(&s->prio_lo, &s->prio_hi)) != cudaSuccess ||
      (e = cudaStreamCreateWithPriority(&s->bstream, cudaStreamNonBlocking, s->prio_hi)) !=
          cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->ustream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->bev, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMalloc((void**)&s->arena, s->arena_bytes)) != cudaSuccess ||
      (e = cudaMalloc((void**)&s->d_inst, cap * sizeof(BInst))) != cudaSuccess ||
      (e = cudaMalloc((void**)&s->d_items, cap * sizeof(BItem))) != cudaSuccess ||
      (e = cudaMalloc((void**)&s->d_energy, cap * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc((void**)&s->d_counter, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc((void**)&s->d_ckpt, (size_t)grid * kCkptAmpsPerCta * sizeof(double2))) !=
          cudaSuccess ||
      (e = cudaMallocHost((void**)&s->h_inst, cap * sizeof(BInst))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&s->h_items, cap * sizeof(BItem))) != cudaSuccess) {
    cudaGetLastError();
    set_error("server allocation failed: %s", cudaGetErrorString(e));
    sv_server_destroy(s);
    return SV_ENOMEM;
  }
  s->alloc.reset(s->arena_bytes);
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return SV_OK;
}

sv_status sv_server_submit(sv_server* s, const sv_instance* inst, const double* theta0,
                           int32_t n_steps, double lr, uint64_t* id) {
  clear_error();
  if (!s || !inst || !id || n_steps < 1) { set_error("bad argument"); return SV_EINVAL; }
  auto rp = std::make_shared<Req>();
  Req& r = *rp;
  sv_status st = lower_circuit(&inst->circuit, inst->circuit.n_qubits, r.hc);
  if (st != SV_OK) return st;
  r.n = r.hc.n;
  r.small = r.n <= SV_BATCH_MAX_QUBITS;
  r.heavy = !r.small && r.n >= s->cfg.heavy_qubits;
  st = lower_ham(&inst->ham, r.n, r.small ? SV_BATCH_MAX_QUBITS : 14, r.hh);
  if (st != SV_OK) return st;
  if (inst->ref >= (1ull << r.n)) { set_error("reference index out of range"); return SV_EINVAL; }
  if (r.hc.n_params > 0 && !theta0) { set_error("theta0 is NULL"); return SV_EINVAL; }
  r.steps = n_steps;
  r.lr = lr;
  r.ref = inst->ref;
  r.theta.assign(theta0, theta0 + r.hc.n_params);
  r.etraj.assign(n_steps, 0.0);
  if (r.small) {
    r.n_ckpt = segment_ops(r.hc.ops, 2, 3, r.segs);
    if (team_ckpt_amps(r.n_ckpt, r.n) * class_teams(r.n) > kCkptAmpsPerCta) {
      set_error("circuit needs %d checkpoints of 2^%d amplitudes, more than the server's "
                "scratch holds", r.n_ckpt, r.n);
      return SV_EINVAL;
    }
    r.cost = batch_instance_flops(r.hc, r.hh, r.segs) + 64.0 * r.hc.ops.size() + 1.0;
    r.footprint = small_footprint(r);
  } else {
    r.hx.assign(inst->ham.x_mask, inst->ham.x_mask + inst->ham.n_terms);
    r.hz.assign(inst->ham.z_mask, inst->ham.z_mask + inst->ham.n_terms);
    r.hcoef.assign(inst->ham.coeff, inst->ham.coeff + inst->ham.n_terms);
    r.footprint = large_footprint(r);
  }
  if (r.footprint > s->cfg.hbm_budget_bytes) {
    set_error("request needs %llu device bytes, the server's budget is %llu",
              (unsigned long long)r.footprint, (unsigned long long)s->cfg.hbm_budget_bytes);
    return SV_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r.id = s->next_id++;
    r.t_submit = now_since(s->t0);
    s->reqs[r.id] = rp;
    s->queue.push_back(r.id);
    ++s->stats.submitted;
  }
  s->cv_work.notify_one();
  *id = r.id;
  return SV_OK;
}

sv_status sv_server_wait(sv_server* s, uint64_t id, int32_t timeout_ms, double* theta_out,
                         double* energy_out, sv_request_info* info) {
  clear_error();
  if (!s) { set_error("NULL server"); return SV_EINVAL; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) { set_error("unknown request %llu", (unsigned long long)id); return SV_EINVAL; }
  std::shared_ptr<Req> rp = it->second;
  auto done = [&] { return rp->state >= Q_DONE; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    set_error("request %llu not finished after %d ms", (unsigned long long)id, timeout_ms);
    return SV_ETIMEOUT;
  }
  Req& r = *rp;
  if (info) {
    info->id = r.id;
    info->status = r.status;
    info->n_qubits = r.n;
    info->n_params = r.hc.n_params;
    info->n_steps = r.steps;
    info->footprint_bytes = r.footprint;
    info->submit_s = r.t_submit;
    info->admit_s = r.t_admit;
    info->done_s = r.t_done;
  }
  if (r.status == SV_OK) {
    if (theta_out) std::memcpy(theta_out, r.theta.data(), r.theta.size() * sizeof(double));
    if (energy_out) std::memcpy(energy_out, r.etraj.data(), r.etraj.size() * sizeof(double));
  } else {
    set_error("%s", r.err.c_str());
  }
  const sv_status st = r.status;
  s->reqs.erase(id);
  return st;
}

sv_status sv_server_cancel(sv_server* s, uint64_t id) {
  clear_error();
  if (!s) { set_error("NULL server"); return SV_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) { set_error("unknown request"); return SV_EINVAL; }
  Req& r = *it->second;
  if (r.state != Q_QUEUED) { set_error("request is running or finished"); return SV_EBUSY; }
  s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), id), s->queue.end());
  finish(s, r, Q_CANCELLED, SV_EINVAL, "cancelled");
  s->cv_done.notify_all();
  return SV_OK;
}

sv_status sv_server_get_stats(sv_server* s, sv_server_stats* out) {
  if (!s || !out) { set_error("NULL argument"); return SV_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queued = (int32_t)s->queue.size();
  return SV_OK;
}

sv_status sv_server_destroy(sv_server* s) {
  if (!s) return SV_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (uint64_t id : s->queue) {
      auto it = s->reqs.find(id);
      if (it != s->reqs.end()) finish(s, *it->second, Q_CANCELLED, SV_EINVAL, "server destroyed");
    }
    s->queue.clear();
    s->cv_done.notify_all();
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  if (s->bstream) cudaStreamSynchronize(s->bstream);
  for (Idle& d : s->idle) free_idle(d);
  s->idle.clear();
  cudaFree(s->arena);
  cudaFree(s->d_inst);
  cudaFree(s->d_items);
  cudaFree(s->d_energy);
  cudaFree(s->d_counter);
  cudaFree(s->d_ckpt);
  cudaFreeHost(s->h_inst);
  cudaFreeHost(s->h_items);
  if (s->bev) cudaEventDestroy(s->bev);
  if (s->bstream) cudaStreamDestroy(s->bstream);
  if (s->ustream) cudaStreamDestroy(s->ustream);
  cudaGetLastError();
  delete s;
  return SV_OK;
}
