// api.cu -- the C ABI of libsvqe.so (include/svqe.h): contexts, Hamiltonians, the single-state
// path and batches.  Host code only; kernels live in k_state.cu and k_batch.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "../../include/svqe.h"
#include "api_internal.h"
#include "host_compile.h"
#include "launch.h"
#include "svqe_types.h"

using namespace svqe;

// ------------------------------------------------------------------------------ handles
struct sv_ctx {
  int n = 0;
  uint64_t N = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool sticky = false;
  uint64_t ref = 0;
  double2* psi = nullptr;
  double2* lam = nullptr;
  double* epart = nullptr;    // kRedBlocks energy partials
  double* scal = nullptr;     // [0] energy
  // circuit-sized buffers, grown on demand
  DOp* ops = nullptr;
  Rot* coef = nullptr;
  double* contrib = nullptr;
  size_t ops_cap = 0, coef_cap = 0, contrib_cap = 0;
  double* gpart = nullptr;    // n_ops x kRedBlocks gradient partials
  size_t gpart_cap = 0;
  double* theta = nullptr;
  double* grad = nullptr;
  size_t theta_cap = 0, grad_cap = 0;
  double* etraj = nullptr;
  size_t etraj_cap = 0;
  FItem* items = nullptr;     // fused-pass items of the staged circuit
  size_t items_cap = 0;
  HostPlan plan;              // fused passes of the staged circuit (empty: per-op kernels)
  // psi checkpoints of commuting layers (sv_set_checkpoint_bytes): the staged circuit's fused
  // passes are planned in chunks, each either a checkpointed layer or a run of other ops
  uint64_t ck_budget = 0;
  std::vector<double2*> ck;   // one state each
  // whole-state diagonal + permutation segments (k_dp.cu) need a third state buffer
  double2* scratch = nullptr;
  bool scratch_failed = false;
  uint32_t* dp_tab = nullptr;   // permutation tables of the staged segments
  size_t dp_tab_cap = 0;
  double2* dp_phase = nullptr;  // their phase tables (written from theta every evaluation)
  size_t dp_phase_cap = 0;
  enum { CH_PASSES = 0, CH_LAYER = 1, CH_DP = 2 };
  struct Chunk {
    int kind;
    int first, count;  // ops
    int ck;            // CH_LAYER: its checkpoint buffer
    int p0, p1;        // CH_PASSES / CH_LAYER: passes [p0, p1) of plan
    DpArgs dp;         // CH_DP
  };
  std::vector<Chunk> chunks;
  int tune = 0;         // sv_set_autotune
  int tile_bits = 11;   // tile size of the staged circuit's fused passes
};

struct sv_ham {
  int n = 0;
  int device = 0;
  int n_groups = 0;
  DGroup* groups = nullptr;
  double2* tables = nullptr;
  size_t groups_cap = 0, tables_cap = 0;  // allocated records / table entries
  uint64_t bytes = 0;
  double l1 = 0.0;
};

struct sv_batch {
  int n_inst = 0;
  int nmax = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool sticky = false;
  int64_t total_params = 0;
  int64_t total_ops = 0;
  int grid = 0;
  size_t smem = 0;
  BInst* inst = nullptr;
  BItem* items = nullptr;
  int n_items = 0;
  DOp* ops = nullptr;
  DGroup* groups = nullptr;
  double2* tables = nullptr;
  Seg* segs = nullptr;
  int32_t* pptr = nullptr;
  int32_t* pops = nullptr;
  Rot* coef = nullptr;
  double* contrib = nullptr;
  double2* ckpt = nullptr;
  int64_t ckpt_slot = 0;
  int* counter = nullptr;
  double* theta = nullptr;   // owned buffers for the host-pointer entry point
  double* energy = nullptr;
  double* grad = nullptr;
  double* adam_m = nullptr;  // Adam moments (allocated on first use) and updates taken
  double* adam_v = nullptr;
  int adam_t = 0;
  double flops = 0.0;        // algorithmic FP64 flops of one run (sv_batch_cost)
  double bytes = 0.0;        // algorithmic HBM bytes of one run
  // CUDA graph of [counter reset, persistent kernel] for one set of device pointers
  cudaGraphExec_t exec = nullptr;
  const void* key[3] = {nullptr, nullptr, nullptr};
  // layout per qubit count (team class, segment widths); cls < 0: no instance of that count
  BLayout lay[SV_BATCH_MAX_QUBITS + 1];
};

// ------------------------------------------------------------------------------ helpers
#define SV_CUDA(call, handle)                                                        \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      set_error("%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      if (handle) (handle)->sticky = true;                                           \
      return SV_ECUDA;                                                               \
    }                                                                                \
  } while (0)

#define SV_CHECK_STICKY(h)                                                  \
  do {                                                                      \
    if ((h)->sticky) {                                                      \
      set_error("handle is unusable after an earlier CUDA error");          \
      return SV_ECUDA;                                                      \
    }                                                                       \
  } while (0)

template <class T>
static cudaError_t grow(T*& p, size_t& cap, size_t need) {
  if (need <= cap && p) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  size_t c = std::max<size_t>(need, 64);
  cudaError_t e = cudaMalloc((void**)&p, c * sizeof(T));
  if (e == cudaSuccess) cap = c;
  return e;
}

const char* sv_status_str(sv_status s) {
  switch (s) {
    case SV_OK: return "SV_OK";
    case SV_EINVAL: return "SV_EINVAL";
    case SV_ENOMEM: return "SV_ENOMEM";
    case SV_ECUDA: return "SV_ECUDA";
    case SV_ETIMEOUT: return "SV_ETIMEOUT";
    case SV_EUNSUPPORTED: return "SV_EUNSUPPORTED";
    case SV_EBUSY: return "SV_EBUSY";
    default: return "SV_UNKNOWN";
  }
}

const char* sv_last_error(void) { return last_error(); }
int32_t sv_abi_version(void) { return 1; }

uint64_t sv_state_bytes(int32_t n) {
  if (n < 0 || n > 62) return 0;
  return (uint64_t)16 << n;
}

uint64_t sv_ctx_device_bytes(int32_t n) {
  if (n < 1 || n > 31) return 0;
  return 2 * sv_state_bytes(n) + (uint64_t)(kRedBlocks + 8) * sizeof(double);
}

// ------------------------------------------------------------------------------ contexts
sv_status sv_create(sv_ctx** out, int32_t n, void* stream) {
  clear_error();
  if (!out) { set_error("out is NULL"); return SV_EINVAL; }
  *out = nullptr;
  if (n < 1 || n > 31) { set_error("n_qubits %d outside [1, 31]", n); return SV_EINVAL; }
  sv_ctx* c = new (std::nothrow) sv_ctx();
  if (!c) { set_error("host allocation failed"); return SV_ENOMEM; }
  c->n = n;
  c->N = 1ull << n;
  cudaGetDevice(&c->device);
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
      delete c;
      return SV_ECUDA;
    }
    c->own_stream = true;
  }
  const size_t sb = sv_state_bytes(n);
  if (cudaMalloc((void**)&c->psi, sb) != cudaSuccess ||
      cudaMalloc((void**)&c->lam, sb) != cudaSuccess ||
      cudaMalloc((void**)&c->epart, kRedBlocks * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&c->scal, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %llu bytes for %d qubits failed",
              (unsigned long long)sv_ctx_device_bytes(n), n);
    sv_destroy(c);
    return SV_ENOMEM;
  }
  c->ref = 0;
  if (fused_prepare() != cudaSuccess || dp_prepare() != cudaSuccess ||
      launch_init_basis(c->psi, n, 0, c->stream) != cudaSuccess) {
    set_error("init kernel launch failed");
    sv_destroy(c);
    return SV_ECUDA;
  }
  *out = c;
  return SV_OK;
}

sv_status sv_destroy(sv_ctx* c) {
  if (!c) return SV_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaFree(c->psi);
  cudaFree(c->lam);
  cudaFree(c->epart);
  cudaFree(c->scal);
  cudaFree(c->ops);
  cudaFree(c->coef);
  cudaFree(c->contrib);
  cudaFree(c->gpart);
  cudaFree(c->theta);
  cudaFree(c->grad);
  cudaFree(c->etraj);
  cudaFree(c->items);
  for (double2* p : c->ck) cudaFree(p);
  cudaFree(c->scratch);
  cudaFree(c->dp_tab);
  cudaFree(c->dp_phase);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
  return SV_OK;
}

// ------------------------------------------------------------------------------ Hamiltonians
static constexpr int kTableBitsState = 14;  // largest per-group table, single-state path

// Lower h for the context's register and copy it into H's device buffers, growing them only
// when the new Pauli sum needs more room than they have.
static sv_status ham_fill(sv_ctx* c, sv_ham* H, const sv_paulisum* h) {
  HostHam hh;
  sv_status st = lower_ham(h, c->n, kTableBitsState, hh);
  if (st != SV_OK) return st;
  const size_t ng = std::max<size_t>(1, hh.groups.size());
  const size_t nt = std::max<size_t>(1, hh.tables.size());
  if (grow(H->groups, H->groups_cap, ng) != cudaSuccess ||
      grow(H->tables, H->tables_cap, nt) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %llu bytes for a Hamiltonian failed",
              (unsigned long long)(ng * sizeof(DGroup) + nt * sizeof(double2)));
    return SV_ENOMEM;
  }
  H->n = c->n;
  H->device = c->device;
  H->n_groups = (int)hh.groups.size();
  H->l1 = hh.l1;
  H->bytes = H->groups_cap * sizeof(DGroup) + H->tables_cap * sizeof(double2);
  if (!hh.groups.empty())
    SV_CUDA(cudaMemcpyAsync(H->groups, hh.groups.data(), hh.groups.size() * sizeof(DGroup),
                            cudaMemcpyHostToDevice, c->stream), c);
  if (!hh.tables.empty())
    SV_CUDA(cudaMemcpyAsync(H->tables, hh.tables.data(), hh.tables.size() * sizeof(double2),
                            cudaMemcpyHostToDevice, c->stream), c);
  SV_CUDA(cudaStreamSynchronize(c->stream), c);
  return SV_OK;
}

sv_status sv_ham_upload(sv_ctx* c, const sv_paulisum* h, sv_ham** out) {
  clear_error();
  if (!c || !out) { set_error("NULL argument"); return SV_EINVAL; }
  *out = nullptr;
  SV_CHECK_STICKY(c);
  sv_ham* H = new (std::nothrow) sv_ham();
  if (!H) { set_error("host allocation failed"); return SV_ENOMEM; }
  H->device = c->device;
  const sv_status st = ham_fill(c, H, h);
  if (st != SV_OK) {
    sv_ham_free(H);
    return st;
  }
  *out = H;
  return SV_OK;
}

namespace svqe {
sv_status ham_reload(sv_ctx* c, sv_ham* H, const sv_paulisum* h) {
  clear_error();
  if (!c || !H) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  if (H->device != c->device) { set_error("Hamiltonian on another device"); return SV_EINVAL; }
  return ham_fill(c, H, h);
}
bool ctx_sticky(const sv_ctx* c) { return c->sticky; }
}  // namespace svqe

sv_status sv_ham_free(sv_ham* H) {
  if (!H) return SV_OK;
  cudaSetDevice(H->device);
  cudaFree(H->groups);
  cudaFree(H->tables);
  cudaGetLastError();
  delete H;
  return SV_OK;
}

sv_status sv_ham_info(const sv_ham* H, int32_t* n_groups, uint64_t* bytes) {
  if (!H) { set_error("NULL handle"); return SV_EINVAL; }
  if (n_groups) *n_groups = H->n_groups;
  if (bytes) *bytes = H->bytes;
  return SV_OK;
}

sv_status sv_ham_lower(const sv_paulisum* h, int32_t kmax, int32_t* n_groups, int64_t* n_table,
                       uint64_t* x, uint64_t* zu, int32_t* cls, int64_t* toff, double* table) {
  clear_error();
  if (!h || !n_groups || !n_table) { set_error("NULL argument"); return SV_EINVAL; }
  HostHam hh;
  sv_status st = lower_ham(h, 0, kmax, hh);
  if (st != SV_OK) return st;
  const int cap_g = *n_groups;
  const int64_t cap_t = *n_table;
  *n_groups = (int32_t)hh.groups.size();
  *n_table = (int64_t)hh.tables.size();
  if (x || zu || cls || toff || table) {
    if (cap_g < (int)hh.groups.size() || cap_t < (int64_t)hh.tables.size()) {
      set_error("output arrays too small (%d groups, %lld table entries needed)",
                (int)hh.groups.size(), (long long)hh.tables.size());
      return SV_EINVAL;
    }
    for (size_t g = 0; g < hh.groups.size(); ++g) {
      if (x) x[g] = hh.groups[g].x;
      if (zu) zu[g] = hh.groups[g].zu;
      if (cls) cls[g] = hh.groups[g].cls;
      if (toff) toff[g] = hh.groups[g].toff;
    }
    if (table)
      for (size_t t = 0; t < hh.tables.size(); ++t) {
        table[2 * t] = hh.tables[t].x;
        table[2 * t + 1] = hh.tables[t].y;
      }
  }
  return SV_OK;
}

sv_status sv_circuit_plan(const sv_circuit* circ, int32_t tile_bits, int32_t* n_passes,
                          int32_t* pass_of_gate) {
  clear_error();
  if (!n_passes) { set_error("NULL argument"); return SV_EINVAL; }
  HostCircuit hc;
  sv_status st = lower_circuit(circ, 0, hc);
  if (st != SV_OK) return st;
  if (tile_bits <= 0) tile_bits = fused_tile_bits();
  if (tile_bits < kMinLowBits + 4 || tile_bits > 11) {
    set_error("tile_bits %d outside [%d, 11]", tile_bits, kMinLowBits + 4);
    return SV_EINVAL;
  }
  HostPlan plan;
  plan_passes(hc.ops, hc.n, tile_bits, plan);
  *n_passes = (int32_t)plan.passes.size();
  if (pass_of_gate) {
    for (size_t p = 0; p < plan.passes.size(); ++p) {
      const FPass& P = plan.passes[p];
      for (int i = 0; i < P.n_items; ++i) {
        const FItem& it = plan.items[P.first_item + i];
        for (int g = 0; g < it.count; ++g) pass_of_gate[it.op + g] = (int32_t)p;
      }
    }
  }
  return SV_OK;
}

sv_status sv_batch_segments(const sv_circuit* circ, int32_t cap, int32_t* segs_out,
                            int32_t* n_segs, int32_t* n_ckpt, int64_t* team_scratch_amps) {
  clear_error();
  if (!n_segs || !n_ckpt) { set_error("NULL argument"); return SV_EINVAL; }
  HostCircuit hc;
  sv_status st = lower_circuit(circ, 0, hc);
  if (st != SV_OK) return st;
  std::vector<Seg> sg;
  const int nc = segment_ops(hc.ops, 2, 3, sg);  // as sv_batch_create segments each circuit
  *n_segs = (int32_t)sg.size();
  *n_ckpt = nc;
  if (team_scratch_amps) *team_scratch_amps = team_ckpt_amps(nc, hc.n);
  if (segs_out) {
    if (cap < (int32_t)sg.size()) {
      set_error("%d segments, room for %d", (int)sg.size(), cap);
      return SV_EINVAL;
    }
    for (size_t i = 0; i < sg.size(); ++i) {
      int32_t* r = segs_out + 5 * i;
      r[0] = sg[i].kind;
      r[1] = sg[i].split;
      r[2] = sg[i].first;
      r[3] = sg[i].count;
      r[4] = sg[i].ckpt;
    }
  }
  return SV_OK;
}

// ------------------------------------------------------------------------------ one state
sv_status sv_init_reference(sv_ctx* c, uint64_t b) {
  clear_error();
  if (!c) { set_error("NULL handle"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  if (b >= c->N) { set_error("basis index %llu >= 2^%d", (unsigned long long)b, c->n); return SV_EINVAL; }
  c->ref = b;
  SV_CUDA(launch_init_basis(c->psi, c->n, b, c->stream), c);
  return SV_OK;
}

// Upload a lowered circuit's ops and make sure every circuit-sized buffer fits.
static sv_status plan_circuit(sv_ctx* c, const HostCircuit& hc, int tile_bits);
static int tune_tile_bits(sv_ctx* c, const HostCircuit& hc);

sv_status svqe::stage_circuit(sv_ctx* c, const HostCircuit& hc, bool may_tune) {
  const size_t n_ops = hc.ops.size();
  SV_CUDA(grow(c->ops, c->ops_cap, n_ops), c);
  SV_CUDA(grow(c->coef, c->coef_cap, n_ops), c);
  SV_CUDA(grow(c->contrib, c->contrib_cap, n_ops), c);
  SV_CUDA(grow(c->gpart, c->gpart_cap, std::max<size_t>(1, n_ops) * kRedBlocks), c);
  SV_CUDA(grow(c->theta, c->theta_cap, (size_t)hc.n_params), c);
  SV_CUDA(grow(c->grad, c->grad_cap, (size_t)hc.n_params), c);
  if (n_ops)
    SV_CUDA(cudaMemcpyAsync(c->ops, hc.ops.data(), n_ops * sizeof(DOp), cudaMemcpyHostToDevice,
                            c->stream), c);
  int m = fused_tile_bits();
  if (may_tune && c->tune && c->n >= kFusedMinQubits && n_ops > 0) m = tune_tile_bits(c, hc);
  if (m <= 0) return SV_ECUDA;
  return plan_circuit(c, hc, m);
}

// Fused-pass plan of a staged circuit with tiles of tile_bits bits (see stage_circuit).
static sv_status plan_circuit(sv_ctx* c, const HostCircuit& hc, int tile_bits) {
  const size_t n_ops = hc.ops.size();
  c->tile_bits = tile_bits;
  c->plan.passes.clear();
  c->plan.items.clear();
  c->chunks.clear();
  if (c->n >= kFusedMinQubits && n_ops > 0) {
    // commuting layers that get a psi checkpoint: as many as the budget (and the device) allow
    std::vector<std::pair<int, int>> layers = commuting_layers(hc.ops, 2);
    const uint64_t sb = sv_state_bytes(c->n);
    size_t n_ck = std::min<size_t>(layers.size(), (size_t)(c->ck_budget / sb));
    while (c->ck.size() < n_ck) {
      double2* buf = nullptr;
      if (cudaMalloc((void**)&buf, sb) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      c->ck.push_back(buf);
    }
    n_ck = std::min(n_ck, c->ck.size());
    layers.resize(n_ck);
    std::vector<int> layer_at(n_ops, -1);
    for (size_t j = 0; j < layers.size(); ++j) layer_at[layers[j].first] = (int)j;
    // diagonal + permutation runs need the third buffer
    if (c->n >= kDpMinQubits && !c->scratch && !c->scratch_failed) {
      if (cudaMalloc((void**)&c->scratch, sb) != cudaSuccess) {
        cudaGetLastError();
        c->scratch = nullptr;
        c->scratch_failed = true;
      }
    }
    const bool use_dp = c->scratch != nullptr && c->n >= kDpMinQubits;
    std::vector<uint32_t> tabs;
    auto is_diag = [&](int t) { return t == SV_GATE_RZ || t == SV_GATE_CZ; };
    auto is_perm = [&](int t) { return t == SV_GATE_CNOT || t == SV_GATE_X; };
    // a run of RZ/CZ (at most kDpMaxRz / kDpMaxCz) then at least two CNOT/X gates, from l
    auto dp_at = [&](int l, int& split, int& len) -> bool {
      int d = l, nrz = 0, ncz = 0;
      while (d < (int)n_ops && is_diag(hc.ops[d].type) &&
             nrz + (hc.ops[d].type == SV_GATE_RZ) <= kDpMaxRz &&
             ncz + (hc.ops[d].type == SV_GATE_CZ) <= kDpMaxCz) {
        nrz += hc.ops[d].type == SV_GATE_RZ;
        ncz += hc.ops[d].type == SV_GATE_CZ;
        ++d;
      }
      int e = d;
      while (e < (int)n_ops && is_perm(hc.ops[e].type)) ++e;
      if (e - d < 2) return false;
      split = d - l;
      len = e - l;
      return true;
    };
    auto plan_chunk = [&](int kind, int first, int count, int ckid) {
      const std::vector<DOp> sub(hc.ops.begin() + first, hc.ops.begin() + first + count);
      HostPlan sp;
      plan_passes(sub, c->n, tile_bits, sp);
      sv_ctx::Chunk ch{};
      ch.kind = kind;
      ch.first = first;
      ch.count = count;
      ch.ck = ckid;
      ch.p0 = (int)c->plan.passes.size();
      const int item0 = (int)c->plan.items.size();
      for (FItem it : sp.items) {
        it.op += first;
        c->plan.items.push_back(it);
      }
      for (FPass P : sp.passes) {
        P.first_item += item0;
        c->plan.passes.push_back(P);
      }
      ch.p1 = (int)c->plan.passes.size();
      c->chunks.push_back(ch);
    };
    auto dp_chunk = [&](int first, int split, int len) {
      sv_ctx::Chunk ch{};
      ch.kind = sv_ctx::CH_DP;
      ch.first = first;
      ch.count = len;
      ch.ck = (int)(tabs.size() / kDpTableWords);  // index of the segment's tables
      DpArgs& d = ch.dp;
      d.n = c->n;
      d.N = c->N;
      for (int l = first; l < first + split; ++l) {
        const DOp& op = hc.ops[l];
        if (op.type == SV_GATE_RZ) {
          d.rz_all[d.n_rz_all++] = l;
          if (op.param >= 0) {
            d.rz_op[d.n_rz] = l;
            d.rz_bit[d.n_rz] = op.bit0;
            ++d.n_rz;
          }
        } else {
          d.cz_mask[d.n_cz++] = (uint32_t)op.lo_or;
        }
      }
      // P(k): the CNOT/X gates' conditional flips in order; tables over bits [0, 11),
      // [11, 22), [22, 31), the first holding P(0)
      auto P = [&](uint32_t k) {
        for (int l = first + split; l < first + len; ++l) {
          const uint32_t lo = (uint32_t)hc.ops[l].lo_or, fl = (uint32_t)hc.ops[l].flip;
          if ((k & lo) == lo) k ^= fl;
        }
        return k;
      };
      const uint32_t c0 = P(0);
      // delta = M^-1 e_0: the linear parts of the gates (a CNOT flips its target where its
      // control is set; an X is a constant) applied to e_0 in reverse order
      uint32_t delta = 1u;
      for (int l = first + len - 1; l >= first + split; --l) {
        const uint32_t lo = (uint32_t)hc.ops[l].lo_or, fl = (uint32_t)hc.ops[l].flip;
        if (lo && (delta & lo) == lo) delta ^= fl;
      }
      d.pair = delta >> 11;
      d.pair_hi = d.pair ? 31 - __builtin_clz(d.pair) : 0;
      for (int t = 0; t < 3; ++t)
        for (uint32_t j = 0; j < 2048; ++j) {
          const uint64_t k = (uint64_t)j << (11 * t);
          tabs.push_back(k < c->N ? (t == 0 ? P((uint32_t)k) : P((uint32_t)k) ^ c0) : 0u);
        }
      c->chunks.push_back(ch);
    };
    int i = 0, pass_start = 0;
    auto flush = [&](int end) {
      if (end > pass_start) plan_chunk(sv_ctx::CH_PASSES, pass_start, end - pass_start, -1);
    };
    while (i < (int)n_ops) {
      int split = 0, len = 0;
      if (layer_at[i] >= 0) {
        flush(i);
        const int j = layer_at[i];
        plan_chunk(sv_ctx::CH_LAYER, layers[j].first, layers[j].second, j);
        i += layers[j].second;
        pass_start = i;
      } else if (use_dp && (i == 0 || !is_diag(hc.ops[i - 1].type) || i == pass_start) &&
                 dp_at(i, split, len)) {
        flush(i);
        dp_chunk(i, split, len);
        i += len;
        pass_start = i;
      } else {
        ++i;
      }
    }
    flush((int)n_ops);
    SV_CUDA(grow(c->items, c->items_cap, std::max<size_t>(1, c->plan.items.size())), c);
    if (!c->plan.items.empty())
      SV_CUDA(cudaMemcpyAsync(c->items, c->plan.items.data(),
                              c->plan.items.size() * sizeof(FItem), cudaMemcpyHostToDevice,
                              c->stream), c);
    const size_t n_dp = tabs.size() / kDpTableWords;
    if (n_dp) {
      SV_CUDA(grow(c->dp_tab, c->dp_tab_cap, tabs.size()), c);
      SV_CUDA(grow(c->dp_phase, c->dp_phase_cap, n_dp * kDpPhaseEntries), c);
      SV_CUDA(cudaMemcpyAsync(c->dp_tab, tabs.data(), tabs.size() * sizeof(uint32_t),
                              cudaMemcpyHostToDevice, c->stream), c);
      for (sv_ctx::Chunk& ch : c->chunks) {
        if (ch.kind != sv_ctx::CH_DP) continue;
        DpArgs& d = ch.dp;
        double2* ph = c->dp_phase + (size_t)ch.ck * kDpPhaseEntries;
        d.perm = c->dp_tab + (size_t)ch.ck * kDpTableWords;
        d.phase_lo = d.phase_lo_w = ph;
        d.phase_b1 = d.phase_b1_w = ph + 2048;
        d.phase_b2 = d.phase_b2_w = ph + 3072;
      }
    }
  }
  return SV_OK;
}

// A pass that holds a single gate runs as that gate's own kernel (k_apply / k_adjoint): it
// touches only the gate's amplitudes (half the state for a CNOT, an eighth for a
// DoubleExcitation) instead of staging every tile.  Returns the op, or -1.
static int single_op(const sv_ctx* c, int p) {
  const FPass& P = c->plan.passes[p];
  if (P.n_items != 1) return -1;
  const FItem& it = c->plan.items[P.first_item];
  return it.kind == 0 ? it.op : -1;
}

// The state buffers a whole-state segment may write: psi, lambda and the scratch buffer.
static double2* free_buffer(sv_ctx* c, const double2* a, const double2* b) {
  double2* pool[3] = {c->lam, c->scratch, c->psi};
  for (double2* p : pool)
    if (p && p != a && p != b) return p;
  return nullptr;
}

// Forward pass of the staged circuit.  With chunks, psi may end in another state buffer
// (whole-state segments are out of place): *psi_out receives where it is.  save: copy psi
// into the checkpoint of every checkpointed layer before the layer runs.
static sv_status forward(sv_ctx* c, const HostCircuit& hc, const double* theta_dev, bool save,
                         double2** psi_out) {
  const int n_ops = (int)hc.ops.size();
  *psi_out = c->psi;
  SV_CUDA(launch_prep_coefs(c->ops, n_ops, theta_dev, c->coef, c->stream), c);
  if (!c->chunks.empty()) {
    double2* psi = c->psi;
    for (const sv_ctx::Chunk& ch : c->chunks) {
      if (ch.kind == sv_ctx::CH_DP) {
        double2* dst = free_buffer(c, psi, nullptr);
        SV_CUDA(launch_dp_setup(ch.dp, c->ops, theta_dev, c->stream), c);
        SV_CUDA(launch_dp_fwd(psi, dst, ch.dp, c->stream), c);
        psi = dst;
        continue;
      }
      if (save && ch.kind == sv_ctx::CH_LAYER)
        SV_CUDA(cudaMemcpyAsync(c->ck[ch.ck], psi, sv_state_bytes(c->n),
                                cudaMemcpyDeviceToDevice, c->stream), c);
      for (int p = ch.p0; p < ch.p1; ++p) {
        const int op = single_op(c, p);
        if (op >= 0)
          SV_CUDA(launch_apply_op(psi, c->n, hc.ops[op], c->coef + op, false, c->stream), c);
        else
          SV_CUDA(launch_fpass(psi, c->plan.passes[p], c->items, c->ops, c->coef, theta_dev,
                               c->stream), c);
      }
    }
    *psi_out = psi;
    return SV_OK;
  }
  for (int l = 0; l < n_ops; ++l)
    SV_CUDA(launch_apply_op(c->psi, c->n, hc.ops[l], c->coef + l, false, c->stream), c);
  return SV_OK;
}

// ------------------------------------------------------------------------------ autotuner
// The fused tile size (2^9 .. 2^11 amplitudes per tile) trades shared memory per block, and so
// occupancy, against the number of passes a circuit needs.  The tuner keys a process-wide
// cache by the circuit's structure (gate types and wires, not the angles).  The cache is
// optionally kept in the text file named by SVQE_TUNE_CACHE, one "n key bits" line per
// entry.  A miss times the forward pass with each tile size (CUDA events, the second of two
// runs) and keeps the fastest.
static std::mutex g_tune_mu;
static std::unordered_map<uint64_t, int> g_tune;
static bool g_tune_loaded = false;

static uint64_t structure_key(int n, const HostCircuit& hc) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)n;
  auto mix = [&h](uint64_t v) {
    h ^= v;
    h *= 1099511628211ull;
  };
  for (const DOp& op : hc.ops) {
    mix((uint64_t)op.type);
    mix(op.lo_or);
    mix(op.flip);
    mix((uint64_t)op.k | (uint64_t)op.sb[0] << 8 | (uint64_t)op.sb[1] << 16 |
        (uint64_t)op.sb[2] << 24 | (uint64_t)op.sb[3] << 32);
  }
  return h;
}

static int tune_tile_bits(sv_ctx* c, const HostCircuit& hc) {
  const uint64_t key = structure_key(c->n, hc);
  const char* path = std::getenv("SVQE_TUNE_CACHE");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_loaded) {
      g_tune_loaded = true;
      if (path) {
        if (FILE* f = std::fopen(path, "r")) {
          int n = 0, bits = 0;
          unsigned long long k = 0;
          while (std::fscanf(f, "%d %llu %d", &n, &k, &bits) == 3)
            if (bits >= 9 && bits <= 11) g_tune[(uint64_t)k] = bits;
          std::fclose(f);
        }
      }
    }
    const auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  // the angles do not change the passes: time with theta = 0
  if (hc.n_params > 0 &&
      cudaMemsetAsync(c->theta, 0, (size_t)hc.n_params * sizeof(double), c->stream) != cudaSuccess)
    return -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return -1;
  }
  int best = fused_tile_bits();
  float best_ms = 1e30f;
  bool ok = true;
  for (int m = 9; m <= 11 && ok; ++m) {
    ok = plan_circuit(c, hc, m) == SV_OK;
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      double2* out = nullptr;
      ok = launch_init_basis(c->psi, c->n, c->ref, c->stream) == cudaSuccess &&
           cudaEventRecord(e0, c->stream) == cudaSuccess &&
           forward(c, hc, c->theta, false, &out) == SV_OK &&
           cudaEventRecord(e1, c->stream) == cudaSuccess &&
           cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    }
    if (ok && ms < best_ms) {
      best_ms = ms;
      best = m;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return -1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  if (path) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%d %llu %d\n", c->n, (unsigned long long)key, best);
      std::fclose(f);
    }
  }
  return best;
}

sv_status sv_set_autotune(sv_ctx* c, int32_t enable) {
  clear_error();
  if (!c) { set_error("NULL handle"); return SV_EINVAL; }
  c->tune = enable ? 1 : 0;
  return SV_OK;
}

sv_status sv_tile_bits(const sv_ctx* c, int32_t* tile_bits) {
  clear_error();
  if (!c || !tile_bits) { set_error("NULL argument"); return SV_EINVAL; }
  *tile_bits = c->tile_bits;
  return SV_OK;
}

// psi = |ref>, forward, lambda = H psi, adjoint sweep; energy -> energy_dev[0], gradient ->
// grad_dev.  Everything stream-ordered on c->stream.
sv_status svqe::adjoint_core(sv_ctx* c, const HostCircuit& hc, const sv_ham* H,
                       const double* theta_dev, double* energy_dev, double* grad_dev) {
  SV_CUDA(launch_init_basis(c->psi, c->n, c->ref, c->stream), c);
  double2* psi = nullptr;
  sv_status st = forward(c, hc, theta_dev, true, &psi);
  if (st != SV_OK) return st;
  double2* lam = psi == c->lam ? c->psi : c->lam;
  SV_CUDA(launch_hpsi(psi, lam, c->n, H->groups, H->n_groups, H->tables, c->epart,
                      c->stream), c);
  SV_CUDA(launch_sum(c->epart, kRedBlocks, energy_dev, c->stream), c);
  const int n_ops = (int)hc.ops.size();
  if (!c->chunks.empty()) {
    // passes over fewer tiles than kRedBlocks launch fewer blocks: their other partials are 0
    SV_CUDA(cudaMemsetAsync(c->gpart, 0, (size_t)std::max(1, n_ops) * kRedBlocks * sizeof(double),
                            c->stream), c);
    for (int ci = (int)c->chunks.size() - 1; ci >= 0; --ci) {
      const sv_ctx::Chunk& ch = c->chunks[ci];
      if (ch.kind == sv_ctx::CH_PASSES) {
        for (int p = ch.p1 - 1; p >= ch.p0; --p) {
          const int op = single_op(c, p);
          if (op >= 0) {
            double* part = hc.ops[op].param >= 0 ? c->gpart + (size_t)op * kRedBlocks : nullptr;
            SV_CUDA(launch_adjoint_op(psi, lam, c->n, hc.ops[op], c->coef + op, part,
                                      c->stream), c);
          } else {
            SV_CUDA(launch_bpass(psi, lam, c->plan.passes[p], c->items, c->ops, c->coef,
                                 theta_dev, c->gpart, c->stream), c);
          }
        }
      } else if (ch.kind == sv_ctx::CH_LAYER) {
        // a checkpointed commuting layer: every gradient from (psi, lambda) at the layer's
        // end, then the layer un-applied to lambda alone; psi before the layer is the
        // checkpoint itself (the buffer is not needed again in this sweep)
        for (int p = ch.p0; p < ch.p1; ++p)
          SV_CUDA(launch_gpass(psi, lam, c->plan.passes[p], c->items, c->ops, c->gpart,
                               c->stream), c);
        for (int p = ch.p1 - 1; p >= ch.p0; --p)
          SV_CUDA(launch_fpass_inv(lam, c->plan.passes[p], c->items, c->ops, c->coef,
                                   theta_dev, c->stream), c);
        psi = c->ck[ch.ck];
      } else {
        // diagonal + permutation: psi gathered and un-phased into a free buffer, then lambda
        // likewise with the RZ gradients from the two un-phased states
        double2* psi_b = free_buffer(c, psi, lam);
        SV_CUDA(launch_dp_bwd_psi(psi, psi_b, ch.dp, c->stream), c);
        double2* lam_b = free_buffer(c, psi_b, lam);
        SV_CUDA(launch_dp_bwd_lam(lam, psi_b, lam_b, ch.dp, c->gpart, c->stream), c);
        psi = psi_b;
        lam = lam_b;
      }
    }
    // psi is back at the reference state; it lives in the context's psi buffer between calls
    if (psi != c->psi)
      SV_CUDA(cudaMemcpyAsync(c->psi, psi, sv_state_bytes(c->n), cudaMemcpyDeviceToDevice,
                              c->stream), c);
  } else {
    for (int l = n_ops - 1; l >= 0; --l) {
      const DOp& op = hc.ops[l];
      double* part = op.param >= 0 ? c->gpart + (size_t)l * kRedBlocks : nullptr;
      SV_CUDA(launch_adjoint_op(c->psi, c->lam, c->n, op, c->coef + l, part, c->stream), c);
    }
  }
  SV_CUDA(launch_reduce_grads(c->ops, n_ops, c->gpart, hc.n_params, c->contrib, grad_dev,
                              c->stream), c);
  return SV_OK;
}

sv_status sv_apply_circuit(sv_ctx* c, const sv_circuit* circ, const double* theta) {
  clear_error();
  if (!c) { set_error("NULL handle"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  HostCircuit hc;
  sv_status st = lower_circuit(circ, c->n, hc);
  if (st != SV_OK) return st;
  if (hc.n_params > 0 && !theta) { set_error("theta is NULL"); return SV_EINVAL; }
  if ((st = stage_circuit(c, hc)) != SV_OK) return st;
  if (hc.n_params)
    SV_CUDA(cudaMemcpyAsync(c->theta, theta, hc.n_params * sizeof(double),
                            cudaMemcpyHostToDevice, c->stream), c);
  double2* psi = nullptr;
  if ((st = forward(c, hc, c->theta, false, &psi)) != SV_OK) return st;
  if (psi != c->psi)
    SV_CUDA(cudaMemcpyAsync(c->psi, psi, sv_state_bytes(c->n), cudaMemcpyDeviceToDevice,
                            c->stream), c);
  return SV_OK;
}

sv_status sv_set_checkpoint_bytes(sv_ctx* c, uint64_t bytes) {
  clear_error();
  if (!c) { set_error("NULL handle"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  c->ck_budget = bytes;
  const size_t keep = (size_t)(bytes / sv_state_bytes(c->n));
  if (c->ck.size() > keep) {
    SV_CUDA(cudaStreamSynchronize(c->stream), c);
    while (c->ck.size() > keep) {
      cudaFree(c->ck.back());
      c->ck.pop_back();
    }
  }
  return SV_OK;
}

sv_status sv_expval_paulisum(sv_ctx* c, const sv_ham* H, double* energy_out) {
  clear_error();
  if (!c || !H || !energy_out) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  if (H->n != c->n) { set_error("Hamiltonian has %d qubits, context %d", H->n, c->n); return SV_EINVAL; }
  SV_CUDA(launch_hpsi(c->psi, nullptr, c->n, H->groups, H->n_groups, H->tables, c->epart,
                      c->stream), c);
  SV_CUDA(launch_sum(c->epart, kRedBlocks, c->scal, c->stream), c);
  SV_CUDA(cudaMemcpyAsync(energy_out, c->scal, sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream), c);
  SV_CUDA(cudaStreamSynchronize(c->stream), c);
  return SV_OK;
}

sv_status sv_adjoint_grad_dev(sv_ctx* c, const sv_circuit* circ, const double* theta_dev,
                              const sv_ham* H, double* energy_dev, double* grad_dev) {
  clear_error();
  if (!c || !H || !energy_dev) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  if (H->n != c->n) { set_error("Hamiltonian has %d qubits, context %d", H->n, c->n); return SV_EINVAL; }
  HostCircuit hc;
  sv_status st = lower_circuit(circ, c->n, hc);
  if (st != SV_OK) return st;
  if (hc.n_params > 0 && (!theta_dev || !grad_dev)) { set_error("theta/grad is NULL"); return SV_EINVAL; }
  if ((st = stage_circuit(c, hc, true)) != SV_OK) return st;
  return adjoint_core(c, hc, H, theta_dev, energy_dev, grad_dev);
}

sv_status sv_adjoint_grad(sv_ctx* c, const sv_circuit* circ, const double* theta,
                          const sv_ham* H, double* energy_out, double* grad_out) {
  clear_error();
  if (!c || !H || !energy_out) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  if (H->n != c->n) { set_error("Hamiltonian has %d qubits, context %d", H->n, c->n); return SV_EINVAL; }
  HostCircuit hc;
  sv_status st = lower_circuit(circ, c->n, hc);
  if (st != SV_OK) return st;
  if (hc.n_params > 0 && (!theta || !grad_out)) { set_error("theta/grad is NULL"); return SV_EINVAL; }
  if ((st = stage_circuit(c, hc, true)) != SV_OK) return st;
  if (hc.n_params)
    SV_CUDA(cudaMemcpyAsync(c->theta, theta, hc.n_params * sizeof(double),
                            cudaMemcpyHostToDevice, c->stream), c);
  if ((st = adjoint_core(c, hc, H, c->theta, c->scal, c->grad)) != SV_OK) return st;
  SV_CUDA(cudaMemcpyAsync(energy_out, c->scal, sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream), c);
  if (hc.n_params)
    SV_CUDA(cudaMemcpyAsync(grad_out, c->grad, hc.n_params * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream), c);
  SV_CUDA(cudaStreamSynchronize(c->stream), c);
  return SV_OK;
}

sv_status svqe::vqe_enqueue(sv_ctx* c, const HostCircuit& hc, const sv_ham* H, const double* theta_in,
                      double lr, int32_t n_steps, double* theta_out, double* energy_out) {
  sv_status st = stage_circuit(c, hc, true);
  if (st != SV_OK) return st;
  SV_CUDA(grow(c->etraj, c->etraj_cap, (size_t)std::max(1, n_steps)), c);
  if (hc.n_params)
    SV_CUDA(cudaMemcpyAsync(c->theta, theta_in, hc.n_params * sizeof(double),
                            cudaMemcpyHostToDevice, c->stream), c);
  for (int t = 0; t < n_steps; ++t) {
    if ((st = adjoint_core(c, hc, H, c->theta, c->scal, c->grad)) != SV_OK) return st;
    SV_CUDA(launch_gd_update(c->theta, c->grad, hc.n_params, lr, c->scal, c->etraj + t,
                             c->stream), c);
  }
  if (hc.n_params)
    SV_CUDA(cudaMemcpyAsync(theta_out, c->theta, hc.n_params * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream), c);
  if (energy_out && n_steps > 0)
    SV_CUDA(cudaMemcpyAsync(energy_out, c->etraj, n_steps * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream), c);
  return SV_OK;
}

cudaStream_t svqe::ctx_stream(sv_ctx* c) { return c->stream; }

sv_status vqe_step(sv_ctx* c, const sv_circuit* circ, const sv_ham* H, double* theta_inout,
                   double lr, int32_t n_steps, double* energy_out) {
  clear_error();
  if (!c || !H) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  if (n_steps < 0) { set_error("n_steps %d < 0", n_steps); return SV_EINVAL; }
  if (H->n != c->n) { set_error("Hamiltonian has %d qubits, context %d", H->n, c->n); return SV_EINVAL; }
  HostCircuit hc;
  sv_status st = lower_circuit(circ, c->n, hc);
  if (st != SV_OK) return st;
  if (hc.n_params > 0 && !theta_inout) { set_error("theta is NULL"); return SV_EINVAL; }
  if ((st = vqe_enqueue(c, hc, H, theta_inout, lr, n_steps, theta_inout, energy_out)) != SV_OK)
    return st;
  SV_CUDA(cudaStreamSynchronize(c->stream), c);
  return SV_OK;
}

sv_status sv_get_state(sv_ctx* c, void* host_out) {
  clear_error();
  if (!c || !host_out) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  SV_CUDA(cudaMemcpyAsync(host_out, c->psi, sv_state_bytes(c->n), cudaMemcpyDeviceToHost,
                          c->stream), c);
  SV_CUDA(cudaStreamSynchronize(c->stream), c);
  return SV_OK;
}

sv_status sv_set_state(sv_ctx* c, const void* host_in) {
  clear_error();
  if (!c || !host_in) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(c);
  SV_CUDA(cudaMemcpyAsync(c->psi, host_in, sv_state_bytes(c->n), cudaMemcpyHostToDevice,
                          c->stream), c);
  SV_CUDA(cudaStreamSynchronize(c->stream), c);
  return SV_OK;
}

sv_status sv_state_device_ptr(sv_ctx* c, void** psi_dev) {
  if (!c || !psi_dev) { set_error("NULL argument"); return SV_EINVAL; }
  *psi_dev = c->psi;
  return SV_OK;
}

// ------------------------------------------------------------------------------ batches
static constexpr int kTableBitsBatch = SV_BATCH_MAX_QUBITS;  // full diagonal tables allowed

// Team class of an instance (see kClassWarps).
int svqe::batch_class(int n) {
  return n <= kClassQubits[2] ? 2 : n <= kClassQubits[3] ? 3 : n <= kClassQubits[1] ? 1 : 0;
}
int svqe::class_teams(int n) { return 8 / kClassWarps[batch_class(n)]; }
BLayout svqe::default_layout(int n) { return BLayout{batch_class(n), 2, 3}; }

// Work items: one instance per team of its class (one, two, eight or four per item).  What
// sets an item's duration is the work of one thread of its slowest team, not the item's flops
// (eight 9-qubit instances on one warp each take about as long as one 12-qubit instance on
// eight warps), so instances are ordered by that estimate -- amplitudes per thread times the
// per-amplitude work of the ops and groups, plus a per-op latency term -- and items by the
// estimate of their first (slowest) instance, slowest first.
static double thread_time(const BInst& B, int cls) {
  const int team = 32 * kClassWarps[cls];
  const double per_thread = std::max(1.0, (double)(1u << B.n) / team);
  return per_thread * (6.0 * B.n_ops + 2.0 * B.n_groups + 8.0) + 150.0 * B.n_ops;
}

std::vector<BItem> svqe::batch_items(const std::vector<BInst>& bi,
                                     const std::vector<double>& cost_in, const int* cls_of_n) {
  (void)cost_in;
  const int n = (int)bi.size();
  std::vector<int> cls(n);
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    cls[i] = cls_of_n ? cls_of_n[bi[i].n] : batch_class(bi[i].n);
    cost[i] = thread_time(bi[i], cls[i]);
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  std::vector<BItem> items;
  std::vector<double> icost;
  BItem open[kNumClasses];
  int fill[kNumClasses], cap[kNumClasses];
  for (int c = 0; c < kNumClasses; ++c) {
    open[c].cls = c;
    for (int t = 0; t < 8; ++t) open[c].inst[t] = -1;
    fill[c] = 0;
    cap[c] = 8 / kClassWarps[c];
  }
  std::vector<double> first_cost(kNumClasses, 0.0);
  for (int i : order) {
    const int c = cls[i];
    if (fill[c] == 0) first_cost[c] = cost[i];
    open[c].inst[fill[c]++] = i;
    if (fill[c] == cap[c]) {
      items.push_back(open[c]);
      icost.push_back(first_cost[c]);
      fill[c] = 0;
      for (int t = 0; t < 8; ++t) open[c].inst[t] = -1;
    }
  }
  for (int c = 0; c < kNumClasses; ++c)
    if (fill[c] > 0) {
      items.push_back(open[c]);
      icost.push_back(first_cost[c]);
    }
  std::vector<int> io(items.size());
  std::iota(io.begin(), io.end(), 0);
  std::stable_sort(io.begin(), io.end(), [&](int a, int c) { return icost[a] > icost[c]; });
  std::vector<BItem> out;
  for (int k : io) out.push_back(items[k]);
  return out;
}

// FP64 flops (FMA = 2) of one instance's forward pass, lambda = H psi and adjoint sweep, as
// k_batch executes its segments: lifting rotation 12 per pair, gradient 8 per pair, H gate 8
// per pair; a diagonal segment (alone or fused with the permutation after it) 12 per
// amplitude forward and 16 + (RZ gates on bits >= 8) backward; a product layer 1 per amplitude
// forward and its gradients (8 per pair) backward; a commuting layer un-applies lambda only; groups 4 (real or imaginary table) or 8
// (complex) per amplitude plus 4 for the energy.
double svqe::batch_instance_flops(const HostCircuit& hc, const HostHam& hh,
                            const std::vector<Seg>& segs) {
  const double N = (double)(1u << hc.n);
  double f = 0.0;
  for (const Seg& s : segs) {
    for (int l = s.first; l < s.first + s.count; ++l) {
      const DOp& op = hc.ops[l];
      const double pairs = N / (double)(1u << op.k);
      const bool rot = is_param_type(op.type);
      if (s.kind == SEG_GATES) {
        if (rot) f += pairs * (12 + 24 + (op.param >= 0 ? 8 : 0));
        else if (op.type == SV_GATE_H) f += pairs * (8 + 16);
      } else if (s.kind == SEG_RLAYER) {
        f += pairs * (s.split == 1 ? 8 : 12 + 8 + 12);
      }
    }
    if (s.kind == SEG_RLAYER && s.split == 1) f += N;  // the product state, one DMUL/amp
    if (s.kind == SEG_DIAG || s.kind == SEG_DIAGPERM) {
      int hi = 0;
      for (int l = s.first; l < s.first + s.count; ++l)
        if (hc.ops[l].type == SV_GATE_RZ && hc.ops[l].bit0 >= 8) ++hi;
      f += N * (12 + 16 + hi);
    }
  }
  for (const DGroup& g : hh.groups) f += N * ((g.cls & 3) == 2 ? 8 : 4);
  f += N * 4;
  return f;
}

sv_status sv_batch_free(sv_batch* b) {
  if (!b) return SV_OK;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->inst);
  cudaFree(b->items);
  cudaFree(b->ops);
  cudaFree(b->groups);
  cudaFree(b->tables);
  cudaFree(b->segs);
  cudaFree(b->pptr);
  cudaFree(b->pops);
  cudaFree(b->coef);
  cudaFree(b->contrib);
  cudaFree(b->ckpt);
  cudaFree(b->counter);
  cudaFree(b->theta);
  cudaFree(b->energy);
  cudaFree(b->grad);
  cudaFree(b->adam_m);
  cudaFree(b->adam_v);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  cudaGetLastError();
  delete b;
  return SV_OK;
}

// Compile and upload a batch with the given layout per qubit count (lay[q] for q-qubit
// instances; a class that cannot hold a q-qubit instance falls back to the fixed rule).
static sv_status batch_build(const sv_instance* inst, int32_t n, void* stream,
                             const BLayout* lay_in, sv_batch** out) {
  *out = nullptr;
  BLayout lay[SV_BATCH_MAX_QUBITS + 1];
  int cls_of_n[SV_BATCH_MAX_QUBITS + 1];
  for (int q = 0; q <= SV_BATCH_MAX_QUBITS; ++q) {
    lay[q] = lay_in ? lay_in[q] : default_layout(q);
    if (lay[q].cls < 0 || lay[q].cls >= kNumClasses || q > kClassQubits[lay[q].cls])
      lay[q].cls = batch_class(q);
    cls_of_n[q] = lay[q].cls;
  }
  std::vector<BInst> bi(n);
  std::vector<DOp> ops;
  std::vector<DGroup> groups;
  std::vector<double2> tables;
  std::vector<Seg> segs;
  std::vector<int32_t> pptr, pops;
  std::vector<double> cost(n);
  double flops = 0.0, bytes = 0.0;
  int nmax = 1;
  int64_t theta_off = 0, ckpt_slot = 1;
  for (int i = 0; i < n; ++i) {
    const sv_instance& I = inst[i];
    if (I.circuit.n_qubits < 1 || I.circuit.n_qubits > SV_BATCH_MAX_QUBITS) {
      set_error("instance %d: n_qubits %d outside [1, %d]", i, I.circuit.n_qubits,
                SV_BATCH_MAX_QUBITS);
      return SV_EINVAL;
    }
    HostCircuit hc;
    sv_status st = lower_circuit(&I.circuit, I.circuit.n_qubits, hc);
    if (st != SV_OK) return st;
    HostHam hh;
    if ((st = lower_ham(&I.ham, I.circuit.n_qubits, kTableBitsBatch, hh)) != SV_OK) return st;
    if (I.ref >= (1ull << hc.n)) { set_error("instance %d: reference index out of range", i); return SV_EINVAL; }
    std::vector<Seg> sg;
    const int n_ckpt = segment_ops(hc.ops, lay[hc.n].min_layer, lay[hc.n].min_diag_rz, sg);
    const double inst_flops = batch_instance_flops(hc, hh, sg);
    flops += inst_flops;
    bytes += (double)hc.ops.size() * (sizeof(DOp) + sizeof(Rot) * 2 + 2 * sizeof(double)) +
             (double)hh.groups.size() * sizeof(DGroup) +
             (double)hh.tables.size() * sizeof(double2) + 3.0 * 8 * hc.n_params + 8 +
             2.0 * n_ckpt * sizeof(double2) * (double)(1u << hc.n);
    for (const Seg& g : sg)  // saved diagonal + permutation tables, written and read once
      if (g.kind == SEG_DIAGPERM) bytes += 2.0 * kDpAuxAmps * sizeof(double2);
    BInst& B = bi[i];
    B = BInst{};
    B.n = hc.n;
    B.n_ops = (int)hc.ops.size();
    B.n_groups = (int)hh.groups.size();
    B.n_params = hc.n_params;
    B.n_segs = (int)sg.size();
    B.n_ckpt = n_ckpt;
    B.ref = I.ref;
    B.op_off = (int64_t)ops.size();
    B.coef_off = B.op_off;
    B.contrib_off = B.op_off;
    B.grp_off = (int64_t)groups.size();
    B.theta_off = theta_off;
    B.grad_off = theta_off;
    B.seg_off = (int64_t)segs.size();
    B.pp_off = (int64_t)pptr.size();
    theta_off += hc.n_params;
    // a CTA's checkpoint region is split evenly among the teams of the instance's class
    ckpt_slot = std::max<int64_t>(ckpt_slot, team_ckpt_amps(n_ckpt, hc.n) *
                                                  (8 / kClassWarps[lay[hc.n].cls]));
    segs.insert(segs.end(), sg.begin(), sg.end());
    // parameter -> ops using it, in op order (CSR)
    std::vector<std::vector<int32_t>> uses(hc.n_params);
    for (int l = 0; l < (int)hc.ops.size(); ++l)
      if (hc.ops[l].param >= 0) uses[hc.ops[l].param].push_back(l);
    for (int p = 0; p < hc.n_params; ++p) {
      pptr.push_back((int32_t)pops.size());
      pops.insert(pops.end(), uses[p].begin(), uses[p].end());
    }
    pptr.push_back((int32_t)pops.size());
    const int64_t toff0 = (int64_t)tables.size();
    B.tab_off = toff0;
    B.tab_n = (int32_t)hh.tables.size();
    for (DGroup g : hh.groups) {
      g.toff += toff0;
      groups.push_back(g);
    }
    tables.insert(tables.end(), hh.tables.begin(), hh.tables.end());
    ops.insert(ops.end(), hc.ops.begin(), hc.ops.end());
    nmax = std::max(nmax, hc.n);
    cost[i] = inst_flops + 64.0 * B.n_ops + 1.0;  // per-op latency matters for tiny states
  }
  sv_batch* b = new (std::nothrow) sv_batch();
  if (!b) { set_error("host allocation failed"); return SV_ENOMEM; }
  b->n_inst = n;
  b->nmax = nmax;
  b->flops = flops;
  b->bytes = bytes;
  b->total_params = theta_off;
  b->total_ops = (int64_t)ops.size();
  cudaGetDevice(&b->device);
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { set_error("cudaStreamCreate: %s", cudaGetErrorString(e)); delete b; return SV_ECUDA; }
    b->own_stream = true;
  }
  const std::vector<BItem> items = batch_items(bi, cost, cls_of_n);
  b->n_items = (int)items.size();
  for (int q = 0; q <= SV_BATCH_MAX_QUBITS; ++q) b->lay[q] = BLayout{-1, 0, 0};
  for (int i = 0; i < n; ++i) b->lay[bi[i].n] = lay[bi[i].n];
  auto alloc = [&](void** p, size_t bytes) {
    return cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess;
  };
  const size_t P = (size_t)std::max<int64_t>(theta_off, 1);
  if (!alloc((void**)&b->inst, n * sizeof(BInst)) ||
      !alloc((void**)&b->items, items.size() * sizeof(BItem)) ||
      !alloc((void**)&b->ops, ops.size() * sizeof(DOp)) ||
      !alloc((void**)&b->groups, groups.size() * sizeof(DGroup)) ||
      !alloc((void**)&b->tables, tables.size() * sizeof(double2)) ||
      !alloc((void**)&b->segs, segs.size() * sizeof(Seg)) ||
      !alloc((void**)&b->pptr, pptr.size() * sizeof(int32_t)) ||
      !alloc((void**)&b->pops, pops.size() * sizeof(int32_t)) ||
      !alloc((void**)&b->coef, ops.size() * sizeof(Rot)) ||
      !alloc((void**)&b->contrib, ops.size() * sizeof(double)) ||
      !alloc((void**)&b->counter, sizeof(int)) || !alloc((void**)&b->theta, P * sizeof(double)) ||
      !alloc((void**)&b->energy, n * sizeof(double)) || !alloc((void**)&b->grad, P * sizeof(double))) {
    cudaGetLastError();
    set_error("device allocation for a batch of %d instances failed", n);
    sv_batch_free(b);
    return SV_ENOMEM;
  }
  auto up = [&](void* d, const void* h, size_t bytes) {
    return bytes == 0 ? cudaSuccess
                      : cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, b->stream);
  };
  cudaError_t e = cudaSuccess;
  if ((e = up(b->inst, bi.data(), n * sizeof(BInst))) != cudaSuccess ||
      (e = up(b->items, items.data(), items.size() * sizeof(BItem))) != cudaSuccess ||
      (e = up(b->ops, ops.data(), ops.size() * sizeof(DOp))) != cudaSuccess ||
      (e = up(b->groups, groups.data(), groups.size() * sizeof(DGroup))) != cudaSuccess ||
      (e = up(b->tables, tables.data(), tables.size() * sizeof(double2))) != cudaSuccess ||
      (e = up(b->segs, segs.data(), segs.size() * sizeof(Seg))) != cudaSuccess ||
      (e = up(b->pptr, pptr.data(), pptr.size() * sizeof(int32_t))) != cudaSuccess ||
      (e = up(b->pops, pops.data(), pops.size() * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaStreamSynchronize(b->stream)) != cudaSuccess ||
      (e = batch_prepare(nmax, &b->grid)) != cudaSuccess) {
    set_error("batch upload failed: %s", cudaGetErrorString(e));
    sv_batch_free(b);
    return SV_ECUDA;
  }
  b->grid = std::min(b->grid, b->n_items);
  b->smem = batch_smem_bytes(nmax);
  b->ckpt_slot = ckpt_slot;
  if (!alloc((void**)&b->ckpt, (size_t)b->grid * ckpt_slot * sizeof(double2))) {
    cudaGetLastError();
    set_error("device allocation of %llu checkpoint bytes failed",
              (unsigned long long)((size_t)b->grid * ckpt_slot * sizeof(double2)));
    sv_batch_free(b);
    return SV_ENOMEM;
  }
  *out = b;
  return SV_OK;
}

// ------------------------------------------------------------------------------ layout tuner
// The batched kernel's layout for q-qubit instances (BLayout) trades threads per instance
// against instances per CTA, and per-segment set-up work (tables, checkpoints, staged gates)
// against per-gate passes; which wins depends on q.  With sv_batch_set_autotune(1),
// sv_batch_create measures, for every qubit count of the batch that the process-wide cache
// does not hold yet, each candidate layout (the smallest team that holds the instance and the
// next larger one, times commuting-layer segments on or off, times diagonal segments on or off)
// on a calibration batch: that count's instances of the batch, repeated to give every CTA two
// items.  One warm-up and three timed runs of the persistent launch (CUDA events on the batch's
// stream); the fastest layout is kept.  The cache is optionally kept in the text file named by
// SVQE_BATCH_TUNE_CACHE, one "q cls min_layer min_diag_rz" line per qubit count.
static std::mutex g_btune_mu;
static std::map<int, BLayout> g_btune;
static bool g_btune_loaded = false;
static std::atomic<int> g_batch_tune{0};
constexpr int kSegOff = 1 << 20;  // a width no run reaches: that segment kind is not used

static sv_status time_batch(sv_batch* b, float* best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaSuccess;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    set_error("cudaEventCreate: %s", cudaGetErrorString(e));
    return SV_ECUDA;
  }
  sv_status st = SV_OK;
  if (cudaMemsetAsync(b->theta, 0, (size_t)std::max<int64_t>(b->total_params, 1) * 8,
                      b->stream) != cudaSuccess) {
    set_error("tuner: theta reset failed");
    st = SV_ECUDA;
  }
  *best_ms = 1e30f;
  for (int rep = 0; rep < 4 && st == SV_OK; ++rep) {
    float ms = 0.0f;
    if (cudaEventRecord(e0, b->stream) != cudaSuccess ||
        (st = sv_batch_run_dev(b, b->theta, b->energy, b->grad)) != SV_OK ||
        cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      if (st == SV_OK) {
        set_error("tuner: timing failed");
        st = SV_ECUDA;
      }
      break;
    }
    if (rep > 0) *best_ms = std::min(*best_ms, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

static sv_status tune_layouts(const sv_instance* inst, int32_t n, void* stream, BLayout* lay) {
  std::vector<int> by_q[SV_BATCH_MAX_QUBITS + 1];
  for (int i = 0; i < n; ++i) {
    const int q = inst[i].circuit.n_qubits;
    if (q >= 1 && q <= SV_BATCH_MAX_QUBITS) by_q[q].push_back(i);
  }
  const char* path = std::getenv("SVQE_BATCH_TUNE_CACHE");
  {
    std::lock_guard<std::mutex> lk(g_btune_mu);
    if (!g_btune_loaded) {
      g_btune_loaded = true;
      if (path) {
        if (FILE* f = std::fopen(path, "r")) {
          int q = 0, c = 0, ml = 0, md = 0;
          while (std::fscanf(f, "%d %d %d %d", &q, &c, &ml, &md) == 4)
            if (q >= 1 && q <= SV_BATCH_MAX_QUBITS && c >= 0 && c < kNumClasses &&
                q <= kClassQubits[c] && ml >= 1 && md >= 1)
              g_btune[q] = BLayout{c, ml, md};
          std::fclose(f);
        }
      }
    }
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_error("cudaDeviceGetAttribute failed");
    return SV_ECUDA;
  }
  for (int q = 1; q <= SV_BATCH_MAX_QUBITS; ++q) {
    if (by_q[q].empty()) continue;
    {
      std::lock_guard<std::mutex> lk(g_btune_mu);
      const auto it = g_btune.find(q);
      if (it != g_btune.end()) {
        lay[q] = it->second;
        continue;
      }
    }
    // candidate team classes: the fixed rule's, and the class with twice its warps if it exists
    std::vector<int> classes{batch_class(q)};
    for (int c = 0; c < kNumClasses; ++c)
      if (kClassWarps[c] == 2 * kClassWarps[classes[0]]) classes.push_back(c);
    const int teams = 8 / kClassWarps[classes[0]];
    const int m = 2 * sms * teams;
    std::vector<sv_instance> cal(m);
    for (int k = 0; k < m; ++k) cal[k] = inst[by_q[q][k % by_q[q].size()]];
    BLayout best = default_layout(q);
    float best_ms = 1e30f;
    for (int c : classes)
      for (int ml : {2, kSegOff})
        for (int md : {3, kSegOff}) {
          BLayout L[SV_BATCH_MAX_QUBITS + 1];
          for (int r = 0; r <= SV_BATCH_MAX_QUBITS; ++r) L[r] = default_layout(r);
          L[q] = BLayout{c, ml, md};
          sv_batch* b = nullptr;
          sv_status st = batch_build(cal.data(), m, stream, L, &b);
          if (st == SV_ENOMEM) {  // a layout that does not fit is not a candidate
            cudaGetLastError();
            continue;
          }
          if (st != SV_OK) return st;
          float ms = 0.0f;
          st = time_batch(b, &ms);
          sv_batch_free(b);
          if (st != SV_OK) return st;
          if (ms < best_ms) {
            best_ms = ms;
            best = L[q];
          }
        }
    lay[q] = best;
    std::lock_guard<std::mutex> lk(g_btune_mu);
    g_btune[q] = best;
    if (path) {
      if (FILE* f = std::fopen(path, "a")) {
        std::fprintf(f, "%d %d %d %d\n", q, best.cls, best.min_layer, best.min_diag_rz);
        std::fclose(f);
      }
    }
  }
  return SV_OK;
}

sv_status sv_batch_set_autotune(int32_t enable) {
  clear_error();
  g_batch_tune.store(enable ? 1 : 0);
  return SV_OK;
}

sv_status sv_batch_set_layout(int32_t n_qubits, int32_t team_warps, int32_t min_layer,
                              int32_t min_diag_rz) {
  clear_error();
  if (n_qubits < 1 || n_qubits > SV_BATCH_MAX_QUBITS) {
    set_error("n_qubits %d outside [1, %d]", n_qubits, SV_BATCH_MAX_QUBITS);
    return SV_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_btune_mu);
  if (team_warps == 0) {
    g_btune.erase(n_qubits);
    return SV_OK;
  }
  int cls = -1;
  for (int c = 0; c < kNumClasses; ++c)
    if (kClassWarps[c] == team_warps) cls = c;
  if (cls < 0 || n_qubits > kClassQubits[cls] || min_layer < 1 || min_diag_rz < 1) {
    set_error("layout (%d warps, widths %d, %d) cannot run %d-qubit instances", team_warps,
              min_layer, min_diag_rz, n_qubits);
    return SV_EINVAL;
  }
  g_btune[n_qubits] = BLayout{cls, min_layer, min_diag_rz};
  return SV_OK;
}

sv_status sv_batch_layout(const sv_batch* b, int32_t n_qubits, int32_t* team_warps,
                          int32_t* min_layer, int32_t* min_diag_rz) {
  clear_error();
  if (!b || n_qubits < 1 || n_qubits > SV_BATCH_MAX_QUBITS) {
    set_error("NULL handle or n_qubits %d outside [1, %d]", n_qubits, SV_BATCH_MAX_QUBITS);
    return SV_EINVAL;
  }
  const BLayout& L = b->lay[n_qubits];
  const bool used = L.cls >= 0;
  if (team_warps) *team_warps = used ? kClassWarps[L.cls] : 0;
  if (min_layer) *min_layer = used ? L.min_layer : 0;
  if (min_diag_rz) *min_diag_rz = used ? L.min_diag_rz : 0;
  return SV_OK;
}

sv_status sv_batch_create(const sv_instance* inst, int32_t n, void* stream, sv_batch** out) {
  clear_error();
  if (!out || (n > 0 && !inst) || n < 1) { set_error("bad arguments (n = %d)", n); return SV_EINVAL; }
  *out = nullptr;
  BLayout lay[SV_BATCH_MAX_QUBITS + 1];
  for (int q = 0; q <= SV_BATCH_MAX_QUBITS; ++q) lay[q] = default_layout(q);
  if (g_batch_tune.load()) {
    for (int i = 0; i < n; ++i)  // invalid instances are reported by batch_build, untuned
      if (inst[i].circuit.n_qubits < 1 || inst[i].circuit.n_qubits > SV_BATCH_MAX_QUBITS)
        return batch_build(inst, n, stream, lay, out);
    const sv_status st = tune_layouts(inst, n, stream, lay);
    if (st != SV_OK) return st;
  }
  return batch_build(inst, n, stream, lay, out);
}

sv_status sv_batch_cost(const sv_batch* b, double* fp64_flops, double* hbm_bytes) {
  if (!b) { set_error("NULL handle"); return SV_EINVAL; }
  if (fp64_flops) *fp64_flops = b->flops;
  if (hbm_bytes) *hbm_bytes = b->bytes;
  return SV_OK;
}

sv_status sv_batch_info(const sv_batch* b, int32_t* n_inst, int64_t* n_params) {
  if (!b) { set_error("NULL handle"); return SV_EINVAL; }
  if (n_inst) *n_inst = b->n_inst;
  if (n_params) *n_params = b->total_params;
  return SV_OK;
}

static BatchArgs batch_args(sv_batch* b, double* theta, double* energy, double* grad,
                            int n_steps, double lr, double* etraj) {
  BatchArgs a;
  a.inst = b->inst;
  a.items = b->items;
  a.n_items = b->n_items;
  a.smem_amps = kBatchSmemAmps;
  a.n_inst = b->n_inst;
  a.ops = b->ops;
  a.groups = b->groups;
  a.tables = b->tables;
  a.segs = b->segs;
  a.pptr = b->pptr;
  a.pops = b->pops;
  a.ckpt = b->ckpt;
  a.ckpt_slot = b->ckpt_slot;
  a.theta = theta;
  a.energy = energy;
  a.grad = grad;
  a.coef = b->coef;
  a.contrib = b->contrib;
  a.counter = b->counter;
  a.n_steps = n_steps;
  a.lr = lr;
  a.lr_inst = nullptr;
  a.etraj = etraj;
  a.opt = 0;
  a.adam_m = nullptr;
  a.adam_v = nullptr;
  a.adam_t0 = 0;
  a.beta1 = 0.9;
  a.beta2 = 0.999;
  a.eps = 1e-8;
  return a;
}

sv_status sv_batch_run_dev(sv_batch* b, const double* theta_dev, double* energy_dev,
                           double* grad_dev) {
  clear_error();
  if (!b || !theta_dev || !energy_dev || !grad_dev) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(b);
  if (b->stream == cudaStreamLegacy || b->stream == cudaStreamPerThread) {
    // default streams cannot be captured: launch directly
    SV_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream), b);
    SV_CUDA(launch_batch(batch_args(b, const_cast<double*>(theta_dev), energy_dev, grad_dev, 0,
                                    0.0, nullptr), b->grid, b->smem, b->stream), b);
    return SV_OK;
  }
  const void* key[3] = {theta_dev, energy_dev, grad_dev};
  if (!b->exec || std::memcmp(key, b->key, sizeof key) != 0) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    cudaGraph_t g = nullptr;
    SV_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), b);
    cudaError_t e1 = cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream);
    cudaError_t e2 = launch_batch(batch_args(b, const_cast<double*>(theta_dev), energy_dev,
                                             grad_dev, 0, 0.0, nullptr),
                                  b->grid, b->smem, b->stream);
    cudaError_t e3 = cudaStreamEndCapture(b->stream, &g);
    SV_CUDA(e1, b);
    SV_CUDA(e2, b);
    SV_CUDA(e3, b);
    cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    SV_CUDA(e, b);
    std::memcpy(b->key, key, sizeof key);
  }
  SV_CUDA(cudaGraphLaunch(b->exec, b->stream), b);
  return SV_OK;
}

sv_status sv_batch_run(sv_batch* b, const double* theta, double* energy, double* grad) {
  clear_error();
  if (!b || (b->total_params > 0 && (!theta || !grad)) || !energy) { set_error("NULL argument"); return SV_EINVAL; }
  SV_CHECK_STICKY(b);
  if (b->total_params)
    SV_CUDA(cudaMemcpyAsync(b->theta, theta, b->total_params * sizeof(double),
                            cudaMemcpyHostToDevice, b->stream), b);
  sv_status st = sv_batch_run_dev(b, b->theta, b->energy, b->grad);
  if (st != SV_OK) return st;
  SV_CUDA(cudaMemcpyAsync(energy, b->energy, b->n_inst * sizeof(double), cudaMemcpyDeviceToHost,
                          b->stream), b);
  if (b->total_params)
    SV_CUDA(cudaMemcpyAsync(grad, b->grad, b->total_params * sizeof(double),
                            cudaMemcpyDeviceToHost, b->stream), b);
  SV_CUDA(cudaStreamSynchronize(b->stream), b);
  return SV_OK;
}

sv_status sv_batch_adam_dev(sv_batch* b, double* theta_dev, double lr, int32_t n_steps,
                            double* energy_traj_dev, int32_t reset) {
  clear_error();
  if (!b || !theta_dev) { set_error("NULL argument"); return SV_EINVAL; }
  if (n_steps < 1) { set_error("n_steps %d < 1", n_steps); return SV_EINVAL; }
  SV_CHECK_STICKY(b);
  const size_t P = (size_t)std::max<int64_t>(b->total_params, 1);
  if (!b->adam_m) {
    if (cudaMalloc((void**)&b->adam_m, P * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&b->adam_v, P * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of Adam moments failed");
      return SV_ENOMEM;
    }
    reset = 1;
  }
  if (reset) {
    SV_CUDA(cudaMemsetAsync(b->adam_m, 0, P * sizeof(double), b->stream), b);
    SV_CUDA(cudaMemsetAsync(b->adam_v, 0, P * sizeof(double), b->stream), b);
    b->adam_t = 0;
  }
  BatchArgs a = batch_args(b, theta_dev, b->energy, b->grad, n_steps, lr, energy_traj_dev);
  a.opt = 1;
  a.adam_m = b->adam_m;
  a.adam_v = b->adam_v;
  a.adam_t0 = b->adam_t;
  SV_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream), b);
  SV_CUDA(launch_batch(a, b->grid, b->smem, b->stream), b);
  b->adam_t += n_steps;
  return SV_OK;
}

sv_status sv_batch_vqe_dev(sv_batch* b, double* theta_dev, double lr, int32_t n_steps,
                           double* energy_traj_dev) {
  clear_error();
  if (!b || !theta_dev) { set_error("NULL argument"); return SV_EINVAL; }
  if (n_steps < 1) { set_error("n_steps %d < 1", n_steps); return SV_EINVAL; }
  SV_CHECK_STICKY(b);
  SV_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream), b);
  SV_CUDA(launch_batch(batch_args(b, theta_dev, b->energy, b->grad, n_steps, lr,
                                  energy_traj_dev), b->grid, b->smem, b->stream), b);
  return SV_OK;
}

