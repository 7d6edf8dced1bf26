// host_compile.cpp -- validation and lowering of circuits and Pauli sums (host C++).
//
// Circuits: each sv_gate becomes a DOp whose amplitude pairs are enumerated by inserting zero
// bits at the gate's sorted wire bits (qubit q <-> basis-index bit n-1-q).
// Pauli sums (Sec. 3.2, the Jordan-Wigner sum H = sum_t c_t P_t): terms are grouped by their
// X-flip mask x, because every term of a group maps |k> to the same |k ^ x>.  A group's
// coefficient function is tabulated with a fast Walsh-Hadamard transform over the bits its z
// masks touch.
#include "host_compile.h"

#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "svqe_types.h"

namespace svqe {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }
const char* last_error() { return g_err.c_str(); }

static int n_wires(int type) {
  switch (type) {
    case SV_GATE_X: case SV_GATE_H: case SV_GATE_RX: case SV_GATE_RY: case SV_GATE_RZ:
      return 1;
    case SV_GATE_CNOT: case SV_GATE_SINGLE_EXC: case SV_GATE_CZ:
      return 2;
    case SV_GATE_DOUBLE_EXC:
      return 4;
    default:
      return -1;
  }
}

sv_status lower_circuit(const sv_circuit* c, int expect_n, HostCircuit& out) {
  if (!c) { set_error("circuit is NULL"); return SV_EINVAL; }
  if (c->n_qubits < 1 || c->n_qubits > 31) {
    set_error("n_qubits %d outside [1, 31]", c->n_qubits);
    return SV_EINVAL;
  }
  if (expect_n > 0 && c->n_qubits != expect_n) {
    set_error("circuit has %d qubits, context has %d", c->n_qubits, expect_n);
    return SV_EINVAL;
  }
  if (c->n_gates < 0 || (c->n_gates > 0 && !c->gates) || c->n_params < 0) {
    set_error("bad gate array (n_gates %d, n_params %d)", c->n_gates, c->n_params);
    return SV_EINVAL;
  }
  const int n = c->n_qubits;
  out.n = n;
  out.n_params = c->n_params;
  out.ops.clear();
  out.ops.reserve(c->n_gates);
  for (int g = 0; g < c->n_gates; ++g) {
    const sv_gate& G = c->gates[g];
    const int k = n_wires(G.type);
    if (k < 0) { set_error("gate %d: unknown type %d", g, G.type); return SV_EINVAL; }
    if (k > n) { set_error("gate %d: needs %d wires, register has %d", g, k, n); return SV_EINVAL; }
    int bits[4];
    for (int a = 0; a < k; ++a) {
      if (G.wires[a] < 0 || G.wires[a] >= n) {
        set_error("gate %d: wire %d out of range [0, %d)", g, G.wires[a], n);
        return SV_EINVAL;
      }
      for (int b = 0; b < a; ++b)
        if (G.wires[a] == G.wires[b]) { set_error("gate %d: duplicate wire %d", g, G.wires[a]); return SV_EINVAL; }
      bits[a] = n - 1 - G.wires[a];
    }
    const bool pg = is_param_type(G.type);
    if (pg) {
      if (G.param < -1 || G.param >= c->n_params) {
        set_error("gate %d: parameter index %d outside [-1, %d)", g, G.param, c->n_params);
        return SV_EINVAL;
      }
      if (G.param < 0 && !std::isfinite(G.fixed_angle)) {
        set_error("gate %d: fixed angle is not finite", g);
        return SV_EINVAL;
      }
    }
    DOp op{};
    op.type = G.type;
    op.param = pg ? G.param : -1;
    op.fixed = pg ? G.fixed_angle : 0.0;
    op.bit0 = bits[0];
    int sb[4] = {0, 0, 0, 0};
    for (int a = 0; a < k; ++a) sb[a] = bits[a];
    std::sort(sb, sb + k);
    for (int a = 0; a < 4; ++a) op.sb[a] = (uint8_t)(a < k ? sb[a] : 0);
    const uint64_t b0 = 1ull << bits[0];
    switch (G.type) {
      case SV_GATE_X: case SV_GATE_H: case SV_GATE_RX: case SV_GATE_RY: case SV_GATE_RZ:
        op.k = 1; op.lo_or = 0; op.flip = b0;
        break;
      case SV_GATE_CNOT:  // control bits[0] = 1, target bits[1] swapped
        op.k = 2; op.lo_or = b0; op.flip = 1ull << bits[1];
        break;
      case SV_GATE_CZ:  // both 1: a single amplitude, negated
        op.k = 2; op.lo_or = b0 | (1ull << bits[1]); op.flip = 0;
        break;
      case SV_GATE_SINGLE_EXC:  // lo = |01> on (w0, w1), hi = |10>
        op.k = 2; op.lo_or = 1ull << bits[1]; op.flip = b0 | (1ull << bits[1]);
        break;
      case SV_GATE_DOUBLE_EXC:  // lo = |0011> on (w0..w3), hi = |1100>
        op.k = 4;
        op.lo_or = (1ull << bits[2]) | (1ull << bits[3]);
        op.flip = b0 | (1ull << bits[1]) | (1ull << bits[2]) | (1ull << bits[3]);
        break;
    }
    out.ops.push_back(op);
  }
  return SV_OK;
}

int segment_ops(std::vector<DOp>& ops, int min_layer, int min_diag_rz,
                std::vector<Seg>& segs) {
  segs.clear();
  int ckpt = 0;
  const int n_ops = (int)ops.size();
  auto push_gates = [&](int first, int count) {
    if (count <= 0) return;
    if (!segs.empty() && segs.back().kind == SEG_GATES &&
        segs.back().first + segs.back().count == first) {
      segs.back().count += count;
    } else {
      segs.push_back(Seg{SEG_GATES, 0, first, count, -1});
    }
  };
  int l = 0;
  while (l < n_ops) {
    const int t = ops[l].type;
    if (t == SV_GATE_RZ || t == SV_GATE_CZ) {
      int e = l, n_rz = 0, n_cz = 0;
      while (e < n_ops && (ops[e].type == SV_GATE_RZ || ops[e].type == SV_GATE_CZ) &&
             n_rz + (ops[e].type == SV_GATE_RZ) <= kMaxLayer &&
             n_cz + (ops[e].type == SV_GATE_CZ) <= kMaxLayer) {
        n_rz += ops[e].type == SV_GATE_RZ;
        n_cz += ops[e].type == SV_GATE_CZ;
        ++e;
      }
      if (n_rz >= min_diag_rz) segs.push_back(Seg{SEG_DIAG, 0, l, e - l, ckpt++});
      else push_gates(l, e - l);
      l = e;
    } else if (t == SV_GATE_RY || t == SV_GATE_RX) {
      uint64_t used = 0;
      int e = l;
      while (e < n_ops && ops[e].type == t && !(used & (1ull << ops[e].bit0)) &&
             e - l < kMaxLayer) {
        used |= 1ull << ops[e].bit0;
        ++e;
      }
      if (e - l >= min_layer) segs.push_back(Seg{SEG_RLAYER, 0, l, e - l, ckpt++});
      else push_gates(l, e - l);
      l = e;
    } else if (t == SV_GATE_CNOT || t == SV_GATE_X) {
      int e = l;
      while (e < n_ops && (ops[e].type == SV_GATE_CNOT || ops[e].type == SV_GATE_X) &&
             e - l < kMaxPerm)
        ++e;
      if (e - l >= 2) segs.push_back(Seg{SEG_PERM, 0, l, e - l, ckpt++});
      else push_gates(l, e - l);
      l = e;
    } else {
      int e = l;
      while (e < n_ops && ops[e].type != SV_GATE_RZ && ops[e].type != SV_GATE_CZ &&
             ops[e].type != SV_GATE_RY && ops[e].type != SV_GATE_RX &&
             ops[e].type != SV_GATE_CNOT && ops[e].type != SV_GATE_X)
        ++e;
      push_gates(l, e - l);
      l = e;
    }
  }
  // A diagonal segment directly followed by a permutation segment becomes one SEG_DIAGPERM
  // with a single checkpoint (psi before the phase); checkpoints are then renumbered in order.
  std::vector<Seg> merged;
  for (size_t s = 0; s < segs.size(); ++s) {
    if (segs[s].kind == SEG_DIAG && s + 1 < segs.size() && segs[s + 1].kind == SEG_PERM &&
        segs[s + 1].first == segs[s].first + segs[s].count) {
      merged.push_back(Seg{SEG_DIAGPERM, (int16_t)segs[s].count, segs[s].first,
                           segs[s].count + segs[s + 1].count, 0});
      ++s;
    } else {
      merged.push_back(segs[s]);
    }
  }
  // A first segment made of RY gates acts on the reference basis state: a product layer.
  if (!merged.empty() && merged[0].kind == SEG_RLAYER && merged[0].first == 0) {
    bool ry = true;
    for (int l = 0; l < merged[0].count; ++l) ry = ry && ops[l].type == SV_GATE_RY;
    if (ry) merged[0].split = 1;
  }
  ckpt = 0;
  for (Seg& s : merged)
    s.ckpt = (s.kind == SEG_GATES || (s.kind == SEG_RLAYER && s.split == 1)) ? -1 : ckpt++;
  segs.swap(merged);
  for (DOp& op : ops) op.flags &= ~kOpCS;
  for (const Seg& s : segs) {
    if (s.kind == SEG_RLAYER && s.split == 1) {
      for (int l = s.first; l < s.first + s.count; ++l) ops[l].flags |= kOpCS;
      continue;
    }
    if (s.kind != SEG_DIAG && s.kind != SEG_DIAGPERM) continue;
    const int nd = s.kind == SEG_DIAG ? s.count : s.split;
    for (int l = s.first; l < s.first + nd; ++l)
      if (ops[l].type == SV_GATE_RZ) ops[l].flags |= kOpCS;
  }
  return ckpt;
}

std::vector<std::pair<int, int>> commuting_layers(const std::vector<DOp>& ops, int min_len) {
  std::vector<std::pair<int, int>> out;
  const int n_ops = (int)ops.size();
  int l = 0;
  while (l < n_ops) {
    const int t = ops[l].type;
    if (t != SV_GATE_RY && t != SV_GATE_RX) {
      ++l;
      continue;
    }
    uint64_t used = 0;
    int e = l;
    while (e < n_ops && ops[e].type == t && !(used & (1ull << ops[e].bit0))) {
      used |= 1ull << ops[e].bit0;
      ++e;
    }
    if (e - l >= min_len) out.push_back({l, e - l});
    l = e;
  }
  return out;
}

namespace {
struct Unit {      // a schedulable unit: one op, or a run of RZ ops (diagonal item)
  int kind;        // 0 op, 1 diag
  int first, count;
  uint64_t pair;   // bits that must lie inside the tile
  uint64_t touch;  // bits the unit acts on
  int slots;       // gradient slots it needs
};
}  // namespace

void plan_passes(const std::vector<DOp>& ops, int n, int m, HostPlan& plan) {
  const int min_low = n <= kL2Qubits ? kMinLowBitsL2 : kMinLowBits;
  plan.passes.clear();
  plan.items.clear();
  std::vector<Unit> units;
  const int n_ops = (int)ops.size();
  for (int l = 0; l < n_ops;) {
    if (ops[l].type == SV_GATE_RZ) {
      int e = l;
      while (e < n_ops && ops[e].type == SV_GATE_RZ && e - l < kMaxSlots) ++e;
      if (e - l >= 3) {
        Unit u{1, l, e - l, 0, 0, 0};
        for (int q = l; q < e; ++q) {
          u.touch |= 1ull << ops[q].bit0;
          u.slots += ops[q].param >= 0;
        }
        units.push_back(u);
        l = e;
        continue;
      }
    }
    const DOp& op = ops[l];
    uint64_t bits = 0;
    for (int a = 0; a < op.k; ++a) bits |= 1ull << op.sb[a];
    units.push_back(Unit{0, l, 1, bits, bits, op.param >= 0 ? 1 : 0});
    ++l;
  }
  m = std::min(m, n);
  const uint64_t low = (1ull << std::min(min_low, n)) - 1ull;
  std::vector<char> done(units.size(), 0);
  size_t left = units.size();
  while (left > 0) {
    uint64_t pair = 0, blocked = 0;
    int slots = 0;
    bool have_diag = false;
    std::vector<int> take;
    for (size_t u = 0; u < units.size(); ++u) {
      if (done[u]) continue;
      const Unit& U = units[u];
      bool ok = !(U.touch & blocked) && __builtin_popcountll(pair | U.pair | low) <= m &&
                slots + U.slots <= kMaxSlots && !(U.kind == 1 && have_diag);
      if (!ok) {
        blocked |= U.touch;
        continue;
      }
      take.push_back((int)u);
      pair |= U.pair;
      slots += U.slots;
      have_diag |= U.kind == 1;
    }
    // Tile bits: the pass's pair bits plus the lowest free bits up to m (contiguous runs).
    uint64_t tile = pair;
    for (int b = 0; b < n && __builtin_popcountll(tile) < m; ++b) tile |= 1ull << b;
    int c = 0;
    while (c < n && (tile >> c & 1ull)) ++c;
    FPass P{};
    P.tile_mask = tile;
    P.outer_mask = ((n == 64) ? ~0ull : ((1ull << n) - 1ull)) & ~tile;
    P.m = __builtin_popcountll(tile);
    P.c = c;
    P.first_item = (int)plan.items.size();
    P.n_items = (int)take.size();
    int slot = 0;
    for (int u : take) {
      const Unit& U = units[u];
      FItem it{};
      it.kind = U.kind;
      it.op = U.first;
      it.count = U.count;
      it.slot = U.slots ? slot : -1;
      slot += U.slots;
      if (U.kind == 0) {
        // translate the op to tile-local bit positions
        auto loc = [&](uint64_t v) {
          uint64_t r = 0;
          int k = 0;
          for (int b = 0; b < n; ++b)
            if (tile >> b & 1ull) {
              if (v >> b & 1ull) r |= 1ull << k;
              ++k;
            }
          return r;
        };
        DOp L = ops[U.first];
        L.bit0 = __builtin_ctzll(loc(1ull << ops[U.first].bit0));
        for (int a = 0; a < L.k; ++a) L.sb[a] = (uint8_t)__builtin_ctzll(loc(1ull << L.sb[a]));
        L.lo_or = loc(L.lo_or);
        L.flip = loc(L.flip);
        it.local = L;
      }
      plan.items.push_back(it);
      done[u] = 1;
      --left;
    }
    P.n_slots = slot;
    plan.passes.push_back(P);
  }
}

static inline int popc64(uint64_t v) { return __builtin_popcountll(v); }

static uint32_t pext_host(uint64_t v, uint64_t m) {
  uint32_t r = 0;
  int k = 0;
  while (m) {
    const int pos = __builtin_ctzll(m);
    r |= (uint32_t)((v >> pos) & 1ull) << k;
    ++k;
    m &= m - 1;
  }
  return r;
}

sv_status lower_ham(const sv_paulisum* h, int expect_n, int kmax, HostHam& out) {
  if (!h) { set_error("Pauli sum is NULL"); return SV_EINVAL; }
  if (h->n_qubits < 1 || h->n_qubits > 31) {
    set_error("n_qubits %d outside [1, 31]", h->n_qubits);
    return SV_EINVAL;
  }
  if (expect_n > 0 && h->n_qubits != expect_n) {
    set_error("Pauli sum has %d qubits, expected %d", h->n_qubits, expect_n);
    return SV_EINVAL;
  }
  if (h->n_terms < 0 || (h->n_terms > 0 && (!h->x_mask || !h->z_mask || !h->coeff))) {
    set_error("bad term arrays (n_terms %d)", h->n_terms);
    return SV_EINVAL;
  }
  const int n = h->n_qubits;
  const uint64_t full = (n == 64) ? ~0ull : ((1ull << n) - 1ull);
  out.n = n;
  out.n_terms = h->n_terms;
  out.l1 = 0.0;
  out.groups.clear();
  out.tables.clear();
  for (int t = 0; t < h->n_terms; ++t) {
    if ((h->x_mask[t] & ~full) || (h->z_mask[t] & ~full)) {
      set_error("term %d: mask has a bit >= n_qubits (%d)", t, n);
      return SV_EINVAL;
    }
    if (!std::isfinite(h->coeff[t])) { set_error("term %d: coefficient not finite", t); return SV_EINVAL; }
    out.l1 += std::fabs(h->coeff[t]);
  }
  std::vector<int> idx(h->n_terms);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int a, int b) { return h->x_mask[a] < h->x_mask[b]; });
  kmax = std::max(1, std::min(kmax, n));
  size_t s = 0;
  while (s < idx.size()) {
    size_t e = s;
    const uint64_t x = h->x_mask[idx[s]];
    while (e < idx.size() && h->x_mask[idx[e]] == x) ++e;
    // Split the terms [s, e) into sub-groups whose z-union has at most kmax bits.
    std::vector<uint64_t> unions;
    std::vector<std::vector<int>> members;
    for (size_t q = s; q < e; ++q) {
      const int t = idx[q];
      const uint64_t z = h->z_mask[t];
      size_t best = unions.size();
      int best_k = 1 << 30;
      for (size_t u = 0; u < unions.size(); ++u) {
        const int k = popc64(unions[u] | z);
        if (k <= kmax && k < best_k) { best = u; best_k = k; }
      }
      if (best == unions.size()) {
        unions.push_back(0);
        members.emplace_back();
      }
      unions[best] |= z;
      members[best].push_back(t);
    }
    for (size_t u = 0; u < unions.size(); ++u) {
      DGroup g{};
      g.x = x;
      g.zu = unions[u];
      g.kz = popc64(g.zu);
      g.toff = (int64_t)out.tables.size();
      const size_t sz = (size_t)1 << g.kz;
      std::vector<double> re(sz, 0.0), im(sz, 0.0);
      bool any_re = false, any_im = false;
      for (int t : members[u]) {
        // c_t (-i)^{popc(x & z_t)}: (-i)^0 = 1, ^1 = -i, ^2 = -1, ^3 = i.
        const double c = h->coeff[t];
        const uint32_t zc = pext_host(h->z_mask[t], g.zu);
        switch (popc64(x & h->z_mask[t]) & 3) {
          case 0: re[zc] += c; any_re = true; break;
          case 1: im[zc] -= c; any_im = true; break;
          case 2: re[zc] -= c; any_re = true; break;
          case 3: im[zc] += c; any_im = true; break;
        }
      }
      // In-place Walsh-Hadamard transform: F[j] = sum_z C[z] (-1)^{popc(z & j)}.
      for (size_t len = 1; len < sz; len <<= 1)
        for (size_t i = 0; i < sz; i += len << 1)
          for (size_t j = i; j < i + len; ++j) {
            const double a = re[j], b = re[j + len];
            re[j] = a + b; re[j + len] = a - b;
            const double c2 = im[j], d = im[j + len];
            im[j] = c2 + d; im[j + len] = c2 - d;
          }
      g.cls = (any_re && any_im) ? 2 : (any_im ? 1 : 0);
      if (members[u].size() == 1) {
        // One term: f(k) = coefficient * (-1)^{popc(z & k)}, no table walk (cls 4 real,
        // 5 imaginary); the single table entry is the coefficient (the transform's entry 0).
        g.cls += 4;
        out.tables.push_back(make_double2(re[0], im[0]));
      } else {
        for (size_t j = 0; j < sz; ++j) out.tables.push_back(make_double2(re[j], im[j]));
      }
      out.groups.push_back(g);
    }
    s = e;
  }
  return SV_OK;
}

}  // namespace svqe
