// k_batch.cu -- the persistent batched kernel: many small independent instances (Sec. 4.1,
// Eq. 7: every bond length / parameter set is its own problem) in one launch.
//
// A CTA (8 warps) takes work items from a cost-sorted queue with an atomic counter (largest
// first, so the tail is made of cheap items).  An item is one 12-qubit instance run by all 8
// warps, two 11-qubit instances on 4 warps each, four 10-qubit instances on 2 warps each, or
// eight instances of at most 9 qubits on one warp each: every instance gets at most 16
// amplitudes per thread, and small instances synchronise with __syncwarp or a named barrier
// instead of the whole CTA.  An
// instance's psi and lambda (2 x 2^n x 16 bytes) live in its team's share of shared memory for
// the forward pass, lambda = H psi and the adjoint sweep.  GB300's FP64 pipe (2 DFMA/clk/SM) is the binding resource, so the
// op list is executed in segments (see Seg) that cut FP64 work:
//   * a run of RZ/CZ is one diagonal phase per amplitude from two half tables (8 FP64 ops per
//     amplitude instead of 3 per RZ gate);
//   * a commuting layer of RY (or RX) gates takes all its gradients at the layer's end, and
//     the sweep un-applies it to lambda only, reloading psi from a checkpoint that the forward
//     pass stored in global memory (bandwidth is plentiful, FP64 issue is not);
//   * several gradients are reduced at once with a transposed warp reduction.
// Every sum runs in a fixed order that does not depend on which CTA or SM ran the instance,
// so an instance's result is bit-identical alone or in any batch.
#include <type_traits>

#include "launch.h"
#include "svqe_internal.cuh"

namespace svqe {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kM = 16;  // values reduced at once (kMaxLayer)
constexpr int kWarps = kBatchThreads / 32;

// A single-qubit gate of a commuting layer: its coefficients, type and qubit bit.
struct LOp {
  Rot r;
  int type;
  int bit;
};

// Per-team scratch in static shared memory.  Its first kDpBlockAmps x 16 bytes (tl .. n_rz)
// are the tables of a diagonal + permutation segment: the forward pass builds them and saves
// the block to the segment's auxiliary checkpoint slot, the sweep copies it back.
struct TeamS {
  double2 tl[64];
  double2 th[64];
  // A run of CNOT/X gates is an affine map of the index bits over GF(2), so its permutation
  // is P(k) = pt_lo[k & 63] ^ pt_hi[k >> 6] (n <= 12), with pt_lo holding the constant part.
  uint32_t pt_lo[64];
  uint32_t pt_hi[64];
  int rz_op[kM];
  int rz_bit[kM];
  uint32_t cz_mask[kM];  // both-bits masks of the segment's CZ gates
  int n_cz;
  int n_rz;
  int pad[2];
  // (end of the saved block)
  double red[kWarps];
  double red16[kWarps][kM];
  double2 cs[kM];
  uint32_t pm_lo[kMaxPerm];  // condition and flip masks of a permutation segment's gates
  uint32_t pm_fl[kMaxPerm];
  LOp lop[kM];               // the gates of a commuting layer, staged once per segment
};
constexpr int kDpBlockAmps = 173;
static_assert(offsetof(TeamS, pad) + sizeof(int) * 2 == kDpBlockAmps * sizeof(double2),
              "diagonal + permutation block layout");
static_assert(kDpBlockAmps <= kDpAuxAmps, "auxiliary checkpoint slot too small");
static_assert(sizeof(TeamS) % 16 == 0, "TeamS alignment");

// A team of nw warps running one instance.  Teams of one warp synchronise with __syncwarp,
// larger teams with named barrier `bar` (barrier 0 is the CTA-wide one).
struct Team {
  int nw, size, log_size, rank, w, bar;
  __device__ __forceinline__ void sync() const {
    if (nw == 1) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(size) : "memory");
    }
  }
};

// Save the segment's tables (the leading block of S) to its auxiliary slot; plain stores.
__device__ __forceinline__ void dp_save(const Team& T, const TeamS& S, double2* dst) {
  const double2* src = reinterpret_cast<const double2*>(&S);
  for (int k = T.rank; k < kDpBlockAmps; k += T.size) dst[k] = src[k];
}

// The diagonal and permutation parts of a SEG_DIAGPERM segment.
__device__ __forceinline__ Seg diag_part(const Seg& sg) {
  Seg s = sg;
  s.count = sg.split;
  return s;
}
__device__ __forceinline__ Seg perm_part(const Seg& sg) {
  Seg s = sg;
  s.first = sg.first + sg.split;
  s.count = sg.count - sg.split;
  return s;
}

// Tabulate a permutation segment's map over the low and high six index bits: the gates'
// conditional flips in order (inv = false: P) or in reverse order (inv = true: P^-1).  The
// gates' masks are loaded in parallel (one lane per gate, at most kMaxPerm) and staged first.
__device__ __forceinline__ void perm_setup(const Team& T, TeamS& S, const DOp* ops, const Seg& sg,
                                           bool inv, uint32_t N) {
  if (T.rank < sg.count) {
    const DOp& o = ops[sg.first + T.rank];
    const int l = inv ? sg.count - 1 - T.rank : T.rank;
    S.pm_lo[l] = (uint32_t)o.lo_or;
    S.pm_fl[l] = (uint32_t)o.flip;
  }
  T.sync();
  uint32_t c0 = 0;
  for (int l = 0; l < sg.count; ++l)
    if ((c0 & S.pm_lo[l]) == S.pm_lo[l]) c0 ^= S.pm_fl[l];
  // only the entries an index below N can reach: min(64, N) low and max(1, N / 64) high
  const int nlo = N < 64u ? (int)N : 64, nhi = N > 64u ? (int)(N >> 6) : 1;
  for (int j = T.rank; j < nlo + nhi; j += T.size) {
    uint32_t k = j < nlo ? (uint32_t)j : (uint32_t)(j - nlo) << 6;
    for (int l = 0; l < sg.count; ++l)
      if ((k & S.pm_lo[l]) == S.pm_lo[l]) k ^= S.pm_fl[l];
    if (j < nlo) S.pt_lo[j] = k;
    else S.pt_hi[j - nlo] = k ^ c0;
  }
  T.sync();
}

__device__ __forceinline__ uint32_t perm_map(const TeamS& S, uint32_t k) {
  return S.pt_lo[k & 63u] ^ S.pt_hi[k >> 6];
}

__device__ __forceinline__ uint32_t insert_zeros32(uint32_t p, const uint8_t* sb, int k) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t < k) {
      const uint32_t low = p & ((1u << sb[t]) - 1u);
      p = ((p >> sb[t]) << (sb[t] + 1)) | low;
    }
  }
  return p;
}

__device__ __forceinline__ uint32_t pext32(uint32_t i, uint32_t m) {
  uint32_t r = 0;
  int k = 0;
  while (m) {
    const int pos = __ffs(m) - 1;
    r |= ((i >> pos) & 1u) << k;
    ++k;
    m &= m - 1;
  }
  return r;
}

// Team sum of one value per thread; valid in team rank 0 (every lane of a one-warp team).
// The caller synchronises the team before S.red is reused.
__device__ __forceinline__ double team_sum(const Team& T, TeamS& S, double v) {
  v = warp_sum(v);
  if (T.nw == 1) return v;
  if ((threadIdx.x & 31) == 0) S.red[T.w] = v;
  T.sync();
  double t = 0.0;
  if (T.w == 0) {
    const int l = threadIdx.x & 31;
    t = l < T.nw ? S.red[l] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Sum over the warp of 16 values per lane by recursive halving (16 DADD per lane instead of
// 80); afterwards lanes 2j and 2j+1 hold the warp total of value j.
__device__ __forceinline__ double warp_sum16(double (&v)[kM]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int o = 16 >> s, h = 8 >> s;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double send = up ? v[i] : v[i + h];
      const double keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

// Team totals of v[0..m): team rank j < m returns the total of value j, others 0.  Ends with
// the team synchronised.
__device__ __forceinline__ double team_sum16(const Team& T, TeamS& S, double (&v)[kM], int m) {
  const double t = warp_sum16(v);
  const int lane = threadIdx.x & 31;
  if (T.nw == 1) {
    const double r = __shfl_sync(kFull, t, (2 * lane) & 31);
    return lane < m ? r : 0.0;
  }
  if ((lane & 1) == 0) S.red16[T.w][lane >> 1] = t;
  T.sync();
  double s = 0.0;
  if (T.rank < m)
    for (int k = 0; k < T.nw; ++k) s += S.red16[k][T.rank];
  T.sync();
  return s;
}

// acc += 2 Im<lambda|G|psi> on one pair, folded into FMAs.
__device__ __forceinline__ void pair_grad_acc(int type, const double2& lx, const double2& ly,
                                              const double2& px, const double2& py,
                                              double& acc) {
  if (type == SV_GATE_RX) {
    acc = fma(lx.x, py.y, acc);
    acc = fma(dneg(lx.y), py.x, acc);
    acc = fma(ly.x, px.y, acc);
    acc = fma(dneg(ly.y), px.x, acc);
  } else if (type == SV_GATE_RZ) {
    acc = fma(lx.x, px.y, acc);
    acc = fma(dneg(lx.y), px.x, acc);
    acc = fma(dneg(ly.x), py.y, acc);
    acc = fma(ly.y, py.x, acc);
  } else {  // RY and the excitations
    acc = fma(ly.x, px.x, acc);
    acc = fma(ly.y, px.y, acc);
    acc = fma(dneg(lx.x), py.x, acc);
    acc = fma(dneg(lx.y), py.y, acc);
  }
}

__device__ __forceinline__ double2 cmul(const double2& a, const double2& b) {
  return make_double2(fma(a.x, b.x, dneg(a.y) * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul_conj(const double2& a, const double2& b) {  // a * conj(b)
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, dneg(a.x) * b.y));
}

// Apply one pair op to buffer v (forward or inverse), pairs strided over the team, two pairs
// per iteration (both loaded before either is stored, so their chains overlap).
__device__ __forceinline__ void op_pass(const Team& T, double2* v, uint32_t N, const DOp& op,
                                        const Rot& r, bool inv) {
  const uint32_t np = N >> op.k;
  const uint32_t lo = (uint32_t)op.lo_or;
  if (op.type == SV_GATE_CZ) {
    for (uint32_t p = T.rank; p < np; p += T.size) {
      const uint32_t i = insert_zeros32(p, op.sb, op.k) | lo;
      v[i] = make_double2(dneg(v[i].x), dneg(v[i].y));
    }
    return;
  }
  const uint32_t fl = (uint32_t)op.flip;
  for (uint32_t p = T.rank; p < np; p += 2 * T.size) {
    const uint32_t p2 = p + T.size;
    const uint32_t i = insert_zeros32(p, op.sb, op.k) | lo;
    const uint32_t i2 = insert_zeros32(p2, op.sb, op.k) | lo;
    double2 x = v[i], y = v[i ^ fl];
    double2 x2, y2;
    const bool two = p2 < np;
    if (two) {
      x2 = v[i2];
      y2 = v[i2 ^ fl];
    }
    pair_apply(op.type, r, inv, x, y);
    if (two) pair_apply(op.type, r, inv, x2, y2);
    v[i] = x;
    v[i ^ fl] = y;
    if (two) {
      v[i2] = x2;
      v[i2 ^ fl] = y2;
    }
  }
}

// Copy N amplitudes between the team's shared buffer and its checkpoint, four loads in flight
// per thread before the stores.
__device__ __forceinline__ void team_copy(const Team& T, double2* dst, const double2* src,
                                          uint32_t N) {
  const uint32_t s = T.size;
  uint32_t k = T.rank;
  for (; k + 3 * s < N; k += 4 * s) {
    const double2 a = src[k], b = src[k + s], c = src[k + 2 * s], d = src[k + 3 * s];
    dst[k] = a;
    dst[k + s] = b;
    dst[k + 2 * s] = c;
    dst[k + 3 * s] = d;
  }
  for (; k < N; k += s) dst[k] = src[k];
}

// Bring [p, p + bytes) into L2 ahead of use, one 128-byte line per prefetch across the team.
__device__ __forceinline__ void team_prefetch_l2(const Team& T, const void* p, int64_t bytes) {
  const char* b = (const char*)p;
  for (int64_t o = (int64_t)T.rank * 128; o < bytes; o += (int64_t)T.size * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(b + o));
}

// Start an asynchronous copy of N amplitudes from global memory into the team's shared buffer
// (16 B per cp.async, L2 only); async_wait() and a team barrier complete it.
__device__ __forceinline__ void async_copy(const Team& T, double2* dst, const double2* src,
                                           uint32_t N) {
  for (uint32_t k = T.rank; k < N; k += T.size) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + k);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + k) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage a commuting layer's gates (coefficients, type, bit) in shared memory: one parallel
// load per gate instead of one dependent load per pass.
__device__ __forceinline__ void layer_setup(const Team& T, TeamS& S, const DOp* ops,
                                            const Rot* coef, const Seg& sg) {
  if (T.rank < sg.count) {
    LOp o;
    o.r = coef[sg.first + T.rank];
    o.type = ops[sg.first + T.rank].type;
    o.bit = ops[sg.first + T.rank].bit0;
    S.lop[T.rank] = o;
  }
  T.sync();
}

// One staged layer gate on v (inv: its inverse).
__device__ __forceinline__ void lop_pass(const Team& T, double2* v, uint32_t N, const LOp& o,
                                         bool inv) {
  const uint32_t fl = 1u << o.bit, low = fl - 1u;
  for (uint32_t p = T.rank; p < (N >> 1); p += T.size) {
    const uint32_t i = ((p & ~low) << 1) | (p & low);
    double2 x = v[i], y = v[i | fl];
    pair_apply(o.type, o.r, inv, x, y);
    v[i] = x;
    v[i | fl] = y;
  }
}

// One layer gate on a pair, with the rotation (and its inverse, for RX) prepared: RY rotates
// (re x, re y) and (im x, im y) by R(phi); RX rotates (re x, im y) by R(-phi) and (im x, re y)
// by R(phi).
template <bool ROTX>
__device__ __forceinline__ void layer_pair(const Rot& r, const Rot& m, double2& x, double2& y) {
  if (ROTX) {
    rot_apply(m, x.x, y.y);
    rot_apply(r, x.y, y.x);
  } else {
    rot_apply(r, x.x, y.x);
    rot_apply(r, x.y, y.y);
  }
}

// Two staged layer gates on distinct bits in one pass: each thread takes the four amplitudes of
// a block (both bits 0, either, both 1), rotates them for the first gate, then for the second,
// in registers (inverse: inverted, in reverse order).  A layer is all RY or all RX.  If ckout
// is set, the amplitudes are also stored there unchanged first: the pass doubles as the
// checkpoint copy.
template <bool ROTX>
__device__ __forceinline__ void lop_pass2_k(const Team& T, double2* v, uint32_t N, const LOp& o1,
                                            const LOp& o2, bool inv, double2* ckout) {
  const uint32_t b1 = 1u << o1.bit, b2 = 1u << o2.bit;
  uint8_t sb[2];
  sb[0] = (uint8_t)min(o1.bit, o2.bit);
  sb[1] = (uint8_t)max(o1.bit, o2.bit);
  const Rot r1 = inv ? rot_inverse(o1.r) : o1.r, r2 = inv ? rot_inverse(o2.r) : o2.r;
  const Rot m1 = rot_inverse(r1), m2 = rot_inverse(r2);
  for (uint32_t p = T.rank; p < (N >> 2); p += T.size) {
    const uint32_t i = insert_zeros32(p, sb, 2);
    double2 a = v[i], b = v[i | b1], c = v[i | b2], d = v[i | b1 | b2];
    if (ckout) {
      ckout[i] = a;
      ckout[i | b1] = b;
      ckout[i | b2] = c;
      ckout[i | b1 | b2] = d;
    }
    if (!inv) {
      layer_pair<ROTX>(r1, m1, a, b);
      layer_pair<ROTX>(r1, m1, c, d);
      layer_pair<ROTX>(r2, m2, a, c);
      layer_pair<ROTX>(r2, m2, b, d);
    } else {
      layer_pair<ROTX>(r2, m2, a, c);
      layer_pair<ROTX>(r2, m2, b, d);
      layer_pair<ROTX>(r1, m1, a, b);
      layer_pair<ROTX>(r1, m1, c, d);
    }
    v[i] = a;
    v[i | b1] = b;
    v[i | b2] = c;
    v[i | b1 | b2] = d;
  }
}

__device__ __forceinline__ void lop_pass2(const Team& T, double2* v, uint32_t N, const LOp& o1,
                                          const LOp& o2, bool inv, double2* ckout) {
  if (o1.type == SV_GATE_RX) lop_pass2_k<true>(T, v, N, o1, o2, inv, ckout);
  else lop_pass2_k<false>(T, v, N, o1, o2, inv, ckout);
}

// Build the diagonal segment's half tables: th[hi] * tl[lo] = prod_RZ e^{-i phi s(k)}, and
// the list of its CZ masks.
__device__ __noinline__ int diag_setup(const Team& T, TeamS& S, const DOp* ops,
                                          const Rot* coef, const Seg& sg, int n) {
  // The segment's ops (at most kM RZ and kM CZ gates) are read in parallel by the lanes of the
  // team's first warp; a ballot gives each RZ (CZ) gate its slot in gate order.
  if (T.w == 0) {
    const int lane = threadIdx.x & 31;
    int type = -1;
    DOp op;
    if (lane < sg.count) {
      op = ops[sg.first + lane];
      type = op.type;
    }
    const unsigned brz = __ballot_sync(kFull, type == SV_GATE_RZ);
    const unsigned bcz = __ballot_sync(kFull, type == SV_GATE_CZ);
    const unsigned below = (1u << lane) - 1u;
    if (type == SV_GATE_RZ) {
      const int i = __popc(brz & below);
      S.rz_op[i] = sg.first + lane;
      S.rz_bit[i] = op.bit0;
      const Rot r = coef[sg.first + lane];  // (cos phi, sin phi), set up with the step's coefficients
      S.cs[i] = make_double2(r.a, r.b);
    } else if (type == SV_GATE_CZ) {
      S.cz_mask[__popc(bcz & below)] = (uint32_t)op.lo_or;
    }
    if (lane == 0) {
      S.n_rz = __popc(brz);
      S.n_cz = __popc(bcz);
    }
  }
  T.sync();
  const int m = S.n_rz;
  const int hl = n < 6 ? n : 6;
  const int nl = 1 << hl, nh = 1 << (n - hl);
  for (int j = T.rank; j < nl + nh; j += T.size) {
    const bool hi = j >= nl;
    const int jj = hi ? j - nl : j;
    double2 p = make_double2(1.0, 0.0);
    for (int g = 0; g < m; ++g) {
      const int b = S.rz_bit[g];
      if ((b >= hl) != hi) continue;
      const int bit = (jj >> (hi ? b - hl : b)) & 1;
      const double2 f = make_double2(S.cs[g].x, bit ? S.cs[g].y : dneg(S.cs[g].y));
      p = cmul(p, f);
    }
    if (hi) S.th[jj] = p; else S.tl[jj] = p;
  }
  T.sync();
  return m;
}

// The fields of a group record that lambda = H psi uses (indices fit 32 bits: n <= 12).
struct GRec {
  uint32_t x, zu;
  int cls;
  int64_t toff;
};
__device__ __forceinline__ GRec grec(const DGroup& G) {
  GRec r;
  r.x = (uint32_t)G.x;
  r.zu = (uint32_t)G.zu;
  r.cls = G.cls;
  r.toff = G.toff;
  return r;
}

// A product layer (first segment: RY gates on the reference basis state |r>): the state it
// makes is prod_b f_b(k_b), with f_b = (cos phi, sin phi) on bit values (0, 1) for a gate on a
// bit with r_b = 0, (-sin phi, cos phi) for r_b = 1, and [k_b == r_b] on a bit without a gate.
// The factors of bits [0, hl) and [hl, n) are multiplied out into the half tables tl and th
// (real parts), so psi[k] = tl[k & lmask] * th[k >> hl].
__device__ __noinline__ void product_setup(const Team& T, TeamS& S, const DOp* ops,
                                           const Rot* coef, const Seg& sg, uint64_t ref, int n) {
  if (T.rank < n) {
    const bool r1 = (ref >> T.rank) & 1ull;
    S.cs[T.rank] = r1 ? make_double2(0.0, 1.0) : make_double2(1.0, 0.0);
  }
  T.sync();
  if (T.rank < sg.count) {
    const int b = ops[sg.first + T.rank].bit0;
    const Rot r = coef[sg.first + T.rank];  // (cos phi, sin phi)
    const bool r1 = (ref >> b) & 1ull;
    S.cs[b] = r1 ? make_double2(dneg(r.b), r.a) : make_double2(r.a, r.b);
  }
  T.sync();
  const int hl = n < 6 ? n : 6;
  const int nl = 1 << hl, nh = 1 << (n - hl);
  for (int j = T.rank; j < nl + nh; j += T.size) {
    const bool hi = j >= nl;
    const int jj = hi ? j - nl : j;
    const int b0 = hi ? hl : 0, b1 = hi ? n : hl;
    double p = 1.0;
    for (int b = b0; b < b1; ++b) {
      const double2 f = S.cs[b];
      p *= ((jj >> (b - b0)) & 1) ? f.y : f.x;
    }
    if (hi) S.th[jj] = make_double2(p, 0.0); else S.tl[jj] = make_double2(p, 0.0);
  }
  T.sync();
}

// b^t for t >= 1 by repeated squaring (about 2 log2 t multiplies instead of a transcendental
// pow; the value depends on t alone, so one long call and many short calls agree bit for bit).
__device__ __forceinline__ double ipow(double b, int t) {
  double r = 1.0;
  while (t > 0) {
    if (t & 1) r *= b;
    b *= b;
    t >>= 1;
  }
  return r;
}

// Sign of the CZ gates of a diagonal segment at amplitude k (true = negative).
__device__ __forceinline__ bool cz_sign(const TeamS& S, int ncz, uint32_t k) {
  uint32_t par = 0;
  for (int c = 0; c < ncz; ++c) par ^= ((k & S.cz_mask[c]) == S.cz_mask[c]);
  return par & 1u;
}

__device__ void run_instance(const BatchArgs& a, int idx, const Team& T, TeamS& S, double2* sm,
                             double2* ck) {
  const BInst I = a.inst[idx];
  const int n = I.n;
  const uint32_t N = 1u << n;
  double2* psi = sm;
  double2* lam = sm + N;
  const DOp* ops = a.ops + I.op_off;
  const DGroup* groups = a.groups + I.grp_off;
  const Seg* segs = a.segs + I.seg_off;
  Rot* coef = a.coef + I.coef_off;
  double* contrib = a.contrib + I.contrib_off;
  double* theta = a.theta + I.theta_off;
  double* grad = a.grad + I.grad_off;
  const int tid = T.rank;
  const int TS = T.size;
  // auxiliary checkpoint slots (saved segment tables) after the I.n_ckpt states
  double2* aux = ck + (size_t)I.n_ckpt * N;
  const int hl = n < 6 ? n : 6;
  const uint32_t lmask = (1u << hl) - 1u;
  const bool per_inst = a.n_steps < 0;
  const int steps = per_inst ? I.steps : (a.n_steps > 0 ? a.n_steps : 1);
  const bool gd = a.n_steps != 0;
  const double lr = per_inst ? I.lr : (a.lr_inst ? a.lr_inst[idx] : a.lr);

  for (int step = 0; step < steps; ++step) {
    for (int g = tid; g < I.n_ops; g += TS) {
      const DOp op = ops[g];
      if (op.flags & kOpCS) {
        const double t = op.param >= 0 ? theta[op.param] : op.fixed;
        Rot r;
        sincos(0.5 * t, &r.b, &r.a);
        r.k = 0;
        r.pad = 0;
        coef[g] = r;
      } else {
        coef[g] = make_coef(op, theta).r;
      }
    }
    for (uint32_t k = tid; k < N; k += TS)
      psi[k] = make_double2(k == (uint32_t)I.ref ? 1.0 : 0.0, 0.0);
    // the group records and tables are first read by lambda = H psi, after the forward pass
    if (step == 0) {
      team_prefetch_l2(T, groups, (int64_t)I.n_groups * (int64_t)sizeof(DGroup));
      team_prefetch_l2(T, a.tables + I.tab_off, (int64_t)I.tab_n * (int64_t)sizeof(double2));
    }
    T.sync();

    // ---------------------------------------------------------------- forward
    for (int s = 0; s < I.n_segs; ++s) {
      const Seg sg = segs[s];
      if (sg.ckpt >= 0 && sg.kind != SEG_DIAGPERM && sg.kind != SEG_RLAYER) {
        team_copy(T, ck + (size_t)sg.ckpt * N, psi, N);
        T.sync();
      }
      if (sg.kind == SEG_DIAGPERM) {
        // one pass: checkpoint psi[k], apply the phase, scatter to P k (the gates' conditional
        // flips in order)
        diag_setup(T, S, ops, coef, diag_part(sg), n);
        perm_setup(T, S, ops, perm_part(sg), false, N);
        dp_save(T, S, aux + (size_t)sg.ckpt * kDpAuxAmps);
        const int ncz = S.n_cz;
        double2* c = ck + (size_t)sg.ckpt * N;
        for (uint32_t k = tid; k < N; k += TS) {
          const double2 p0 = psi[k];
          c[k] = p0;
          const double2 ph = cmul(S.th[k >> hl], S.tl[k & lmask]);
          double2 v = cmul(p0, ph);
          if (ncz && cz_sign(S, ncz, k)) v = make_double2(dneg(v.x), dneg(v.y));
          lam[perm_map(S, k)] = v;
        }
        T.sync();
        double2* t = psi;
        psi = lam;
        lam = t;
      } else if (sg.kind == SEG_PERM) {
        // psi'[j] = psi[P^-1 j] with P = C_last ... C_first (each CNOT/X is its own inverse)
        perm_setup(T, S, ops, sg, true, N);
        for (uint32_t j = tid; j < N; j += TS) lam[j] = psi[perm_map(S, j)];
        T.sync();
        double2* t = psi;
        psi = lam;
        lam = t;
      } else if (sg.kind == SEG_DIAG) {
        diag_setup(T, S, ops, coef, sg, n);
        const int ncz = S.n_cz;
        for (uint32_t k = tid; k < N; k += TS) {
          const double2 ph = cmul(S.th[k >> hl], S.tl[k & lmask]);
          double2 v = cmul(psi[k], ph);
          if (ncz && cz_sign(S, ncz, k)) v = make_double2(dneg(v.x), dneg(v.y));
          psi[k] = v;
        }
        T.sync();
      } else if (sg.kind == SEG_RLAYER && sg.split == 1) {
        product_setup(T, S, ops, coef, sg, I.ref, n);
        for (uint32_t k = tid; k < N; k += TS)
          psi[k] = make_double2(S.tl[k & lmask].x * S.th[k >> hl].x, 0.0);
        T.sync();
      } else if (sg.kind == SEG_RLAYER) {
        // the layer's first pass also writes the checkpoint (a layer has at least two gates)
        layer_setup(T, S, ops, coef, sg);
        int g = 0;
        for (; g + 1 < sg.count; g += 2) {
          lop_pass2(T, psi, N, S.lop[g], S.lop[g + 1], false,
                    g == 0 ? ck + (size_t)sg.ckpt * N : nullptr);
          T.sync();
        }
        if (g < sg.count) {
          lop_pass(T, psi, N, S.lop[g], false);
          T.sync();
        }
      } else {
        for (int l = sg.first; l < sg.first + sg.count; ++l) {
          op_pass(T, psi, N, ops[l], coef[l], false);
          T.sync();
        }
      }
    }

    // ---------------------------------------------------------------- lambda = H psi
    // Each thread carries all of its amplitudes (at most kHU = 16 in every team class) through
    // the group loop: kHU independent multiply-add chains and table loads in flight, and one
    // group-record load per thread per group.
    double e = 0.0;
    constexpr int kHU = 16;
    // u runs over the thread's amplitudes k = k0 + u TS: nu of them (N <= kHU TS in every
    // class, so one k0 per thread)
    const int nu = N >= (uint32_t)TS ? (int)(N >> T.log_size) : 1;
    // the group loop runs in two forms: every slot u valid (FULL, the common case for the
    // larger registers), or stopping at u = nu
    auto hpsi = [&](auto full_tag) {
      constexpr bool FULL = decltype(full_tag)::value;
      for (uint32_t k0 = tid; k0 < N; k0 += kHU * TS) {
        double2 acc[kHU];
  #pragma unroll
        for (int u = 0; u < kHU; ++u) acc[u] = make_double2(0.0, 0.0);
        // group records are loaded two groups ahead and the first table entry (a single-term
        // group's coefficient) one group ahead, so neither load waits in the loop
        const int ng = I.n_groups;
        GRec Gn, Gnn;
        double2 cn = make_double2(0.0, 0.0);
        if (ng > 0) {
          Gn = grec(groups[0]);
          Gnn = grec(groups[ng > 1 ? 1 : 0]);
          cn = a.tables[Gn.toff];
        }
        for (int g = 0; g < ng; ++g) {
          const GRec G = Gn;
          const double2 c = cn;
          Gn = Gnn;
          cn = a.tables[Gn.toff];
          Gnn = grec(groups[g + 2 < ng ? g + 2 : ng - 1]);
          const uint32_t x = G.x, zu = G.zu;
          if (G.cls == 4) {
            // real coefficient: acc += s c psi[k ^ x], s = (-1)^popc(k & zu) as a sign bit
  #pragma unroll
            for (int u = 0; u < kHU; ++u) {
              if (!FULL && u >= nu) break;
              const uint32_t k = k0 + u * TS;
              {
                const double2 v = psi[k ^ x];
                const double f = (__popc(k & zu) & 1) ? dneg(c.x) : c.x;
                acc[u].x = fma(f, v.x, acc[u].x);
                acc[u].y = fma(f, v.y, acc[u].y);
              }
            }
          } else if (G.cls == 5) {
            // imaginary coefficient i c: acc += s (-c v.y, c v.x)
  #pragma unroll
            for (int u = 0; u < kHU; ++u) {
              if (!FULL && u >= nu) break;
              const uint32_t k = k0 + u * TS;
              {
                const double2 v = psi[k ^ x];
                const double f = (__popc(k & zu) & 1) ? dneg(c.y) : c.y;
                acc[u].x = fma(dneg(f), v.y, acc[u].x);
                acc[u].y = fma(f, v.x, acc[u].y);
              }
            }
          } else {
            // table index pext(k, zu) with k = k0 + u TS (k0 < TS: N <= kHU TS in every class):
            // the bits of zu below log_size give a per-thread base, and each set bit b of u adds
            // d[b] (zero unless bit log_size + b is in zu)
            const uint32_t zl = zu & (uint32_t)(TS - 1), zh = zu >> T.log_size;
            const uint32_t base = pext32(k0, zl);
            const int sh = __popc(zl);
            uint32_t d[4];
  #pragma unroll
            for (int b = 0; b < 4; ++b)
              d[b] = ((zh >> b) & 1u) << (sh + __popc(zh & ((1u << b) - 1u)));
            // a real or imaginary table is read one component at a time (8 bytes per entry)
            const double* tab = reinterpret_cast<const double*>(a.tables + G.toff);
            if (G.cls == 0) {
  #pragma unroll
              for (int u = 0; u < kHU; ++u) {
                if (!FULL && u >= nu) break;
                const uint32_t k = k0 + u * TS;
                {
                  uint32_t ti = base;
  #pragma unroll
                  for (int b = 0; b < 4; ++b)
                    if ((u >> b) & 1) ti += d[b];
                  const double f = tab[2 * ti];
                  const double2 v = psi[k ^ x];
                  acc[u].x = fma(f, v.x, acc[u].x);
                  acc[u].y = fma(f, v.y, acc[u].y);
                }
              }
            } else if (G.cls == 1) {
  #pragma unroll
              for (int u = 0; u < kHU; ++u) {
                if (!FULL && u >= nu) break;
                const uint32_t k = k0 + u * TS;
                {
                  uint32_t ti = base;
  #pragma unroll
                  for (int b = 0; b < 4; ++b)
                    if ((u >> b) & 1) ti += d[b];
                  const double f = tab[2 * ti + 1];
                  const double2 v = psi[k ^ x];
                  acc[u].x = fma(dneg(f), v.y, acc[u].x);
                  acc[u].y = fma(f, v.x, acc[u].y);
                }
              }
            } else {
  #pragma unroll
              for (int u = 0; u < kHU; ++u) {
                if (!FULL && u >= nu) break;
                const uint32_t k = k0 + u * TS;
                {
                  uint32_t ti = base;
  #pragma unroll
                  for (int b = 0; b < 4; ++b)
                    if ((u >> b) & 1) ti += d[b];
                  group_madd(2, a.tables[G.toff + ti], psi[k ^ x], acc[u]);
                }
              }
            }
          }
        }
  #pragma unroll
        for (int u = 0; u < kHU; ++u) {
          if (!FULL && u >= nu) break;
          const uint32_t k = k0 + u * TS;
          {
            lam[k] = acc[u];
            const double2 p = psi[k];
            e = fma(p.x, acc[u].x, e);
            e = fma(p.y, acc[u].y, e);
          }
        }
      }
    };
    if (nu == kHU) hpsi(std::true_type{});
    else hpsi(std::false_type{});
    const double E = team_sum(T, S, e);
    T.sync();

    // ---------------------------------------------------------------- adjoint sweep
    int pre_dp = -1;  // segment whose saved tables are already in S
    for (int s = I.n_segs - 1; s >= 0; --s) {
      const Seg sg = segs[s];
      if (sg.kind == SEG_GATES) {
        for (int l = sg.first + sg.count - 1; l >= sg.first; --l) {
          const DOp op = ops[l];
          const Rot r = coef[l];
          const uint32_t np = N >> op.k;
          const bool pg = op.param >= 0;
          const uint32_t lo = (uint32_t)op.lo_or, fl = (uint32_t)op.flip;
          double acc = 0.0;
          for (uint32_t p = tid; p < np; p += TS) {
            const uint32_t i = insert_zeros32(p, op.sb, op.k) | lo;
            if (op.type == SV_GATE_CZ) {
              psi[i] = make_double2(dneg(psi[i].x), dneg(psi[i].y));
              lam[i] = make_double2(dneg(lam[i].x), dneg(lam[i].y));
            } else {
              const uint32_t j = i ^ fl;
              double2 px = psi[i], py = psi[j], lx = lam[i], ly = lam[j];
              if (pg) pair_grad_acc(op.type, lx, ly, px, py, acc);
              pair_apply(op.type, r, true, px, py);
              pair_apply(op.type, r, true, lx, ly);
              psi[i] = px;
              psi[j] = py;
              lam[i] = lx;
              lam[j] = ly;
            }
          }
          if (pg) {
            const double t = team_sum(T, S, acc);
            if (tid == 0) contrib[l] = t;
          }
          T.sync();
        }
        continue;
      }
      if (sg.kind == SEG_PERM) {
        // lambda_before[j] = lambda_after[P j], gathered into the psi buffer (psi is reloaded
        // from the checkpoint below), then the buffers swap roles
        perm_setup(T, S, ops, sg, false, N);
        for (uint32_t j = tid; j < N; j += TS) psi[j] = lam[perm_map(S, j)];
        T.sync();
        double2* t = psi;
        psi = lam;
        lam = t;
        team_copy(T, psi, ck + (size_t)sg.ckpt * N, N);
        T.sync();
        continue;
      }
      double v[kM];
#pragma unroll
      for (int g = 0; g < kM; ++g) v[g] = 0.0;
      if (sg.kind == SEG_DIAGPERM) {
        // psi and lambda at the diagonal part's end are psi[P k] and lambda[P k]: gather both,
        // take the signed bit sums of w_k = Im(conj(lambda) psi) as for SEG_DIAG, and keep the
        // un-phased lambda in registers until every gather of the team is done (at most kHU
        // amplitudes per thread in every team class)
        // the tables the forward pass built at the same parameters (already loaded when the
        // commuting layer after this segment prefetched them)
        if (pre_dp != s) {
          async_copy(T, reinterpret_cast<double2*>(&S), aux + (size_t)sg.ckpt * kDpAuxAmps,
                     kDpBlockAmps);
          async_wait();
          T.sync();
        }
        const int m = S.n_rz;
        const int ncz = S.n_cz;
        constexpr int kHB = 4;
        constexpr int kHU = 16;
        const int nhb = n - T.log_size;
        double W = 0.0, hb[kHB] = {0.0, 0.0, 0.0, 0.0}, wq[4];
        double2 lr[kHU];
        // the thread's amplitudes are k = tid + u TS for u < nu (index bit log_size + q is
        // bit q of u)
        const int nu = N >= (uint32_t)TS ? (int)(N >> T.log_size) : ((uint32_t)tid < N ? 1 : 0);
#pragma unroll
        for (int u = 0; u < kHU; ++u) {
          if (u >= nu) break;
          const uint32_t k = tid + u * TS;
          {
            const uint32_t src = perm_map(S, k);
            const double2 pk = psi[src];
            double2 lk = lam[src];
            const double w = fma(lk.x, pk.y, dneg(lk.y) * pk.x);
            if (nu >= 4) {
              // nu = 2^nhb >= 4: the sums over slots u are reduced four at a time, a partial
              // butterfly (3 DADD per amplitude instead of 1 + nhb)
              wq[u & 3] = w;
              if ((u & 3) == 3) {
                const double s01 = wq[0] + wq[1], d01 = wq[0] - wq[1];
                const double s23 = wq[2] + wq[3], d23 = wq[2] - wq[3];
                const double Sq = s01 + s23;
                W += Sq;
                hb[0] += d01 + d23;
                hb[1] += s01 - s23;
#pragma unroll
                for (int q = 2; q < kHB; ++q)
                  if (q < nhb) hb[q] += ((u >> q) & 1) ? dneg(Sq) : Sq;
              }
            } else {
              W += w;
#pragma unroll
              for (int q = 0; q < kHB; ++q)
                if (q < nhb) hb[q] += ((u >> q) & 1) ? dneg(w) : w;
            }
            const double2 ph = cmul(S.th[k >> hl], S.tl[k & lmask]);
            lk = cmul_conj(lk, ph);
            if (ncz && cz_sign(S, ncz, k)) lk = make_double2(dneg(lk.x), dneg(lk.y));
            lr[u] = lk;
          }
        }
        T.sync();
        // psi before the segment: the checkpoint copy overlaps the stores and the reduction
        async_copy(T, psi, ck + (size_t)sg.ckpt * N, N);
#pragma unroll
        for (int u = 0; u < kHU; ++u) {
          if (u >= nu) break;
          lam[tid + u * TS] = lr[u];
        }
#pragma unroll
        for (int g = 0; g < kM; ++g) {
          if (g >= m) break;
          const int b = S.rz_bit[g];
          double val = (((uint32_t)tid >> (b < T.log_size ? b : 0)) & 1u) ? dneg(W) : W;
#pragma unroll
          for (int q = 0; q < kHB; ++q)
            if (b == T.log_size + q) val = hb[q];
          v[g] = val;
        }
        const double tot = team_sum16(T, S, v, m);
        if (tid < m) contrib[S.rz_op[tid]] = tot;
        async_wait();
        T.sync();
        continue;
      } else if (sg.kind == SEG_RLAYER) {
        // a diagonal + permutation segment next in the sweep: start reloading its tables now
        // (this segment does not use that block; its final wait completes the copy)
        if (sg.split != 1 && s > 0 && segs[s - 1].kind == SEG_DIAGPERM) {
          async_copy(T, reinterpret_cast<double2*>(&S),
                     aux + (size_t)segs[s - 1].ckpt * kDpAuxAmps, kDpBlockAmps);
          pre_dp = s - 1;
        }
        // gradients of every gate from (psi, lambda) at the layer's end, two gates per pass:
        // each thread reads a block of four amplitudes of psi and lambda and accumulates both
        // gates' pair terms from it
        layer_setup(T, S, ops, coef, sg);
        int g = 0;
        for (; g + 1 < sg.count; g += 2) {
          const LOp& o1 = S.lop[g];
          const LOp& o2 = S.lop[g + 1];
          const uint32_t b1 = 1u << o1.bit, b2 = 1u << o2.bit;
          uint8_t sb[2];
          sb[0] = (uint8_t)min(o1.bit, o2.bit);
          sb[1] = (uint8_t)max(o1.bit, o2.bit);
          double a1 = 0.0, a2 = 0.0;
          // a layer is all RY or all RX: one loop per kind, no per-pair dispatch
          auto grads = [&](auto kind_tag) {
            constexpr int KIND = decltype(kind_tag)::value;
            for (uint32_t p = tid; p < (N >> 2); p += TS) {
              const uint32_t i = insert_zeros32(p, sb, 2);
              const double2 pa = psi[i], pb = psi[i | b1], pc = psi[i | b2],
                            pd = psi[i | b1 | b2];
              const double2 la = lam[i], lb = lam[i | b1], lc = lam[i | b2],
                            ld = lam[i | b1 | b2];
              pair_grad_acc(KIND, la, lb, pa, pb, a1);
              pair_grad_acc(KIND, lc, ld, pc, pd, a1);
              pair_grad_acc(KIND, la, lc, pa, pc, a2);
              pair_grad_acc(KIND, lb, ld, pb, pd, a2);
            }
          };
          if (o1.type == SV_GATE_RX) grads(std::integral_constant<int, SV_GATE_RX>{});
          else grads(std::integral_constant<int, SV_GATE_RY>{});
#pragma unroll
          for (int q = 0; q < kM; ++q) {
            if (q == g) v[q] = a1;
            if (q == g + 1) v[q] = a2;
          }
        }
        if (g < sg.count) {
          const LOp& o = S.lop[g];
          const uint32_t fl = 1u << o.bit, low = fl - 1u;
          double acc = 0.0;
          for (uint32_t p = tid; p < (N >> 1); p += TS) {
            const uint32_t i = ((p & ~low) << 1) | (p & low);
            pair_grad_acc(o.type, lam[i], lam[i | fl], psi[i], psi[i | fl], acc);
          }
#pragma unroll
          for (int q = 0; q < kM; ++q)
            if (q == g) v[q] = acc;
        }
        const double tot = team_sum16(T, S, v, sg.count);
        if (tid < sg.count) contrib[sg.first + tid] = tot;
        if (sg.split == 1) {  // a product layer: nothing before it needs psi or lambda
          T.sync();
          continue;
        }
        // psi before the layer: the checkpoint copy runs while the layer is un-applied to
        // lambda (its gates commute: pairs in forward order, inverted), which leaves psi alone
        async_copy(T, psi, ck + (size_t)sg.ckpt * N, N);
        g = 0;
        for (; g + 1 < sg.count; g += 2) {
          lop_pass2(T, lam, N, S.lop[g], S.lop[g + 1], true, nullptr);
          T.sync();
        }
        if (g < sg.count) {
          lop_pass(T, lam, N, S.lop[g], true);
          T.sync();
        }
        async_wait();
        T.sync();
        continue;
      } else {  // SEG_DIAG
        const int m = diag_setup(T, S, ops, coef, sg, n);
        const int ncz = S.n_cz;
        // Signed sums per bit: the bits below log_size are fixed within a thread (one running
        // sum W suffices); at most kHB higher bits vary across the thread's amplitudes.
        constexpr int kHB = 4;
        const int nhb = n - T.log_size;
        double W = 0.0, hb[kHB] = {0.0, 0.0, 0.0, 0.0};
        for (uint32_t k = tid; k < N; k += TS) {
          const double2 pk = psi[k];
          double2 lk = lam[k];
          const double w = fma(lk.x, pk.y, dneg(lk.y) * pk.x);  // Im(conj(lambda) psi)
          W += w;
#pragma unroll
          for (int q = 0; q < kHB; ++q)
            if (q < nhb) hb[q] += ((k >> (T.log_size + q)) & 1u) ? dneg(w) : w;
          const double2 ph = cmul(S.th[k >> hl], S.tl[k & lmask]);
          lk = cmul_conj(lk, ph);
          if (ncz && cz_sign(S, ncz, k)) lk = make_double2(dneg(lk.x), dneg(lk.y));
          lam[k] = lk;
        }
#pragma unroll
        for (int g = 0; g < kM; ++g) {
          if (g >= m) break;
          const int b = S.rz_bit[g];
          double val = (((uint32_t)tid >> (b < T.log_size ? b : 0)) & 1u) ? dneg(W) : W;
#pragma unroll
          for (int q = 0; q < kHB; ++q)
            if (b == T.log_size + q) val = hb[q];
          v[g] = val;
        }
        const double tot = team_sum16(T, S, v, m);
        if (tid < m) contrib[S.rz_op[tid]] = tot;
      }
      // psi before the segment, from the forward pass's checkpoint
      team_copy(T, psi, ck + (size_t)sg.ckpt * N, N);
      T.sync();
    }

    // ---------------------------------------------------------------- gradients, update
    for (int p = tid; p < I.n_params; p += TS) {
      double g = 0.0;
      for (int j = a.pptr[I.pp_off + p]; j < a.pptr[I.pp_off + p + 1]; ++j)
        g += contrib[a.pops[j]];
      grad[p] = g;
      if (gd) {
        if (a.opt == 1) {
          // Adam (the paper's optimizer, Sec. 3.4): bias-corrected moment estimates
          const size_t q = (size_t)I.grad_off + p;
          const double m = fma(a.beta1, a.adam_m[q], (1.0 - a.beta1) * g);
          const double v = fma(a.beta2, a.adam_v[q], (1.0 - a.beta2) * g * g);
          a.adam_m[q] = m;
          a.adam_v[q] = v;
          const int t = a.adam_t0 + step + 1;
          const double mh = m / (1.0 - ipow(a.beta1, t));
          const double vh = v / (1.0 - ipow(a.beta2, t));
          theta[p] -= lr * mh / (sqrt(vh) + a.eps);
        } else {
          theta[p] = fma(-lr, g, theta[p]);
        }
      }
    }
    if (tid == 0) {
      if (gd && a.etraj) {
        if (per_inst) a.etraj[I.etraj_off + step] = E;
        else a.etraj[(size_t)step * a.n_inst + idx] = E;
      }
      a.energy[idx] = E;
    }
    T.sync();
  }
}

__global__ void __launch_bounds__(kBatchThreads, 1) k_batch(BatchArgs a) {
  extern __shared__ double2 sm[];
  __shared__ TeamS S[kWarps];
  __shared__ int s_item;
  const int wi = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= a.n_items) break;
    const int cls = a.items[item].cls;
    // team layout of the item's class (kClassWarps): 1 x 8, 2 x 4, 8 x 1 or 4 x 2 warps
    const int nw = cls == 0 ? 8 : cls == 1 ? 4 : cls == 3 ? 2 : 1;
    const int team = wi / nw;
    Team T;
    T.nw = nw;
    T.size = nw * 32;
    T.log_size = nw == 8 ? 8 : nw == 4 ? 7 : nw == 2 ? 6 : 5;
    T.rank = threadIdx.x - team * T.size;
    T.w = wi - team * nw;
    T.bar = 1 + team;
    const int inst = a.items[item].inst[team];
    if (inst >= 0) {
      const int nteams = kWarps / nw;
      double2* region = sm + (size_t)team * (a.smem_amps / nteams);
      double2* ck = a.ckpt + (size_t)blockIdx.x * a.ckpt_slot +
                    (size_t)team * (a.ckpt_slot / nteams);
      run_instance(a, inst, T, S[team], region, ck);
    }
    __syncthreads();
  }
}

}  // namespace

size_t batch_smem_bytes(int nmax) {
  (void)nmax;
  return (size_t)kBatchSmemAmps * sizeof(double2);
}

cudaError_t batch_prepare(int nmax, int* grid_out) {
  const size_t smem = batch_smem_bytes(nmax);
  cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kBatchThreads,
                                                         smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid_out = sms * per_sm;
  return cudaSuccess;
}

cudaError_t launch_batch(const BatchArgs& a, int grid, size_t smem, cudaStream_t s) {
  k_batch<<<grid, kBatchThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace svqe
