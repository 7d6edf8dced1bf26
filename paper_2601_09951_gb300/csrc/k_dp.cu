// k_dp.cu -- whole-state diagonal + permutation segments of the single-state path.
//
// In a hardware-efficient layer a run of RZ (and CZ) gates is directly followed by a run of
// CNOT (and X) gates.  Fused shared-memory passes need four or more passes for such a run when
// the CNOTs chain through all qubits (a ring or a ladder), each pass moving psi and lambda
// through HBM for very little arithmetic.  Here the run is one streaming pass over the state:
//   * the CNOT/X run is an affine map of the index bits over GF(2), P(k) = T0[k & 2047] ^
//     T1[(k >> 11) & 2047] ^ T2[k >> 22], from three tables staged in shared memory;
//   * the diagonal part is one phase per amplitude, e^{-i sum_q phi_q s_q(k)} (times -1 for
//     the CZ gates that fire), from a table over the 11 low bits (staged) and a factor per
//     block of 2048 amplitudes from two tables over the block index;
//   * the RZ gradients 2 Im<lambda|Z_q/2|psi> = sum_k s_q(k) w_k, w_k = Im(conj(lambda_k)
//     psi_k), are the same at either end of the diagonal part (the phase cancels in w_k), so
//     they are taken from the un-phased lambda and psi: a per-thread sum for the bits fixed in
//     a thread (0-7), three sums for the bits that vary within a block (8-10), and one sum per
//     block-index bit (11 and up).
// Blocks of 2048 consecutive amplitudes are handled by 256 threads, 8 amplitudes each (k =
// base + tid + 256 i).  Out of place: the gather/scatter needs a second buffer.
#include <algorithm>

#include "launch.h"
#include "svqe_internal.cuh"

namespace svqe {

namespace {

constexpr int kDT = 256;     // threads per CTA
constexpr int kDB = 11;      // bits per block
constexpr int kDBlock = 1 << kDB;

__device__ __forceinline__ double2 cmul(const double2& a, const double2& b) {
  return make_double2(fma(a.x, b.x, dneg(a.y) * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul_conj(const double2& a, const double2& b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, dneg(a.x) * b.y));
}

// Dynamic shared memory of every k_dp kernel (56 KiB + reduction scratch).
struct DpShared {
  double2 p0[kDBlock];       // phase over the 11 low bits
  uint32_t t[3][kDBlock];    // permutation tables
  double red[kDT / 32];
};

__device__ __forceinline__ void dp_stage(DpShared& S, const DpArgs& a) {
  for (int j = threadIdx.x; j < 3 * kDBlock; j += kDT) (&S.t[0][0])[j] = a.perm[j];
  for (int j = threadIdx.x; j < kDBlock; j += kDT) S.p0[j] = a.phase_lo[j];
  __syncthreads();
}

__device__ __forceinline__ uint32_t dp_map(const DpShared& S, uint64_t k) {
  return S.t[0][k & (kDBlock - 1)] ^ S.t[1][(k >> kDB) & (kDBlock - 1)] ^ S.t[2][k >> (2 * kDB)];
}

__device__ __forceinline__ double2 dp_outer(const DpArgs& a, uint64_t blk) {
  return cmul(a.phase_b1[blk & 1023], a.phase_b2[blk >> 10]);
}

// The block of visit index t (see DpArgs::pair): bit 0 of t selects pair, bit pair_hi of t
// selects block bit 0, every other bit of t is the same block bit.  A bijection on the block
// indices, because pair has bit pair_hi set.
__device__ __forceinline__ uint64_t dp_block(const DpArgs& a, uint64_t t) {
  if (a.pair <= 1u) return t;
  const uint64_t ep = 1ull << a.pair_hi;
  uint64_t b = t & ~(ep | 1ull);
  if (t & 1ull) b ^= a.pair;
  if (t & ep) b ^= 1ull;
  return b;
}

__device__ __forceinline__ bool dp_cz(const DpArgs& a, uint64_t k) {
  uint32_t par = 0;
  for (int c = 0; c < a.n_cz; ++c) par ^= ((k & a.cz_mask[c]) == a.cz_mask[c]);
  return par & 1u;
}

// Forward: out[P(k)] = phase(k) in[k].
__global__ void __launch_bounds__(kDT) k_dp_fwd(const double2* __restrict__ in,
                                                double2* __restrict__ out, DpArgs a) {
  extern __shared__ double2 dsm[];
  DpShared& S = *reinterpret_cast<DpShared*>(dsm);
  dp_stage(S, a);
  const uint64_t nblk = a.N >> kDB;
  for (uint64_t t = blockIdx.x; t < nblk; t += gridDim.x) {
    const uint64_t blk = dp_block(a, t);
    const double2 o = dp_outer(a, blk);
#pragma unroll
    for (int i = 0; i < kDBlock / kDT; ++i) {
      const uint32_t j = threadIdx.x + i * kDT;
      const uint64_t k = (blk << kDB) | j;
      double2 v = cmul(in[k], cmul(S.p0[j], o));
      if (a.n_cz && dp_cz(a, k)) v = make_double2(dneg(v.x), dneg(v.y));
      out[dp_map(S, k)] = v;
    }
  }
}

// Backward, psi: out[k] = conj(phase(k)) in[P(k)].
__global__ void __launch_bounds__(kDT) k_dp_bwd_psi(const double2* __restrict__ in,
                                                    double2* __restrict__ out, DpArgs a) {
  extern __shared__ double2 dsm[];
  DpShared& S = *reinterpret_cast<DpShared*>(dsm);
  dp_stage(S, a);
  const uint64_t nblk = a.N >> kDB;
  for (uint64_t t = blockIdx.x; t < nblk; t += gridDim.x) {
    const uint64_t blk = dp_block(a, t);
    const double2 o = dp_outer(a, blk);
#pragma unroll
    for (int i = 0; i < kDBlock / kDT; ++i) {
      const uint32_t j = threadIdx.x + i * kDT;
      const uint64_t k = (blk << kDB) | j;
      double2 v = cmul_conj(in[dp_map(S, k)], cmul(S.p0[j], o));
      if (a.n_cz && dp_cz(a, k)) v = make_double2(dneg(v.x), dneg(v.y));
      out[k] = v;
    }
  }
}

// Backward, lambda: out[k] = conj(phase(k)) lam[P(k)], and the RZ gradient shares from
// w_k = Im(conj(out[k]) psi_b[k]) with psi_b the un-phased psi (k_dp_bwd_psi's output):
// partial[op * kRedBlocks + block] for every parameterised RZ op of the segment.  The first
// G = min(blocks, 1024) CTAs do the work, CTA c taking visit indices t = c, c + G, c + 2G, ...
// (block dp_block(t)): bits of t below log2 G are fixed per CTA (their signs apply to the
// CTA's total), and the bits above it are bits of the round r (one sum each, at most 10).
// The other CTAs write zeros.
__global__ void __launch_bounds__(kDT, 2) k_dp_bwd_lam(const double2* __restrict__ lam,
                                                    const double2* __restrict__ psi_b,
                                                    double2* __restrict__ out, DpArgs a,
                                                    double* __restrict__ partial) {
  extern __shared__ double2 dsm[];
  DpShared& S = *reinterpret_cast<DpShared*>(dsm);
  dp_stage(S, a);
  const uint64_t nblk = a.N >> kDB;
  const uint64_t G = nblk < 1024 ? nblk : 1024;
  const int lg = __popcll(G - 1);  // log2 G
  const int nrb = a.n - kDB - lg;  // round bits
  constexpr int kMaxRound = 10;
  double W = 0.0, mid[3] = {0.0, 0.0, 0.0}, hr[kMaxRound];
#pragma unroll
  for (int b = 0; b < kMaxRound; ++b) hr[b] = 0.0;
  if (blockIdx.x < G) {
    uint64_t r = 0;
    for (uint64_t t = blockIdx.x; t < nblk; t += G, ++r) {
      const uint64_t blk = dp_block(a, t);
      const double2 o = dp_outer(a, blk);
      double wb = 0.0;
#pragma unroll
      for (int i = 0; i < kDBlock / kDT; ++i) {
        const uint32_t j = threadIdx.x + i * kDT;
        const uint64_t k = (blk << kDB) | j;
        double2 v = cmul_conj(lam[dp_map(S, k)], cmul(S.p0[j], o));
        if (a.n_cz && dp_cz(a, k)) v = make_double2(dneg(v.x), dneg(v.y));
        out[k] = v;
        const double2 p = psi_b[k];
        const double w = fma(v.x, p.y, dneg(v.y) * p.x);
        wb += w;
#pragma unroll
        for (int q = 0; q < 3; ++q) mid[q] += ((i >> q) & 1) ? dneg(w) : w;
      }
      W += wb;
#pragma unroll
      for (int b = 0; b < kMaxRound; ++b)
        if (b < nrb) hr[b] += ((r >> b) & 1ull) ? dneg(wb) : wb;
    }
  }
  // one CTA reduction per parameterised RZ op
  const int tid = threadIdx.x;
  for (int g = 0; g < a.n_rz; ++g) {
    const int bit = a.rz_bit[g];
    double v;
    if (bit < 8) {
      v = ((tid >> bit) & 1) ? dneg(W) : W;
    } else if (bit < kDB) {
      v = bit == 8 ? mid[0] : bit == 9 ? mid[1] : mid[2];
    } else {
      // block bit jb of the block visited at t = blockIdx.x + r G is bit src of t, flipped by
      // t's bit 0 where pair has bit jb (dp_block); bits of t below lg are the CTA's, the
      // others the round's
      const int jb = bit - kDB;
      const bool paired = a.pair > 1u;
      const bool t0 = blockIdx.x & 1u;
      int src = jb;
      bool flip = false;
      if (paired) {
        if (jb == a.pair_hi) src = 0;
        else if (jb == 0) src = a.pair_hi;
        flip = jb != a.pair_hi && t0 && ((a.pair >> jb) & 1u);
      }
      if (src < lg) {
        v = ((blockIdx.x >> src) & 1u) ? dneg(W) : W;
      } else {
        v = 0.0;
#pragma unroll
        for (int b = 0; b < kMaxRound; ++b)
          if (b == src - lg) v = hr[b];
      }
      if (flip) v = dneg(v);
    }
    v = warp_sum(v);
    if ((tid & 31) == 0) S.red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
      double u = tid < kDT / 32 ? S.red[tid] : 0.0;
      u = warp_sum(u);
      if (tid == 0) partial[(size_t)a.rz_op[g] * kRedBlocks + blockIdx.x] = u;
    }
    __syncthreads();
  }
}

// Phase tables from the step's coefficients: coef of an RZ op holds Rot(theta/2) in lifting
// form, so (cos, sin) are recomputed here from theta (one thread per table entry).
__global__ void k_dp_setup(DpArgs a, const DOp* __restrict__ ops, const double* __restrict__ theta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // entries: [0, 2048) low table, then 1024 + 1024 block tables
  if (t >= kDBlock + 2048) return;
  int lo_bit, nbits;
  uint32_t idx;
  double2* dst;
  if (t < kDBlock) {
    lo_bit = 0; nbits = kDB; idx = (uint32_t)t; dst = a.phase_lo_w + t;
  } else if (t < kDBlock + 1024) {
    lo_bit = kDB; nbits = 10; idx = (uint32_t)(t - kDBlock); dst = a.phase_b1_w + idx;
  } else {
    lo_bit = kDB + 10; nbits = 10; idx = (uint32_t)(t - kDBlock - 1024); dst = a.phase_b2_w + idx;
  }
  double2 p = make_double2(1.0, 0.0);
  for (int g = 0; g < a.n_rz_all; ++g) {
    const DOp op = ops[a.rz_all[g]];
    const int b = op.bit0;
    if (b < lo_bit || b >= lo_bit + nbits) continue;
    const double th = op.param >= 0 ? theta[op.param] : op.fixed;
    double s, c;
    sincos(0.5 * th, &s, &c);
    const bool one = (idx >> (b - lo_bit)) & 1u;
    p = cmul(p, make_double2(c, one ? s : dneg(s)));  // e^{-i phi} on |0>, e^{+i phi} on |1>
  }
  *dst = p;
}

}  // namespace

cudaError_t dp_prepare() {
  const int sm = (int)sizeof(DpShared);
  cudaError_t e = cudaFuncSetAttribute(k_dp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_dp_bwd_psi, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_dp_bwd_lam, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

cudaError_t launch_dp_setup(const DpArgs& a, const DOp* ops, const double* theta,
                            cudaStream_t s) {
  k_dp_setup<<<(kDBlock + 2048 + 255) / 256, 256, 0, s>>>(a, ops, theta);
  return cudaGetLastError();
}

static int dp_grid(const DpArgs& a) {
  const uint64_t nblk = a.N >> kDB;
  return (int)std::min<uint64_t>(nblk, kRedBlocks);
}

cudaError_t launch_dp_fwd(const double2* in, double2* out, const DpArgs& a, cudaStream_t s) {
  k_dp_fwd<<<dp_grid(a), kDT, sizeof(DpShared), s>>>(in, out, a);
  return cudaGetLastError();
}

cudaError_t launch_dp_bwd_psi(const double2* in, double2* out, const DpArgs& a,
                              cudaStream_t s) {
  k_dp_bwd_psi<<<dp_grid(a), kDT, sizeof(DpShared), s>>>(in, out, a);
  return cudaGetLastError();
}

cudaError_t launch_dp_bwd_lam(const double2* lam, const double2* psi_b, double2* out,
                              const DpArgs& a, double* partial, cudaStream_t s) {
  // every block writes its share of every RZ op: the grid must be kRedBlocks
  k_dp_bwd_lam<<<kRedBlocks, kDT, sizeof(DpShared), s>>>(lam, psi_b, out, a, partial);
  return cudaGetLastError();
}

}  // namespace svqe
