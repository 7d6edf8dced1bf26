// k_fused.cu -- fused passes of the single-state path (see FPass): a tile of 2^m amplitudes
// is staged in shared memory, a whole run of gates is applied to it, and it is written back,
// so the run costs one read and one write of the HBM-resident state instead of one per gate.
//
// Forward:  k_fpass applies the pass's items to psi.
// Backward: k_bpass stages psi and lambda, walks the items in reverse, accumulates each
//           parameterised item's 2 Im<lambda|G|psi> in a per-thread shared-memory slot (one
//           DADD per item per tile instead of a warp reduction), un-applies the items to both,
//           and reduces every slot once at the end into partial[op * kRedBlocks + block] (one
//           block per tile up to kRedBlocks; the caller zeroes the partials beforehand, so the
//           entries of blocks a small pass does not launch read as zero).
// A run of RZ gates is one diagonal phase per amplitude: half tables over the tile's local
// bits times a per-tile factor for the RZ gates on outer bits.
#include <algorithm>

#include "launch.h"
#include "svqe_internal.cuh"

namespace svqe {

namespace {

constexpr int kFT = 256;  // threads per CTA of the fused kernels

struct DiagS {
  double2 cs[kMaxSlotsDev];  // (cos phi, sin phi) per RZ gate of the item
  int loc[kMaxSlotsDev];     // local bit, or -1 - global bit for a gate on an outer bit
  double2 tl[64];            // phase over local bits [0, hl)
  double2 th[64];            // phase over local bits [hl, m), times the tile's outer factor
  double2 th0[64];           // phase over local bits [hl, m) alone
  int m_rz;
  int hl;
};

__device__ __forceinline__ double2 cmul(const double2& a, const double2& b) {
  return make_double2(fma(a.x, b.x, dneg(a.y) * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul_conj(const double2& a, const double2& b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, dneg(a.x) * b.y));
}
__device__ __forceinline__ double2 rz_factor(const double2& cs, int bit) {
  return make_double2(cs.x, bit ? cs.y : dneg(cs.y));  // e^{-i phi} on |0>, e^{+i phi} on |1>
}

__device__ __forceinline__ uint64_t pdep64(uint64_t v, uint64_t m) {
  uint64_t r = 0;
  while (m) {
    const uint64_t low = m & (0ull - m);
    if (v & 1ull) r |= low;
    v >>= 1;
    m &= m - 1;
  }
  return r;
}

// Per-CTA setup of a diagonal item: cos/sin, local bits and the inner half tables.
__device__ void diag_setup(DiagS& D, const FPass& P, const FItem& it, const DOp* gops,
                           const double* theta) {
  if (threadIdx.x == 0) {
    D.m_rz = it.count;
    D.hl = P.m / 2;
  }
  if ((int)threadIdx.x < it.count) {
    const DOp op = gops[it.op + threadIdx.x];
    const double t = op.param >= 0 ? theta[op.param] : op.fixed;
    double s, c;
    sincos(0.5 * t, &s, &c);
    D.cs[threadIdx.x] = make_double2(c, s);
    const uint64_t b = 1ull << op.bit0;
    D.loc[threadIdx.x] = (P.tile_mask & b) ? __popcll(P.tile_mask & (b - 1ull)) : -1 - op.bit0;
  }
  __syncthreads();
  const int hl = D.hl;
  const int nl = 1 << hl, nh = 1 << (P.m - hl);
  for (int j = threadIdx.x; j < nl + nh; j += blockDim.x) {
    const bool hi = j >= nl;
    const int jj = hi ? j - nl : j;
    double2 p = make_double2(1.0, 0.0);
    for (int g = 0; g < D.m_rz; ++g) {
      const int lb = D.loc[g];
      if (lb < 0 || (lb >= hl) != hi) continue;
      p = cmul(p, rz_factor(D.cs[g], (jj >> (hi ? lb - hl : lb)) & 1));
    }
    if (hi) D.th0[jj] = p; else D.tl[jj] = p;
  }
  __syncthreads();
}

// Per-tile: th = th0 * (product of the outer-bit RZ factors for this tile).
__device__ void diag_tile(DiagS& D, const FPass& P, uint64_t outer) {
  double2 f = make_double2(1.0, 0.0);
  for (int g = 0; g < D.m_rz; ++g)
    if (D.loc[g] < 0) f = cmul(f, rz_factor(D.cs[g], (int)((outer >> (-1 - D.loc[g])) & 1ull)));
  const int nh = 1 << (P.m - D.hl);
  for (int j = threadIdx.x; j < nh; j += blockDim.x) D.th[j] = cmul(D.th0[j], f);
}

__device__ __forceinline__ double2 diag_phase(const DiagS& D, uint32_t j) {
  return cmul(D.th[j >> D.hl], D.tl[j & ((1u << D.hl) - 1u)]);
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only): a tile's loads are all in
// flight at once instead of one round trip per loop iteration; cp_async_wait_all and a
// barrier complete them.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Tile-local index j -> global amplitude index.
__device__ __forceinline__ uint64_t gidx(const uint64_t* hoff, uint32_t j, int c,
                                         uint64_t outer) {
  return hoff[j >> c] | (uint64_t)(j & ((1u << c) - 1u)) | outer;
}

__device__ void setup_hoff(uint64_t* hoff, const FPass& P) {
  const uint64_t hm = P.tile_mask & ~((1ull << P.c) - 1ull);
  for (int j = threadIdx.x; j < (1 << (P.m - P.c)); j += blockDim.x) hoff[j] = pdep64(j, hm);
}

enum FKind { F_SWAP = 0, F_H = 1, F_ROTY = 2, F_ROTX = 3, F_ROTZ = 4, F_NEG = 5 };

__device__ __forceinline__ int fkind_of(int type) {
  switch (type) {
    case SV_GATE_H: return F_H;
    case SV_GATE_RY: case SV_GATE_SINGLE_EXC: case SV_GATE_DOUBLE_EXC: return F_ROTY;
    case SV_GATE_RX: return F_ROTX;
    case SV_GATE_RZ: return F_ROTZ;
    case SV_GATE_CZ: return F_NEG;
    default: return F_SWAP;
  }
}

// One pair of one kind with oriented coefficients (the caller takes the inverse).
template <int KIND>
__device__ __forceinline__ void fapply(const Rot& r, double2& x, double2& y) {
  if (KIND == F_SWAP) {
    const double2 t = x; x = y; y = t;
  } else if (KIND == F_H) {
    pair_apply(SV_GATE_H, r, false, x, y);
  } else if (KIND == F_ROTY) {
    rot_apply(r, x.x, y.x);
    rot_apply(r, x.y, y.y);
  } else if (KIND == F_ROTX) {
    const Rot m = rot_inverse(r);
    rot_apply(m, x.x, y.y);
    rot_apply(r, x.y, y.x);
  } else if (KIND == F_ROTZ) {
    const Rot m = rot_inverse(r);
    rot_apply(m, x.x, x.y);
    rot_apply(r, y.x, y.y);
  }
}

// acc += 2 Im<lambda|G|psi> on one pair, folded into FMAs.
template <int KIND>
__device__ __forceinline__ void fgrad(const double2& lx, const double2& ly, const double2& px,
                                      const double2& py, double& acc) {
  if (KIND == F_ROTX) {
    acc = fma(lx.x, py.y, acc);
    acc = fma(dneg(lx.y), py.x, acc);
    acc = fma(ly.x, px.y, acc);
    acc = fma(dneg(ly.y), px.x, acc);
  } else if (KIND == F_ROTZ) {
    acc = fma(lx.x, px.y, acc);
    acc = fma(dneg(lx.y), px.x, acc);
    acc = fma(dneg(ly.x), py.y, acc);
    acc = fma(ly.y, py.x, acc);
  } else if (KIND == F_ROTY) {
    acc = fma(ly.x, px.x, acc);
    acc = fma(ly.y, px.y, acc);
    acc = fma(dneg(lx.x), py.x, acc);
    acc = fma(dneg(lx.y), py.y, acc);
  }
}

template <int KIND>
__device__ __forceinline__ void tile_op_k(double2* v, uint32_t M, const DOp& op, const Rot& r) {
  const uint32_t np = M >> op.k;
  const uint32_t lo = (uint32_t)op.lo_or, fl = (uint32_t)op.flip;
  for (uint32_t p = threadIdx.x; p < np; p += kFT) {
    const uint32_t i = (uint32_t)insert_zeros(p, op.sb, op.k) | lo;
    if (KIND == F_NEG) {
      v[i] = make_double2(dneg(v[i].x), dneg(v[i].y));
    } else {
      double2 x = v[i], y = v[i ^ fl];
      fapply<KIND>(r, x, y);
      v[i] = x;
      v[i ^ fl] = y;
    }
  }
}

__device__ __forceinline__ void tile_op(double2* v, uint32_t M, const DOp& op, const Rot& rf,
                                        bool inv) {
  const Rot r = inv ? rot_inverse(rf) : rf;
  switch (fkind_of(op.type)) {
    case F_SWAP: tile_op_k<F_SWAP>(v, M, op, r); break;
    case F_H: tile_op_k<F_H>(v, M, op, r); break;
    case F_ROTY: tile_op_k<F_ROTY>(v, M, op, r); break;
    case F_ROTX: tile_op_k<F_ROTX>(v, M, op, r); break;
    case F_ROTZ: tile_op_k<F_ROTZ>(v, M, op, r); break;
    default: tile_op_k<F_NEG>(v, M, op, r); break;
  }
}

// Adjoint step of one op on the psi and lambda tiles: gradient share into acc (if grad), then
// un-apply to both.
template <int KIND>
__device__ __forceinline__ void tile_adj_k(double2* tp, double2* tl, uint32_t M, const DOp& op,
                                           const Rot& ri, bool grad, double& acc) {
  const uint32_t np = M >> op.k;
  const uint32_t lo = (uint32_t)op.lo_or, fl = (uint32_t)op.flip;
  for (uint32_t p = threadIdx.x; p < np; p += kFT) {
    const uint32_t a = (uint32_t)insert_zeros(p, op.sb, op.k) | lo;
    if (KIND == F_NEG) {
      tp[a] = make_double2(dneg(tp[a].x), dneg(tp[a].y));
      tl[a] = make_double2(dneg(tl[a].x), dneg(tl[a].y));
    } else {
      double2 px = tp[a], py = tp[a ^ fl], lx = tl[a], ly = tl[a ^ fl];
      if (grad) fgrad<KIND>(lx, ly, px, py, acc);
      fapply<KIND>(ri, px, py);
      fapply<KIND>(ri, lx, ly);
      tp[a] = px;
      tp[a ^ fl] = py;
      tl[a] = lx;
      tl[a ^ fl] = ly;
    }
  }
}

// INV: apply the pass's items inverted, in reverse order (un-applying the pass).
template <bool INV>
__global__ void __launch_bounds__(kFT) k_fpass(double2* __restrict__ psi, FPass P,
                                               const FItem* __restrict__ items,
                                               const DOp* __restrict__ gops,
                                               const Rot* __restrict__ coef,
                                               const double* __restrict__ theta) {
  extern __shared__ double2 tile[];
  __shared__ uint64_t hoff[1 << (11 - kMinLowBitsL2)];
  __shared__ DiagS D;
  const uint32_t M = 1u << P.m;
  const uint64_t ntiles = 1ull << __popcll(P.outer_mask);
  int diag = -1;
  for (int i = 0; i < P.n_items; ++i)
    if (items[P.first_item + i].kind == 1) diag = i;
  setup_hoff(hoff, P);
  if (diag >= 0) diag_setup(D, P, items[P.first_item + diag], gops, theta);
  __syncthreads();
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t outer = pdep64(t, P.outer_mask);
    for (uint32_t j = threadIdx.x; j < M; j += kFT)
      cp_async16(&tile[j], &psi[gidx(hoff, j, P.c, outer)]);
    cp_async_wait_all();
    if (diag >= 0) diag_tile(D, P, outer);
    __syncthreads();
    for (int ii = 0; ii < P.n_items; ++ii) {
      const int i = INV ? P.n_items - 1 - ii : ii;
      const FItem it = items[P.first_item + i];
      if (it.kind == 0) {
        tile_op(tile, M, it.local, coef[it.op], INV);
      } else if (INV) {
        for (uint32_t j = threadIdx.x; j < M; j += kFT)
          tile[j] = cmul_conj(tile[j], diag_phase(D, j));
      } else {
        for (uint32_t j = threadIdx.x; j < M; j += kFT) tile[j] = cmul(tile[j], diag_phase(D, j));
      }
      __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < M; j += kFT) psi[gidx(hoff, j, P.c, outer)] = tile[j];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kFT) k_bpass(double2* __restrict__ psi,
                                               double2* __restrict__ lam, FPass P,
                                               const FItem* __restrict__ items,
                                               const DOp* __restrict__ gops,
                                               const Rot* __restrict__ coef,
                                               const double* __restrict__ theta,
                                               double* __restrict__ partial) {
  extern __shared__ double2 smem[];
  __shared__ uint64_t hoff[1 << (11 - kMinLowBitsL2)];
  __shared__ DiagS D;
  __shared__ double red[kFT / 32];
  const uint32_t M = 1u << P.m;
  double2* tp = smem;
  double2* tlam = smem + M;
  double* accp = (double*)(smem + 2 * M);  // [n_slots][kFT]
  const uint64_t ntiles = 1ull << __popcll(P.outer_mask);
  const int tid = threadIdx.x;
  int diag = -1;
  for (int i = 0; i < P.n_items; ++i)
    if (items[P.first_item + i].kind == 1) diag = i;
  for (int s = 0; s < P.n_slots; ++s) accp[s * kFT + tid] = 0.0;
  setup_hoff(hoff, P);
  if (diag >= 0) diag_setup(D, P, items[P.first_item + diag], gops, theta);
  __syncthreads();
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t outer = pdep64(t, P.outer_mask);
    for (uint32_t j = tid; j < M; j += kFT) {
      const uint64_t k = gidx(hoff, j, P.c, outer);
      cp_async16(&tp[j], &psi[k]);
      cp_async16(&tlam[j], &lam[k]);
    }
    cp_async_wait_all();
    if (diag >= 0) diag_tile(D, P, outer);
    __syncthreads();
    for (int i = P.n_items - 1; i >= 0; --i) {
      const FItem it = items[P.first_item + i];
      if (it.kind == 0) {
        const DOp& op = it.local;
        const Rot ri = rot_inverse(coef[it.op]);
        const bool gr = it.slot >= 0;
        double acc = 0.0;
        switch (fkind_of(op.type)) {
          case F_SWAP: tile_adj_k<F_SWAP>(tp, tlam, M, op, ri, false, acc); break;
          case F_H: tile_adj_k<F_H>(tp, tlam, M, op, ri, false, acc); break;
          case F_ROTY: tile_adj_k<F_ROTY>(tp, tlam, M, op, ri, gr, acc); break;
          case F_ROTX: tile_adj_k<F_ROTX>(tp, tlam, M, op, ri, gr, acc); break;
          case F_ROTZ: tile_adj_k<F_ROTZ>(tp, tlam, M, op, ri, gr, acc); break;
          default: tile_adj_k<F_NEG>(tp, tlam, M, op, ri, false, acc); break;
        }
        if (gr) accp[it.slot * kFT + tid] += acc;
      } else {
        // gradients of the RZ gates: 2 Im<lambda|Z_q/2|psi> = sum_k s_q(k) Im(conj(l_k) p_k)
        double W = 0.0;
        double hi[3] = {0.0, 0.0, 0.0};  // RZ gates on local bits 8..10 (vary within a thread)
        for (uint32_t j = tid; j < M; j += kFT) {
          const double2 pk = tp[j], lk = tlam[j];
          const double w = fma(lk.x, pk.y, dneg(lk.y) * pk.x);
          W += w;
#pragma unroll
          for (int q = 0; q < 3; ++q) hi[q] += ((j >> (8 + q)) & 1u) ? dneg(w) : w;
          const double2 ph = diag_phase(D, j);
          tp[j] = cmul_conj(pk, ph);
          tlam[j] = cmul_conj(lk, ph);
        }
        int s = it.slot;
        for (int g = 0; g < it.count; ++g) {
          const DOp op = gops[it.op + g];
          if (op.param < 0) continue;
          const int lb = D.loc[g];
          double v;
          if (lb < 0) {
            v = ((outer >> (-1 - lb)) & 1ull) ? dneg(W) : W;
          } else if (lb < 8) {
            v = ((tid >> lb) & 1) ? dneg(W) : W;
          } else {
            v = lb == 8 ? hi[0] : lb == 9 ? hi[1] : hi[2];
          }
          accp[s * kFT + tid] += v;
          ++s;
        }
      }
      __syncthreads();
    }
    for (uint32_t j = tid; j < M; j += kFT) {
      const uint64_t k = gidx(hoff, j, P.c, outer);
      psi[k] = tp[j];
      lam[k] = tlam[j];
    }
    __syncthreads();
  }
  // one block reduction per slot, written to the slot's op
  int s = 0;
  for (int i = 0; i < P.n_items; ++i) {
    const FItem it = items[P.first_item + i];
    if (it.slot < 0) continue;
    const int cnt = it.kind == 0 ? 1 : it.count;
    for (int g = 0; g < cnt; ++g) {
      const int op = it.op + g;
      if (gops[op].param < 0) continue;
      double v = warp_sum(accp[s * kFT + tid]);
      if ((tid & 31) == 0) red[tid >> 5] = v;
      __syncthreads();
      if (tid < 32) {
        double u = tid < kFT / 32 ? red[tid] : 0.0;
        u = warp_sum(u);
        if (tid == 0) partial[(size_t)op * kRedBlocks + blockIdx.x] = u;
      }
      __syncthreads();
      ++s;
    }
  }
}

// Gradients only: 2 Im<lambda|G|psi> of every parameterised single-op item of the pass from
// the unchanged psi and lambda tiles (no un-apply, no stores).  Used for a commuting layer
// whose gradients are all taken at the layer's end; the tiles are read-only, so the items need
// no barrier between them.
__global__ void __launch_bounds__(kFT) k_gpass(const double2* __restrict__ psi,
                                               const double2* __restrict__ lam, FPass P,
                                               const FItem* __restrict__ items,
                                               double* __restrict__ partial) {
  extern __shared__ double2 smem[];
  __shared__ uint64_t hoff[1 << (11 - kMinLowBitsL2)];
  __shared__ double red[kFT / 32];
  const uint32_t M = 1u << P.m;
  double2* tp = smem;
  double2* tlam = smem + M;
  double* accp = (double*)(smem + 2 * M);  // [n_slots][kFT]
  const uint64_t ntiles = 1ull << __popcll(P.outer_mask);
  const int tid = threadIdx.x;
  for (int s = 0; s < P.n_slots; ++s) accp[s * kFT + tid] = 0.0;
  setup_hoff(hoff, P);
  __syncthreads();
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t outer = pdep64(t, P.outer_mask);
    for (uint32_t j = tid; j < M; j += kFT) {
      const uint64_t k = gidx(hoff, j, P.c, outer);
      cp_async16(&tp[j], &psi[k]);
      cp_async16(&tlam[j], &lam[k]);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int i = 0; i < P.n_items; ++i) {
      const FItem it = items[P.first_item + i];
      if (it.kind != 0 || it.slot < 0) continue;
      const DOp& op = it.local;
      const uint32_t np = M >> op.k;
      const uint32_t lo = (uint32_t)op.lo_or, fl = (uint32_t)op.flip;
      const int kind = fkind_of(op.type);
      double acc = 0.0;
      for (uint32_t p = tid; p < np; p += kFT) {
        const uint32_t a = (uint32_t)insert_zeros(p, op.sb, op.k) | lo;
        const double2 px = tp[a], py = tp[a ^ fl], lx = tlam[a], ly = tlam[a ^ fl];
        if (kind == F_ROTX) fgrad<F_ROTX>(lx, ly, px, py, acc);
        else if (kind == F_ROTZ) fgrad<F_ROTZ>(lx, ly, px, py, acc);
        else fgrad<F_ROTY>(lx, ly, px, py, acc);
      }
      accp[it.slot * kFT + tid] += acc;
    }
    __syncthreads();
  }
  for (int i = 0; i < P.n_items; ++i) {
    const FItem it = items[P.first_item + i];
    if (it.kind != 0 || it.slot < 0) continue;
    double v = warp_sum(accp[it.slot * kFT + tid]);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
      double u = tid < kFT / 32 ? red[tid] : 0.0;
      u = warp_sum(u);
      if (tid == 0) partial[(size_t)it.op * kRedBlocks + blockIdx.x] = u;
    }
    __syncthreads();
  }
}

}  // namespace

int fused_tile_bits() { return 11; }

size_t fpass_smem(int m) { return ((size_t)1 << m) * sizeof(double2); }
size_t bpass_smem(int m, int slots) {
  return 2 * ((size_t)1 << m) * sizeof(double2) + (size_t)slots * kFT * sizeof(double);
}

cudaError_t fused_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_fpass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fpass_smem(12));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fpass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fpass_smem(12));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gpass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bpass_smem(11, kMaxSlotsDev));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_bpass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bpass_smem(11, kMaxSlotsDev));
}

cudaError_t launch_fpass(double2* psi, const FPass& P, const FItem* items, const DOp* gops,
                         const Rot* coef, const double* theta, cudaStream_t s) {
  const uint64_t ntiles = 1ull << __builtin_popcountll(P.outer_mask);
  const int grid = (int)std::min<uint64_t>(ntiles, kRedBlocks);
  k_fpass<false><<<grid, kFT, fpass_smem(P.m), s>>>(psi, P, items, gops, coef, theta);
  return cudaGetLastError();
}

cudaError_t launch_fpass_inv(double2* v, const FPass& P, const FItem* items, const DOp* gops,
                             const Rot* coef, const double* theta, cudaStream_t s) {
  const uint64_t ntiles = 1ull << __builtin_popcountll(P.outer_mask);
  const int grid = (int)std::min<uint64_t>(ntiles, kRedBlocks);
  k_fpass<true><<<grid, kFT, fpass_smem(P.m), s>>>(v, P, items, gops, coef, theta);
  return cudaGetLastError();
}

cudaError_t launch_gpass(const double2* psi, const double2* lam, const FPass& P,
                         const FItem* items, const DOp* gops, double* partial, cudaStream_t s) {
  (void)gops;
  const uint64_t ntiles = 1ull << __builtin_popcountll(P.outer_mask);
  const int grid = (int)std::min<uint64_t>(ntiles, kRedBlocks);
  k_gpass<<<grid, kFT, bpass_smem(P.m, P.n_slots), s>>>(psi, lam, P, items, partial);
  return cudaGetLastError();
}

cudaError_t launch_bpass(double2* psi, double2* lam, const FPass& P, const FItem* items,
                         const DOp* gops, const Rot* coef, const double* theta, double* partial,
                         cudaStream_t s) {
  const uint64_t ntiles = 1ull << __builtin_popcountll(P.outer_mask);
  const int grid = (int)std::min<uint64_t>(ntiles, kRedBlocks);
  k_bpass<<<grid, kFT, bpass_smem(P.m, P.n_slots), s>>>(psi, lam, P, items, gops, coef,
                                                               theta, partial);
  return cudaGetLastError();
}

}  // namespace svqe
