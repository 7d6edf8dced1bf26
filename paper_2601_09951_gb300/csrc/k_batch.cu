// k_batch.cu -- the persistent batched kernel: many small independent instances (Sec. 4.1,
// Eq. 7: every bond length / parameter set is its own problem) in one launch.
//
// One CTA runs one instance at a time, taken from a cost-sorted queue with an atomic counter
// (largest first, so the tail is made of cheap instances).  The instance's psi and lambda
// (2 x 2^n x 16 bytes, n <= 12) live in shared memory for the forward pass, lambda = H psi
// and the adjoint sweep.  GB300's FP64 pipe (2 DFMA/clk/SM) is the binding resource, so the
// op list is executed in segments (see Seg) that cut FP64 work:
//   * a run of RZ/CZ is one diagonal phase per amplitude from two half tables (8 FP64 ops per
//     amplitude instead of 3 per RZ gate);
//   * a commuting layer of RY (or RX) gates takes all its gradients at the layer's end, and
//     the sweep un-applies it to lambda only, reloading psi from a checkpoint that the forward
//     pass stored in global memory (bandwidth is plentiful, FP64 issue is not);
//   * several gradients are reduced at once with a transposed warp reduction.
// Every sum runs in a fixed order that does not depend on which CTA or SM ran the instance,
// so an instance's result is bit-identical alone or in any batch.
#include "launch.h"
#include "svqe_internal.cuh"

namespace svqe {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kM = 16;  // values reduced at once (kMaxLayer)

template <int BT>
struct Smem {
  double red[BT / 32];
  double red16[BT / 32][kM];
  double2 tl[64];
  double2 th[64];
  double2 cs[kM];
  int rz_op[kM];
  int rz_bit[kM];
  int item;
};

// Sum over the block of one value per thread; result valid in thread 0.  Caller syncs
// before `red` is reused.
template <int BT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < BT / 32) ? red[l] : 0.0;
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

// Block totals of v[0..m): thread j < m returns the total of value j (fixed order); other
// threads return 0.  Ends synchronised.
template <int BT>
__device__ __forceinline__ double block_sum16(double (&v)[kM], int m, double (*red16)[kM]) {
  const double t = warp_sum16(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if ((l & 1) == 0) red16[w][l >> 1] = t;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < m) {
#pragma unroll
    for (int k = 0; k < BT / 32; ++k) s += red16[k][threadIdx.x];
  }
  __syncthreads();
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

// Apply one pair op to buffer v (forward or inverse), pairs strided over the block.
template <int BT>
__device__ __forceinline__ void op_pass(double2* v, uint32_t N, const DOp& op, const Rot& r,
                                        bool inv) {
  const uint32_t np = N >> op.k;
  for (uint32_t p = threadIdx.x; p < np; p += BT) {
    const uint32_t i = (uint32_t)insert_zeros(p, op.sb, op.k) | (uint32_t)op.lo_or;
    if (op.type == SV_GATE_CZ) {
      v[i] = make_double2(dneg(v[i].x), dneg(v[i].y));
    } else {
      const uint32_t j = i ^ (uint32_t)op.flip;
      double2 x = v[i], y = v[j];
      pair_apply(op.type, r, inv, x, y);
      v[i] = x;
      v[j] = y;
    }
  }
}

// Build the diagonal segment's half tables: th[hi] * tl[lo] = prod_RZ e^{-i phi s(k)}.
template <int BT>
__device__ __forceinline__ int diag_setup(Smem<BT>& S, const DOp* ops, const Seg& sg,
                                          const double* theta, int n) {
  int m = 0;
  for (int l = 0; l < sg.count; ++l)
    if (ops[sg.first + l].type == SV_GATE_RZ) {
      if (threadIdx.x == 0) {
        S.rz_op[m] = sg.first + l;
        S.rz_bit[m] = ops[sg.first + l].bit0;
      }
      ++m;
    }
  __syncthreads();
  if (threadIdx.x < m) {
    const DOp op = ops[S.rz_op[threadIdx.x]];
    const double t = op.param >= 0 ? theta[op.param] : op.fixed;
    double sn, cs;
    sincos(0.5 * t, &sn, &cs);
    S.cs[threadIdx.x] = make_double2(cs, sn);
  }
  __syncthreads();
  const int hl = n < 6 ? n : 6;
  const int nl = 1 << hl, nh = 1 << (n - hl);
  for (int j = threadIdx.x; j < nl + nh; j += BT) {
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
  __syncthreads();
  return m;
}

// Sign of the CZ gates of a diagonal segment at amplitude k (true = negative).
__device__ __forceinline__ bool cz_sign(const DOp* ops, const Seg& sg, uint32_t k) {
  uint32_t par = 0;
  for (int l = 0; l < sg.count; ++l) {
    const DOp& op = ops[sg.first + l];
    if (op.type == SV_GATE_CZ) par ^= ((k & (uint32_t)op.lo_or) == (uint32_t)op.lo_or);
  }
  return par & 1u;
}

template <int BT>
__device__ void run_instance(const BatchArgs& a, int idx, double2* sm, Smem<BT>& S) {
  const BInst I = a.inst[idx];
  const int n = I.n;
  const uint32_t N = 1u << n;
  double2* psi = sm;
  double2* lam = sm + N;
  const DOp* ops = a.ops + I.op_off;
  const DGroup* groups = a.groups + I.grp_off;
  const Seg* segs = a.segs + I.seg_off;
  Rot* coef = a.coef + I.op_off;
  double* contrib = a.contrib + I.op_off;
  double* theta = a.theta + I.theta_off;
  double* grad = a.grad + I.theta_off;
  double2* ck = a.ckpt + (size_t)blockIdx.x * a.ckpt_slot;
  const int tid = threadIdx.x;
  const int hl = n < 6 ? n : 6;
  const uint32_t lmask = (1u << hl) - 1u;
  const int steps = a.n_steps > 0 ? a.n_steps : 1;
  const double lr = a.lr_inst ? a.lr_inst[idx] : a.lr;
  constexpr int kLogBT = BT == 128 ? 7 : BT == 256 ? 8 : BT == 512 ? 9 : 10;

  for (int step = 0; step < steps; ++step) {
    for (int g = tid; g < I.n_ops; g += BT) coef[g] = make_coef(ops[g], theta).r;
    for (uint32_t k = tid; k < N; k += BT)
      psi[k] = make_double2(k == (uint32_t)I.ref ? 1.0 : 0.0, 0.0);
    __syncthreads();

    // ---------------------------------------------------------------- forward
    for (int s = 0; s < I.n_segs; ++s) {
      const Seg sg = segs[s];
      if (sg.ckpt >= 0) {
        double2* dst = ck + (size_t)sg.ckpt * N;
        for (uint32_t k = tid; k < N; k += BT) dst[k] = psi[k];
        __syncthreads();
      }
      if (sg.kind == SEG_DIAG) {
        diag_setup<BT>(S, ops, sg, theta, n);
        for (uint32_t k = tid; k < N; k += BT) {
          const double2 ph = cmul(S.th[k >> hl], S.tl[k & lmask]);
          double2 v = cmul(psi[k], ph);
          if (cz_sign(ops, sg, k)) v = make_double2(dneg(v.x), dneg(v.y));
          psi[k] = v;
        }
        __syncthreads();
      } else {
        for (int l = sg.first; l < sg.first + sg.count; ++l) {
          op_pass<BT>(psi, N, ops[l], coef[l], false);
          __syncthreads();
        }
      }
    }

    // ---------------------------------------------------------------- lambda = H psi
    double e = 0.0;
    for (uint32_t k = tid; k < N; k += BT) {
      double2 acc = make_double2(0.0, 0.0);
      for (int g = 0; g < I.n_groups; ++g) {
        const DGroup G = groups[g];
        const double2 v = psi[k ^ (uint32_t)G.x];
        const uint32_t ti = (G.zu == (uint64_t)(N - 1)) ? k : pext64(k, G.zu);
        const double2 f = a.tables[G.toff + ti];
        group_madd(G.cls, f, v, acc);
      }
      lam[k] = acc;
      const double2 p = psi[k];
      e = fma(p.x, acc.x, e);
      e = fma(p.y, acc.y, e);
    }
    const double E = block_sum<BT>(e, S.red);
    __syncthreads();

    // ---------------------------------------------------------------- adjoint sweep
    for (int s = I.n_segs - 1; s >= 0; --s) {
      const Seg sg = segs[s];
      if (sg.kind == SEG_GATES) {
        for (int l = sg.first + sg.count - 1; l >= sg.first; --l) {
          const DOp op = ops[l];
          const Rot r = coef[l];
          const uint32_t np = N >> op.k;
          const bool pg = op.param >= 0;
          double acc = 0.0;
          for (uint32_t p = tid; p < np; p += BT) {
            const uint32_t i = (uint32_t)insert_zeros(p, op.sb, op.k) | (uint32_t)op.lo_or;
            if (op.type == SV_GATE_CZ) {
              psi[i] = make_double2(dneg(psi[i].x), dneg(psi[i].y));
              lam[i] = make_double2(dneg(lam[i].x), dneg(lam[i].y));
            } else {
              const uint32_t j = i ^ (uint32_t)op.flip;
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
            const double t = block_sum<BT>(acc, S.red);
            if (tid == 0) contrib[l] = t;
          }
          __syncthreads();
        }
        continue;
      }
      double v[kM];
#pragma unroll
      for (int g = 0; g < kM; ++g) v[g] = 0.0;
      if (sg.kind == SEG_RLAYER) {
        // gradients of every gate from (psi, lambda) at the layer's end
        for (int g = 0; g < sg.count; ++g) {
          const DOp op = ops[sg.first + g];
          double acc = 0.0;
          const uint32_t np = N >> 1;
          for (uint32_t p = tid; p < np; p += BT) {
            const uint32_t i = (uint32_t)insert_zeros(p, op.sb, 1);
            const uint32_t j = i ^ (uint32_t)op.flip;
            pair_grad_acc(op.type, lam[i], lam[j], psi[i], psi[j], acc);
          }
#pragma unroll
          for (int q = 0; q < kM; ++q)
            if (q == g) v[q] = acc;
        }
        const double tot = block_sum16<BT>(v, sg.count, S.red16);
        if (tid < sg.count) contrib[sg.first + tid] = tot;
        // un-apply the layer to lambda
        for (int l = sg.first + sg.count - 1; l >= sg.first; --l) {
          op_pass<BT>(lam, N, ops[l], coef[l], true);
          __syncthreads();
        }
      } else {  // SEG_DIAG
        const int m = diag_setup<BT>(S, ops, sg, theta, n);
        double W = 0.0;
        for (uint32_t k = tid; k < N; k += BT) {
          const double2 pk = psi[k];
          double2 lk = lam[k];
          const double w = fma(lk.x, pk.y, dneg(lk.y) * pk.x);  // Im(conj(lambda) psi)
          W += w;
#pragma unroll
          for (int g = 0; g < kM; ++g)
            if (g < m && S.rz_bit[g] >= kLogBT)
              v[g] += ((k >> S.rz_bit[g]) & 1u) ? dneg(w) : w;
          const double2 ph = cmul(S.th[k >> hl], S.tl[k & lmask]);
          lk = cmul_conj(lk, ph);
          if (cz_sign(ops, sg, k)) lk = make_double2(dneg(lk.x), dneg(lk.y));
          lam[k] = lk;
        }
#pragma unroll
        for (int g = 0; g < kM; ++g)
          if (g < m && S.rz_bit[g] < kLogBT)
            v[g] = (((uint32_t)tid >> S.rz_bit[g]) & 1u) ? dneg(W) : W;
        const double tot = block_sum16<BT>(v, m, S.red16);
        if (tid < m) contrib[S.rz_op[tid]] = tot;
      }
      // psi before the segment, from the forward pass's checkpoint
      const double2* src = ck + (size_t)sg.ckpt * N;
      for (uint32_t k = tid; k < N; k += BT) psi[k] = src[k];
      __syncthreads();
    }

    // ---------------------------------------------------------------- gradients, update
    for (int p = tid; p < I.n_params; p += BT) {
      double g = 0.0;
      for (int j = a.pptr[I.pp_off + p]; j < a.pptr[I.pp_off + p + 1]; ++j)
        g += contrib[a.pops[j]];
      grad[p] = g;
      if (a.n_steps > 0) theta[p] = fma(-lr, g, theta[p]);
    }
    if (tid == 0) {
      if (a.n_steps > 0 && a.etraj) a.etraj[(size_t)step * a.n_inst + idx] = E;
      a.energy[idx] = E;
    }
    __syncthreads();
  }
}

template <int BT>
__global__ void __launch_bounds__(BT, 1) k_batch(BatchArgs a) {
  extern __shared__ double2 sm[];
  __shared__ Smem<BT> S;
  for (;;) {
    if (threadIdx.x == 0) S.item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = S.item;
    __syncthreads();
    if (item >= a.n_inst) break;
    run_instance<BT>(a, a.order[item], sm, S);
  }
}

}  // namespace

size_t batch_smem_bytes(int nmax) { return (size_t)2 * ((size_t)1 << nmax) * sizeof(double2); }

cudaError_t batch_prepare(int nmax, int* grid_out) {
  const size_t smem = batch_smem_bytes(nmax);
  cudaError_t e = cudaFuncSetAttribute(k_batch<kBatchThreads>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<kBatchThreads>,
                                                         kBatchThreads, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid_out = sms * per_sm;
  return cudaSuccess;
}

cudaError_t launch_batch(const BatchArgs& a, int grid, size_t smem, cudaStream_t s) {
  k_batch<kBatchThreads><<<grid, kBatchThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace svqe
