// k_batch.cu -- the persistent batched kernel: many small independent instances (Sec. 4.1,
// Eq. 7: every bond length / parameter set is its own problem) in one launch.
//
// One CTA runs one instance at a time, taken from a cost-sorted queue with an atomic counter
// (largest first, so the tail is made of cheap instances).  The instance's psi and lambda
// (2 x 2^n x 16 bytes, n <= 12) live in shared memory for the whole forward pass, the
// lambda = H psi pass and the adjoint sweep, so HBM carries only ops, Hamiltonian tables,
// parameters and results.  Every sum runs in a fixed order that does not depend on which CTA
// or SM ran the instance, so an instance's result is bit-identical alone or in any batch.
#include "launch.h"
#include "svqe_internal.cuh"

namespace svqe {

namespace {

template <int BT>
__device__ __forceinline__ double block_sum_bt(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < BT / 32) ? red[l] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0; caller syncs before red is reused
}

template <int BT>
__device__ void run_instance(const BatchArgs& a, int idx, double2* sm, double* red) {
  const BInst I = a.inst[idx];
  const int n = I.n;
  const uint32_t N = 1u << n;
  double2* psi = sm;
  double2* lam = sm + N;
  const DOp* ops = a.ops + I.op_off;
  const DGroup* groups = a.groups + I.grp_off;
  Rot* coef = a.coef + I.op_off;
  double* contrib = a.contrib + I.op_off;
  double* theta = a.theta + I.theta_off;
  double* grad = a.grad + I.theta_off;
  const int tid = threadIdx.x;
  const int steps = a.n_steps > 0 ? a.n_steps : 1;
  const double lr = a.lr_inst ? a.lr_inst[idx] : a.lr;

  for (int step = 0; step < steps; ++step) {
    for (int g = tid; g < I.n_ops; g += BT) coef[g] = make_coef(ops[g], theta).r;
    for (uint32_t k = tid; k < N; k += BT)
      psi[k] = make_double2(k == (uint32_t)I.ref ? 1.0 : 0.0, 0.0);
    __syncthreads();

    // Forward: psi <- U_l psi for l = 0 .. n_ops-1.
    for (int l = 0; l < I.n_ops; ++l) {
      const DOp op = ops[l];
      const Rot r = coef[l];
      const uint32_t np = N >> op.k;
      for (uint32_t p = tid; p < np; p += BT) {
        const uint32_t i = (uint32_t)insert_zeros(p, op.sb, op.k) | (uint32_t)op.lo_or;
        if (op.type == SV_GATE_CZ) {
          psi[i] = make_double2(dneg(psi[i].x), dneg(psi[i].y));
        } else {
          const uint32_t j = i ^ (uint32_t)op.flip;
          double2 x = psi[i], y = psi[j];
          pair_apply(op.type, r, false, x, y);
          psi[i] = x;
          psi[j] = y;
        }
      }
      __syncthreads();
    }

    // lambda = H psi; E = Re<psi|lambda>.
    double e = 0.0;
    for (uint32_t k = tid; k < N; k += BT) {
      double2 acc = make_double2(0.0, 0.0);
      for (int g = 0; g < I.n_groups; ++g) {
        const DGroup G = groups[g];
        const double2 v = psi[k ^ (uint32_t)G.x];
        const double2 f = a.tables[G.toff + pext64(k, G.zu)];
        group_madd(G.cls, f, v, acc);
      }
      lam[k] = acc;
      const double2 p = psi[k];
      e = fma(p.x, acc.x, e);
      e = fma(p.y, acc.y, e);
    }
    const double E = block_sum_bt<BT>(e, red);
    __syncthreads();

    // Adjoint sweep: l = n_ops-1 .. 0.
    for (int l = I.n_ops - 1; l >= 0; --l) {
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
          if (pg) acc += pair_grad(op.type, lx, ly, px, py);
          pair_apply(op.type, r, true, px, py);
          pair_apply(op.type, r, true, lx, ly);
          psi[i] = px;
          psi[j] = py;
          lam[i] = lx;
          lam[j] = ly;
        }
      }
      if (pg) {
        const double t = block_sum_bt<BT>(acc, red);
        if (tid == 0) contrib[l] = t;
      }
      __syncthreads();
    }

    // Gradient per parameter: contributions summed in op order.
    for (int p = tid; p < I.n_params; p += BT) {
      double g = 0.0;
      for (int l = 0; l < I.n_ops; ++l)
        if (ops[l].param == p) g += contrib[l];
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
__global__ void __launch_bounds__(BT) k_batch(BatchArgs a) {
  extern __shared__ double2 sm[];
  __shared__ double red[BT / 32];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= a.n_inst) break;
    run_instance<BT>(a, a.order[item], sm, red);
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
