// k_state.cu -- single-state kernels over an HBM-resident complex128 vector (2^n, n <= 31).
//
// Each kernel streams amplitude pairs with coalesced 16-byte loads, four pairs in flight per
// thread, 64-bit indices.  Gate arithmetic follows svqe_internal.cuh (lifting rotations,
// integer sign flips).  Reductions use a fixed grid of kRedBlocks blocks and fixed-order
// sums, so results do not depend on scheduling.
#include "launch.h"
#include "svqe_internal.cuh"

namespace svqe {

namespace {

enum Kind { K_SWAP = 0, K_H = 1, K_ROTY = 2, K_ROTX = 3, K_ROTZ = 4, K_NEG = 5 };

__host__ __device__ inline int kind_of(int type) {
  switch (type) {
    case SV_GATE_X: case SV_GATE_CNOT: return K_SWAP;
    case SV_GATE_H: return K_H;
    case SV_GATE_RY: case SV_GATE_SINGLE_EXC: case SV_GATE_DOUBLE_EXC: return K_ROTY;
    case SV_GATE_RX: return K_ROTX;
    case SV_GATE_RZ: return K_ROTZ;
    case SV_GATE_CZ: return K_NEG;
    default: return K_SWAP;
  }
}

template <int KIND>
__device__ __forceinline__ void apply_kind(const Rot& r, double2& x, double2& y) {
  if (KIND == K_SWAP) {
    const double2 t = x; x = y; y = t;
  } else if (KIND == K_H) {
    pair_apply(SV_GATE_H, r, false, x, y);
  } else if (KIND == K_ROTY) {
    rot_apply(r, x.x, y.x);
    rot_apply(r, x.y, y.y);
  } else if (KIND == K_ROTX) {
    const Rot m = rot_inverse(r);
    rot_apply(m, x.x, y.y);
    rot_apply(r, x.y, y.x);
  } else if (KIND == K_ROTZ) {
    const Rot m = rot_inverse(r);
    rot_apply(m, x.x, x.y);
    rot_apply(r, y.x, y.y);
  }
}

template <int KIND>
__device__ __forceinline__ double grad_kind(const double2& lx, const double2& ly,
                                            const double2& px, const double2& py) {
  if (KIND == K_ROTY) return pair_grad(SV_GATE_RY, lx, ly, px, py);
  if (KIND == K_ROTX) return pair_grad(SV_GATE_RX, lx, ly, px, py);
  if (KIND == K_ROTZ) return pair_grad(SV_GATE_RZ, lx, ly, px, py);
  return 0.0;
}

constexpr int kUnroll = 4;

__global__ void k_init_basis(double2* __restrict__ psi, uint64_t N, uint64_t b) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride)
    psi[i] = make_double2(i == b ? 1.0 : 0.0, 0.0);
}

__global__ void k_prep_coefs(const DOp* __restrict__ ops, int n_ops,
                             const double* __restrict__ theta, Rot* __restrict__ coefs) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n_ops) coefs[g] = make_coef(ops[g], theta).r;
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 4) k_apply(double2* __restrict__ psi, uint64_t npairs,
                                                    DOp op, const Rot* __restrict__ coef,
                                                    int inv) {
  Rot r = *coef;
  if (inv) r = rot_inverse(r);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p0 < npairs;
       p0 += kUnroll * stride) {
    uint64_t ii[kUnroll];
    double2 x[kUnroll], y[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t p = p0 + u * stride;
      ii[u] = insert_zeros(p, op.sb, op.k) | op.lo_or;
      if (p < npairs) {
        x[u] = psi[ii[u]];
        if (KIND != K_NEG) y[u] = psi[ii[u] ^ op.flip];
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t p = p0 + u * stride;
      if (p < npairs) {
        if (KIND == K_NEG) {
          psi[ii[u]] = make_double2(dneg(x[u].x), dneg(x[u].y));
        } else {
          apply_kind<KIND>(r, x[u], y[u]);
          psi[ii[u]] = x[u];
          psi[ii[u] ^ op.flip] = y[u];
        }
      }
    }
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_adjoint(double2* __restrict__ psi,
                                                      double2* __restrict__ lam, uint64_t npairs,
                                                      DOp op, const Rot* __restrict__ coef,
                                                      double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const Rot r = rot_inverse(*coef);
  const bool want = partial != nullptr;
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p0 < npairs;
       p0 += kUnroll * stride) {
    uint64_t ii[kUnroll];
    double2 px[kUnroll], py[kUnroll], lx[kUnroll], ly[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t p = p0 + u * stride;
      ii[u] = insert_zeros(p, op.sb, op.k) | op.lo_or;
      if (p < npairs) {
        px[u] = psi[ii[u]];
        lx[u] = lam[ii[u]];
        if (KIND != K_NEG) {
          py[u] = psi[ii[u] ^ op.flip];
          ly[u] = lam[ii[u] ^ op.flip];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t p = p0 + u * stride;
      if (p < npairs) {
        if (KIND == K_NEG) {
          psi[ii[u]] = make_double2(dneg(px[u].x), dneg(px[u].y));
          lam[ii[u]] = make_double2(dneg(lx[u].x), dneg(lx[u].y));
        } else {
          if (want) acc += grad_kind<KIND>(lx[u], ly[u], px[u], py[u]);
          apply_kind<KIND>(r, px[u], py[u]);
          apply_kind<KIND>(r, lx[u], ly[u]);
          psi[ii[u]] = px[u];
          psi[ii[u] ^ op.flip] = py[u];
          lam[ii[u]] = lx[u];
          lam[ii[u] ^ op.flip] = ly[u];
        }
      }
    }
  }
  if (want) {
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

// lambda[k] = sum_g f_g(k) psi[k ^ x_g];  partial[b] = block share of Re<psi|lambda>.
__global__ void __launch_bounds__(kThreads) k_hpsi(const double2* __restrict__ psi,
                                                   double2* __restrict__ lam, uint64_t N,
                                                   const DGroup* __restrict__ groups,
                                                   int n_groups,
                                                   const double2* __restrict__ tables,
                                                   double* __restrict__ partial) {
  __shared__ DGroup sg[128];
  __shared__ double red[kThreads / 32];
  double e = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tile = kUnroll * stride;
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < N; base += tile) {
    const uint64_t k0 = base + threadIdx.x;
    double2 acc[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) acc[u] = make_double2(0.0, 0.0);
    for (int g0 = 0; g0 < n_groups; g0 += 128) {
      const int cnt = min(128, n_groups - g0);
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) sg[t] = groups[g0 + t];
      __syncthreads();
      for (int g = 0; g < cnt; ++g) {
        const DGroup G = sg[g];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const uint64_t k = k0 + u * stride;
          if (k < N) {
            const double2 v = psi[k ^ G.x];
            double2 f;
            const int cls = group_value(G, k, tables, f);
            group_madd(cls, f, v, acc[u]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t k = k0 + u * stride;
      if (k < N) {
        const double2 p = psi[k];
        e = fma(p.x, acc[u].x, e);
        e = fma(p.y, acc[u].y, e);
        if (lam) lam[k] = acc[u];
      }
    }
  }
  const double t = block_sum(e, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Energy only: E = <psi|H|psi> (Eq. 2), H the Pauli sum of Eq. 3 grouped by X mask:
// E = sum_g sum_k conj(psi[k]) f_g(k) psi[k ^ x_g].
// A group's operator is Hermitian (its strings carry real coefficients), so f_g(k ^ x_g) is
// the conjugate of f_g(k) and the terms at k and k ^ x_g are complex conjugates of each other:
// the sum runs over one member k of each pair (the top bit of x_g clear) and counts
// 2 Re(conj(psi[k]) f_g(k) psi[k ^ x_g]).  psi is still read once per group, with half the FP64
// work of the full lambda = H psi product: for a one-term group the sign (-1)^popc(zu & k) is
// folded into psi[k ^ x_g] by an integer op and the coefficient applied once per group and
// warp, one DFMA per amplitude.  The diagonal group (x_g = 0) takes k and k + N/2 together, each once.
// Work unit: one warp, a chunk of min(N/2, 32 kEU) consecutive pair indices of one group
// (lane l takes pair indices l, l + 32, ...), so the group record and its class are uniform.
constexpr int kEULog = 2;
constexpr int kEU = 1 << kEULog;

__device__ __forceinline__ double2 sign_flip(const double2& w, uint32_t sm) {
  return make_double2(__hiloint2double(__double2hiint(w.x) ^ sm, __double2loint(w.x)),
                      __hiloint2double(__double2hiint(w.y) ^ sm, __double2loint(w.y)));
}

__global__ void __launch_bounds__(kThreads, 4) k_expval(const double2* __restrict__ psi, int n,
                                                        const DGroup* __restrict__ groups,
                                                        int n_groups,
                                                        const double2* __restrict__ tables,
                                                        double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int lane = threadIdx.x & 31;
  const int h_log = n - 1;  // N/2 pairs per group
  const int c_log = min(h_log, 5 + kEULog);
  const int upg_log = h_log - c_log;  // chunks per group (log2)
  const uint32_t C = 1u << c_log;
  const uint64_t units = (uint64_t)n_groups << upg_log;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t umask = (1ull << upg_log) - 1ull;
  double e = 0.0;
  uint64_t unit = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  while (unit < units) {
    // One run of this warp's chunks of group g: the class dispatch and the coefficient are
    // taken once per run, outside the amplitude loop.
    const int g = (int)(unit >> upg_log);
    const uint64_t gend = min(units, (uint64_t)(g + 1) << upg_log);
    const DGroup G = groups[g];
    // Indices fit in 32 bits (n <= 31).
    const uint32_t xp = G.x ? (uint32_t)G.x : (1u << h_log);  // partner mask
    const uint32_t lo = (1u << (31 - __clz((int)xp))) - 1u;
    double acc = 0.0;
    // body(k, psi[k], psi[k ^ xp]) for every pair of the run; k is pair index c0 + lane + 32 u
    // with a zero bit inserted at the top bit of xp.
    auto sweep = [&](auto body) {
      for (; unit < gend; unit += nwarps) {
        const uint32_t c0 = (uint32_t)((unit & umask) << c_log);
        uint32_t k[kEU];
        double2 v[kEU], w[kEU];
#pragma unroll
        for (int u = 0; u < kEU; ++u) {
          const uint32_t t = c0 + lane + 32 * u;
          k[u] = ((t & ~lo) << 1) | (t & lo);
          if ((uint32_t)(lane + 32 * u) < C) {
            v[u] = psi[k[u]];
            w[u] = psi[k[u] ^ xp];
          } else {
            v[u] = make_double2(0.0, 0.0);
            w[u] = v[u];
          }
        }
#pragma unroll
        for (int u = 0; u < kEU; ++u) body(k[u], v[u], w[u]);
      }
    };
    double scale = 2.0;
    if (G.x == 0) {
      // Diagonal: Re f(k) |psi[k]|^2 for both members of the (k, k + N/2) pair.
      scale = 1.0;
      sweep([&](uint32_t kv, const double2& a, const double2& b) {
        double2 f1, f2;
        group_value(G, kv, tables, f1);
        group_value(G, kv ^ xp, tables, f2);
        acc = fma(f1.x, fma(a.x, a.x, a.y * a.y), acc);
        acc = fma(f2.x, fma(b.x, b.x, b.y * b.y), acc);
      });
    } else if (G.cls == 4) {
      // One term, f(k) = c (-1)^popc(zu & k) with c real: c s (v.x w.x + v.y w.y).
      scale = 2.0 * tables[G.toff].x;
      const uint32_t zu = (uint32_t)G.zu;
      sweep([&](uint32_t kv, const double2& a, const double2& b) {
        const double2 bs = sign_flip(b, (uint32_t)(__popc(kv & zu) & 1) << 31);
        acc = fma(a.x, bs.x, acc);
        acc = fma(a.y, bs.y, acc);
      });
    } else if (G.cls == 5) {
      // One term with c imaginary: Re(i c s conj(v) w) = c s (v.y w.x - v.x w.y).
      scale = 2.0 * tables[G.toff].y;
      const uint32_t zu = (uint32_t)G.zu;
      sweep([&](uint32_t kv, const double2& a, const double2& b) {
        const double2 bs = sign_flip(b, (uint32_t)(__popc(kv & zu) & 1) << 31);
        acc = fma(a.y, bs.x, acc);
        acc = fma(dneg(a.x), bs.y, acc);
      });
    } else {
      // Tabulated f(k): Re(f conj(v) w) = Re f (v.x w.x + v.y w.y) + Im f (v.y w.x - v.x w.y).
      sweep([&](uint32_t kv, const double2& a, const double2& b) {
        double2 f;
        const int cls = group_value(G, kv, tables, f);
        if (cls != 1) acc = fma(f.x, fma(a.x, b.x, a.y * b.y), acc);
        if (cls != 0) acc = fma(f.y, fma(a.y, b.x, dneg(a.x) * b.y), acc);
      });
    }
    e = fma(scale, acc, e);
  }
  const double t = block_sum(e, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_sum(const double* __restrict__ partial, int count, double* __restrict__ out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += partial[i];
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) out[0] = t;
}

// One warp per op: contrib[l] = sum_b partial[l * kRedBlocks + b] (lane-strided, fixed order).
__global__ void k_op_contrib(const DOp* __restrict__ ops, int n_ops,
                             const double* __restrict__ partial, double* __restrict__ contrib) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, l = threadIdx.x & 31;
  if (w >= n_ops) return;
  double v = 0.0;
  if (ops[w].param >= 0)
    for (int b = l; b < kRedBlocks; b += 32) v += partial[(size_t)w * kRedBlocks + b];
  v = warp_sum(v);
  if (l == 0) contrib[w] = v;
}

__global__ void k_param_sum(const DOp* __restrict__ ops, int n_ops,
                            const double* __restrict__ contrib, int n_params,
                            double* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_params) return;
  double g = 0.0;
  for (int l = 0; l < n_ops; ++l)
    if (ops[l].param == p) g += contrib[l];
  grad[p] = g;
}

__global__ void k_gd_update(double* __restrict__ theta, const double* __restrict__ grad, int n,
                            double lr, const double* __restrict__ energy,
                            double* __restrict__ traj) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) theta[p] = fma(-lr, grad[p], theta[p]);
  if (p == 0 && traj) traj[0] = energy[0];
}

inline int grid_for(uint64_t work) {
  const uint64_t per = (uint64_t)kThreads * kUnroll;
  uint64_t g = (work + per - 1) / per;
  if (g < 1) g = 1;
  if (g > (uint64_t)kRedBlocks) g = kRedBlocks;
  return (int)g;
}

}  // namespace

cudaError_t launch_init_basis(double2* psi, int n, uint64_t b, cudaStream_t s) {
  const uint64_t N = 1ull << n;
  k_init_basis<<<grid_for(N), kThreads, 0, s>>>(psi, N, b);
  return cudaGetLastError();
}

cudaError_t launch_prep_coefs(const DOp* ops, int n_ops, const double* theta, Rot* coefs,
                              cudaStream_t s) {
  if (n_ops <= 0) return cudaSuccess;
  k_prep_coefs<<<(n_ops + 127) / 128, 128, 0, s>>>(ops, n_ops, theta, coefs);
  return cudaGetLastError();
}

cudaError_t launch_apply_op(double2* psi, int n, const DOp& op, const Rot* coef, bool inv,
                            cudaStream_t s) {
  const uint64_t npairs = 1ull << (n - op.k);
  const int g = grid_for(npairs);
  switch (kind_of(op.type)) {
    case K_SWAP: k_apply<K_SWAP><<<g, kThreads, 0, s>>>(psi, npairs, op, coef, inv); break;
    case K_H: k_apply<K_H><<<g, kThreads, 0, s>>>(psi, npairs, op, coef, inv); break;
    case K_ROTY: k_apply<K_ROTY><<<g, kThreads, 0, s>>>(psi, npairs, op, coef, inv); break;
    case K_ROTX: k_apply<K_ROTX><<<g, kThreads, 0, s>>>(psi, npairs, op, coef, inv); break;
    case K_ROTZ: k_apply<K_ROTZ><<<g, kThreads, 0, s>>>(psi, npairs, op, coef, inv); break;
    case K_NEG: k_apply<K_NEG><<<g, kThreads, 0, s>>>(psi, npairs, op, coef, inv); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_op(double2* psi, double2* lam, int n, const DOp& op, const Rot* coef,
                              double* partial, cudaStream_t s) {
  const uint64_t npairs = 1ull << (n - op.k);
  const int g = partial ? kRedBlocks : grid_for(npairs);
  switch (kind_of(op.type)) {
    case K_SWAP: k_adjoint<K_SWAP><<<g, kThreads, 0, s>>>(psi, lam, npairs, op, coef, nullptr); break;
    case K_H: k_adjoint<K_H><<<g, kThreads, 0, s>>>(psi, lam, npairs, op, coef, nullptr); break;
    case K_ROTY: k_adjoint<K_ROTY><<<g, kThreads, 0, s>>>(psi, lam, npairs, op, coef, partial); break;
    case K_ROTX: k_adjoint<K_ROTX><<<g, kThreads, 0, s>>>(psi, lam, npairs, op, coef, partial); break;
    case K_ROTZ: k_adjoint<K_ROTZ><<<g, kThreads, 0, s>>>(psi, lam, npairs, op, coef, partial); break;
    case K_NEG: k_adjoint<K_NEG><<<g, kThreads, 0, s>>>(psi, lam, npairs, op, coef, nullptr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_hpsi(const double2* psi, double2* lam, int n, const DGroup* groups,
                        int n_groups, const double2* tables, double* partial, cudaStream_t s) {
  const uint64_t N = 1ull << n;
  if (!lam && partial)
    k_expval<<<kRedBlocks, kThreads, 0, s>>>(psi, n, groups, n_groups, tables, partial);
  else
    k_hpsi<<<kRedBlocks, kThreads, 0, s>>>(psi, lam, N, groups, n_groups, tables, partial);
  return cudaGetLastError();
}

cudaError_t launch_sum(const double* partial, int count, double* out, cudaStream_t s) {
  k_sum<<<1, 1024, 0, s>>>(partial, count, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_grads(const DOp* ops, int n_ops, const double* partial, int n_params,
                                double* contrib, double* grad, cudaStream_t s) {
  if (n_ops > 0) {
    const int warps_per_block = 8;
    k_op_contrib<<<(n_ops + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0,
                   s>>>(ops, n_ops, partial, contrib);
  }
  if (n_params > 0)
    k_param_sum<<<(n_params + 127) / 128, 128, 0, s>>>(ops, n_ops, contrib, n_params, grad);
  return cudaGetLastError();
}

cudaError_t launch_gd_update(double* theta, const double* grad, int n, double lr,
                             const double* energy, double* traj, cudaStream_t s) {
  k_gd_update<<<(n + 127) / 128 > 0 ? (n + 127) / 128 : 1, 128, 0, s>>>(theta, grad, n, lr,
                                                                         energy, traj);
  return cudaGetLastError();
}

}  // namespace svqe
