// launch.h -- host-callable launchers of the single-state kernels (k_state.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "svqe_types.h"

namespace svqe {

// Fixed grid for reductions: partial arrays hold at most kRedBlocks values per launch.
constexpr int kRedBlocks = 1216;  // 152 SMs x 8
constexpr int kThreads = 256;

cudaError_t launch_init_basis(double2* psi, int n, uint64_t b, cudaStream_t s);
cudaError_t launch_prep_coefs(const DOp* ops, int n_ops, const double* theta, Rot* coefs,
                              cudaStream_t s);
// Apply (inv = false) or un-apply one op on psi; coef points at the op's Rot.
cudaError_t launch_apply_op(double2* psi, int n, const DOp& op, const Rot* coef, bool inv,
                            cudaStream_t s);
// Adjoint step for one op: if the op is parameterised, partial[b] (b < kRedBlocks) receives
// block b's share of 2 Im<lambda|G|psi>; then psi and lambda are un-applied.
cudaError_t launch_adjoint_op(double2* psi, double2* lam, int n, const DOp& op, const Rot* coef,
                              double* partial, cudaStream_t s);
// lambda = H psi (if lam != nullptr) and partial[b] = block b's share of Re<psi|H psi>.
cudaError_t launch_hpsi(const double2* psi, double2* lam, int n, const DGroup* groups,
                        int n_groups, const double2* tables, double* partial, cudaStream_t s);
// out[0] = sum of partial[0..count) in a fixed order.
cudaError_t launch_sum(const double* partial, int count, double* out, cudaStream_t s);
// grad[p] = sum over ops l with param p (in op order) of sum_b partial[l * kRedBlocks + b].
cudaError_t launch_reduce_grads(const DOp* ops, int n_ops, const double* partial, int n_params,
                                double* contrib, double* grad, cudaStream_t s);
// theta -= lr * grad (n entries); optionally records energy[0] into traj[step].
cudaError_t launch_gd_update(double* theta, const double* grad, int n, double lr,
                             const double* energy, double* traj, cudaStream_t s);

}  // namespace svqe

namespace svqe {

// Fused passes of the single-state path (k_fused.cu).  Tiles of fused_tile_bits() bits (all
// of the state when it is smaller); used for registers of at least kFusedMinQubits qubits.
// Whole-state diagonal + permutation segments (k_dp.cu, blocks of 2048 amplitudes) need at
// least kDpMinQubits.
constexpr int kFusedMinQubits = 1;
constexpr int kDpMinQubits = 14;
int fused_tile_bits();
cudaError_t fused_prepare();
cudaError_t launch_fpass(double2* psi, const FPass& P, const FItem* items, const DOp* gops,
                         const Rot* coef, const double* theta, cudaStream_t s);
// The pass's items inverted and in reverse order, on v (un-applying the pass).
cudaError_t launch_fpass_inv(double2* v, const FPass& P, const FItem* items, const DOp* gops,
                             const Rot* coef, const double* theta, cudaStream_t s);
// Whole-state diagonal + permutation segment of the single-state path (k_dp.cu): a run of
// RZ/CZ gates followed by a run of CNOT/X gates, applied in one out-of-place streaming pass
// for n >= 14.  perm: the permutation P of the CNOT/X run (gates in order) as three
// 2048-entry tables over index bits [0, 11), [11, 22), [22, 31) (the first including P(0));
// phase tables (written by launch_dp_setup from theta): e^{-i sum phi s(k)} of
// the RZ gates over the 11 low bits, and over block-index bits [0, 10) and [10, 20).
constexpr int kDpMaxRz = 32;
constexpr int kDpMaxCz = 16;
struct DpArgs {
  uint64_t N;
  int n;
  const uint32_t* perm;
  const double2* phase_lo;
  const double2* phase_b1;
  const double2* phase_b2;
  double2* phase_lo_w;
  double2* phase_b1_w;
  double2* phase_b2_w;
  int n_cz;
  uint32_t cz_mask[kDpMaxCz];
  int n_rz;                  // parameterised RZ ops: gradient targets
  int rz_op[kDpMaxRz];
  int rz_bit[kDpMaxRz];
  int n_rz_all;              // every RZ op of the diagonal part: phase factors
  int rz_all[kDpMaxRz];
  // Block pairing of the gather/scatter.  The amplitude P(k) ^ 1, which shares P(k)'s 32-byte
  // sector, is P(k ^ delta) with delta = M^-1 e_0 (M the linear part of P); pair is the block
  // part delta >> 11 and pair_hi its highest set bit.  With pair > 1 the kernels visit block
  // B(t) for t = 0, 1, ..., where B(t) and B(t ^ 1) differ by pair, so adjacent CTAs read (or
  // write) the two halves of the same sectors in the same round.
  uint32_t pair;
  int pair_hi;
};
constexpr size_t kDpTableWords = 3 * 2048;     // uint32 per permutation
constexpr size_t kDpPhaseEntries = 2048 + 2048;  // double2 per segment (low + two block tables)
cudaError_t dp_prepare();
cudaError_t launch_dp_setup(const DpArgs& a, const DOp* ops, const double* theta, cudaStream_t s);
// out[P(k)] = phase(k) in[k]
cudaError_t launch_dp_fwd(const double2* in, double2* out, const DpArgs& a, cudaStream_t s);
// out[k] = conj(phase(k)) in[P(k)]
cudaError_t launch_dp_bwd_psi(const double2* in, double2* out, const DpArgs& a, cudaStream_t s);
// out[k] = conj(phase(k)) lam[P(k)]; RZ gradient shares from w_k = Im(conj(out[k]) psi_b[k])
// into partial[op * kRedBlocks + block]
cudaError_t launch_dp_bwd_lam(const double2* lam, const double2* psi_b, double2* out,
                              const DpArgs& a, double* partial, cudaStream_t s);

// Gradient shares only (psi and lambda unchanged) of a pass whose items are single ops:
// partial[op * kRedBlocks + b] as for launch_bpass.
cudaError_t launch_gpass(const double2* psi, const double2* lam, const FPass& P,
                         const FItem* items, const DOp* gops, double* partial, cudaStream_t s);
// Backward pass: partial[op * kRedBlocks + b] receives block b's gradient share of every
// parameterised op of the pass, for the min(tiles, kRedBlocks) blocks launched; the caller
// zeroes the partials beforehand.
cudaError_t launch_bpass(double2* psi, double2* lam, const FPass& P, const FItem* items,
                         const DOp* gops, const Rot* coef, const double* theta, double* partial,
                         cudaStream_t s);

// One instance of a compiled batch (device record).  steps, lr and etraj_off are used when
// BatchArgs::n_steps < 0 (per-instance step counts, as the serving loop runs them).
struct BInst {
  int32_t n, n_ops, n_groups, n_params, n_segs, n_ckpt;
  int32_t steps;
  int32_t tab_n;  // the instance's group tables: tab_n double2 entries from tab_off
  uint64_t ref;
  int64_t op_off, grp_off, theta_off, seg_off, pp_off, etraj_off;
  int64_t coef_off, contrib_off;  // scratch offsets (Rot / double units)
  int64_t grad_off;               // gradient offset (double units)
  double lr;
  int64_t tab_off;
};
static_assert(sizeof(BInst) == 128, "BInst layout");

// A work item of the batched kernel: the instances of one team class (see kClassWarps), one
// per team; unused entries of inst are -1.
struct BItem {
  int32_t cls;
  int32_t inst[8];
};
static_assert(sizeof(BItem) == 36, "BItem layout");
// Team classes of the batched kernel (8 warps per CTA): warps per team and the largest
// instance each class runs, so that every thread holds at most 16 of the 2^n amplitudes.
//   class 0: one team of 8 warps, n = 12;   class 1: two teams of 4 warps, n = 11;
//   class 2: eight teams of 1 warp, n <= 9; class 3: four teams of 2 warps, n = 10.
constexpr int kNumClasses = 4;
constexpr int kClassWarps[kNumClasses] = {8, 4, 1, 2};
constexpr int kClassQubits[kNumClasses] = {12, 11, 9, 10};

struct BatchArgs {
  const BInst* inst;
  int n_inst;
  const BItem* items;      // most expensive first
  int n_items;
  const DOp* ops;
  const DGroup* groups;
  const double2* tables;
  const Seg* segs;
  const int32_t* pptr;     // per instance n_params+1 offsets into pops (absolute)
  const int32_t* pops;     // op indices (relative to the instance) using each parameter
  double* theta;           // concatenated parameters (updated in place when n_steps != 0)
  double* energy;          // [n_inst]
  double* grad;            // concatenated gradients
  Rot* coef;               // scratch, one per op
  double* contrib;         // scratch, one per op
  double2* ckpt;           // scratch, ckpt_slot amplitudes per CTA, split evenly among teams
                           // (team_ckpt_amps per instance)
  int64_t ckpt_slot;
  int64_t smem_amps;       // dynamic shared memory per CTA, in amplitudes
  int* counter;            // work-queue head, zeroed before each launch
  int n_steps;             // 0: one evaluation; > 0: that many updates; < 0: BInst::steps
  double lr;               // step when lr_inst == nullptr (n_steps > 0)
  const double* lr_inst;   // per-instance steps, or nullptr
  double* etraj;           // energies before each update ([n_steps x n_inst], or per
                           // instance at BInst::etraj_off when n_steps < 0), or nullptr
  // Optimizer of the update step: 0 gradient descent; 1 Adam with first/second moments
  // adam_m/adam_v (indexed like grad) and t0 updates already taken.
  int opt;
  double* adam_m;
  double* adam_v;
  int adam_t0;
  double beta1, beta2, eps;
};

// A team's checkpoint scratch for an instance: n_ckpt states of 2^n amplitudes, then one block
// of kDpAuxAmps amplitudes per checkpoint slot, where a diagonal + permutation segment keeps
// the tables its forward pass built (phases, permutation, RZ slots) for the sweep to reload.
constexpr int kDpAuxAmps = 176;
inline int64_t team_ckpt_amps(int n_ckpt, int n) {
  return (int64_t)n_ckpt * ((int64_t(1) << n) + kDpAuxAmps);
}

// Threads per CTA of the batched kernel and its dynamic shared memory for nmax qubits.
constexpr int kBatchThreads = 256;
constexpr int64_t kBatchSmemAmps = 2 * 4096;  // psi + lambda of one 12-qubit instance
size_t batch_smem_bytes(int nmax);
cudaError_t batch_prepare(int nmax, int* grid_out);
cudaError_t launch_batch(const BatchArgs& a, int grid, size_t smem, cudaStream_t s);

}  // namespace svqe
