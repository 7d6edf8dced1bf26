// api_internal.h -- library-internal entry points shared by api.cu and serve.cu.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/svqe.h"
#include "host_compile.h"
#include "launch.h"

namespace svqe {

// Stage a lowered circuit on a context (ops, coefficient and gradient buffers, fused plan).
// Upload a lowered circuit and plan its fused passes.  may_tune: with autotuning on
// (sv_set_autotune), a circuit structure not seen before has its tile size measured first
// (the forward pass is run on the context's psi, so only callers that re-initialise psi
// afterwards pass true).
sv_status stage_circuit(sv_ctx* c, const HostCircuit& hc, bool may_tune = false);
// psi = |ref>, forward, lambda = H psi, adjoint sweep; stream-ordered.
sv_status adjoint_core(sv_ctx* c, const HostCircuit& hc, const sv_ham* H,
                       const double* theta_dev, double* energy_dev, double* grad_dev);
// n_steps of gradient descent, enqueued on the context's stream without synchronising:
// theta_in is read before the call returns; theta_out (n_params) and energy_out (n_steps)
// are written when the stream reaches them (pinned host memory for real asynchrony).
sv_status vqe_enqueue(sv_ctx* c, const HostCircuit& hc, const sv_ham* H, const double* theta_in,
                      double lr, int32_t n_steps, double* theta_out, double* energy_out);
cudaStream_t ctx_stream(sv_ctx* c);
// Replace the Pauli sum held by H (lowered for c's register), reusing H's device buffers when
// they are large enough, so that a pooled context takes a new request without allocating.
sv_status ham_reload(sv_ctx* c, sv_ham* H, const sv_paulisum* h);
// True once a CUDA error has made the context unusable.
bool ctx_sticky(const sv_ctx* c);

// Layout of the batched kernel for the instances of one qubit count: the team class of their
// work items (kClassWarps) and the segment widths their circuits are cut with (segment_ops: a
// run of RY/RX gates on distinct qubits becomes a commuting-layer segment when it has at least
// min_layer gates, a run of RZ/CZ a diagonal segment when it has at least min_diag_rz RZ
// gates; shorter runs are applied gate by gate).
struct BLayout {
  int cls;
  int min_layer;
  int min_diag_rz;
};
// The fixed rule: the smallest team that holds the instance, widths 2 and 3.
BLayout default_layout(int n);

// Batched-kernel helpers: team class of an n-qubit instance under the fixed rule, teams per CTA
// of that class, work items from per-instance costs (cls_of_n: team class per qubit count, or
// nullptr for the fixed rule), and the FP64 flop count of one instance.
int batch_class(int n);
int class_teams(int n);
std::vector<BItem> batch_items(const std::vector<BInst>& bi, const std::vector<double>& cost,
                               const int* cls_of_n = nullptr);
double batch_instance_flops(const HostCircuit& hc, const HostHam& hh,
                            const std::vector<Seg>& segs);

}  // namespace svqe
