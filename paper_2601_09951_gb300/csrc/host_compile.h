// host_compile.h -- host-side validation and lowering of circuits and Pauli sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/svqe.h"
#include "svqe_types.h"

namespace svqe {

struct DOp;
struct DGroup;
struct Seg;
struct FPass;
struct FItem;

// Thread-local error message (sv_last_error).
void set_error(const char* fmt, ...);
void clear_error();
const char* last_error();

// A circuit lowered to device op records (see DOp).  Gates are validated: known type, wires
// in [0, n), distinct wires, parameter index in [-1, n_params).
struct HostCircuit {
  int n = 0;
  int n_params = 0;
  std::vector<DOp> ops;
};
sv_status lower_circuit(const sv_circuit* c, int expect_n, HostCircuit& out);

// Split a lowered op list into segments for the batched kernel (see Seg).  A run of RZ/CZ
// becomes SEG_DIAG when it holds at least `min_diag_rz` RZ gates (and at most kMaxLayer RZ and
// kMaxLayer CZ gates); a run of RY (or RX) gates on distinct qubits becomes SEG_RLAYER when it
// holds at least `min_layer` gates (and at most kMaxLayer); a run of two to kMaxPerm CNOT/X
// gates becomes SEG_PERM; a SEG_DIAG directly followed by a SEG_PERM becomes one
// SEG_DIAGPERM; everything else is SEG_GATES.  A first SEG_RLAYER of RY gates is marked as a
// product layer (split = 1, no checkpoint).  The RZ gates of diagonal segments and the gates
// of a product layer get the kOpCS flag (their coefficient is (cos, sin) instead of the
// lifting form).  Returns the number of checkpoints used.
constexpr int kMaxLayer = 16;
int segment_ops(std::vector<DOp>& ops, int min_layer, int min_diag_rz,
                std::vector<Seg>& segs);

// Runs of RY (or RX) gates on distinct qubits with at least min_len gates, as (first, count):
// the commuting layers whose gradients the single-state path can take at the layer's end.
std::vector<std::pair<int, int>> commuting_layers(const std::vector<DOp>& ops, int min_len);

// Plan the fused passes of an n-qubit circuit with tiles of m bits (see FPass): ops are taken
// greedily in order into the current pass while the pass's pair bits fit the tile; an op may
// move ahead of ops skipped for this pass only if it shares no qubit with them (so it
// commutes with them).  Runs of >= 3 consecutive RZ gates become one diagonal item (at most
// one per pass, at most kMaxSlots RZ gates).  A pass holds at most kMaxSlots gradient slots.
// Every tile includes the kMinLowBits lowest bits (kMinLowBitsL2 for n <= kL2Qubits).
constexpr int kMaxSlots = kMaxSlotsDev;
struct HostPlan {
  std::vector<FPass> passes;
  std::vector<FItem> items;
};
void plan_passes(const std::vector<DOp>& ops, int n, int m, HostPlan& plan);

// A Pauli sum grouped by X mask.  Every group's f(k) = sum_t c_t (-i)^{popc(x&z_t)}
// (-1)^{popc(z_t&k)} is tabulated over the kz bits of the union zu of its z masks, so that
// (H psi)[k] = sum_g f_g(k) psi[k ^ x_g].  A group whose union would exceed kmax bits is split
// into several groups with the same x.  The x = 0 group, if any, comes first.
struct HostHam {
  int n = 0;
  int n_terms = 0;
  double l1 = 0.0;  // sum |c_t|
  std::vector<DGroup> groups;
  std::vector<double2> tables;
};
sv_status lower_ham(const sv_paulisum* h, int expect_n, int kmax, HostHam& out);

}  // namespace svqe
