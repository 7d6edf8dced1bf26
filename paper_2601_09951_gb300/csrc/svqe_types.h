// svqe_types.h -- record layouts shared by host lowering and device kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/svqe.h"

namespace svqe {

// ------------------------------------------------------------------------------ op records
// A compiled gate.  Its amplitude "pairs" are enumerated by inserting zero bits at the
// sorted positions sb[0..k) into a counter p in [0, 2^(n-k)), OR-ing `lo_or`, and pairing the
// result i with j = i ^ flip (flip = 0: a single amplitude, e.g. CZ).
struct DOp {
  int32_t type;    // SV_GATE_*
  int32_t param;   // theta index or -1
  int32_t k;       // number of inserted zero bits
  int32_t bit0;    // basis-index bit of the first wire (1-qubit gates)
  uint8_t sb[4];   // sorted bit positions of the wires
  int32_t flags;   // kOpCS: the batched kernel wants (cos, sin) for this op (see below)
  uint64_t lo_or;  // bits set in the first amplitude of each pair
  uint64_t flip;   // XOR mask from the first to the second amplitude
  double fixed;    // angle when param < 0
};
static_assert(sizeof(DOp) == 48, "DOp layout");
// The batched kernel needs (cos phi, sin phi), phi = theta/2, rather than the lifting form for
// the RZ gates of a diagonal segment (applied as one phase) and for the RY gates of a
// product-state layer: for an op with this flag its coefficient slot holds
// Rot{a = cos phi, b = sin phi, k = 0}.
constexpr int32_t kOpCS = 1;

// Lifting form of the rotation R(phi) = [[c, -s], [s, c]] (phi = theta/2):
// R(phi) = L(a) S(b) L(a) R(k pi/2), a = -tan(r/2), b = sin(r), r = phi - k pi/2 in
// [-pi/4, pi/4].
struct Rot {
  double a, b;
  int32_t k;
  int32_t pad;
};
static_assert(sizeof(Rot) == 24, "Rot layout");

// An X-mask group of Pauli terms, (H psi)[k] += f(k) psi[k ^ x]:
//   cls 0/1/2: f(k) = table[toff + pext(k, zu)], a real / imaginary / complex table over the
//              kz bits of the union zu of the group's z masks;
//   cls 4/5:   a single term, f(k) = table[toff] * (-1)^{popc(zu & k)} with zu its z mask and
//              table[toff] real (4) or imaginary (5).
struct DGroup {
  uint64_t x;
  uint64_t zu;
  int32_t kz;
  int32_t cls;
  int64_t toff;  // offset of the table (double2 entries)
};
static_assert(sizeof(DGroup) == 32, "DGroup layout");

// A segment of a circuit's op list, as the batched kernel executes it.
//   SEG_GATES : ops applied one at a time; the adjoint sweep un-applies each op to psi and
//               lambda and takes its gradient in between.
//   SEG_RLAYER: RY (or RX) gates on distinct qubits.  They commute, so every gradient of the
//               layer is taken from (psi, lambda) at the layer's end; the sweep then
//               un-applies the layer to lambda only and reloads psi from a checkpoint saved
//               on the forward pass.  With split = 1 (the first segment, RY gates only) the
//               layer acts on the reference basis state, so its output is a product state,
//               written directly from two half tables; the sweep takes its gradients and stops
//               there (no un-apply, no checkpoint).
//   SEG_DIAG  : RZ and CZ gates (diagonal, mutually commuting), applied as one phase
//               e^{-i sum_q phi_q s_q(k)} (+-1 for CZ) per amplitude from two half tables;
//               gradients from w_k = Im(conj(lambda_k) psi_k); psi reloaded from a checkpoint.
//   SEG_PERM  : CNOT and X gates: their product is one permutation of basis indices, applied
//               as a single gather into the other buffer (the psi and lambda buffers then swap
//               roles); the sweep gathers lambda back and reloads psi from a checkpoint.
//   SEG_DIAGPERM: a SEG_DIAG run (its first `split` ops) directly followed by a SEG_PERM run
//               (the pattern of every hardware-efficient layer), done in one pass each way: the
//               forward pass writes the checkpoint, applies the phase and scatters to the
//               permuted index; the sweep gathers lambda and psi through the permutation,
//               takes the diagonal gradients, un-applies the phase to lambda and reloads psi
//               from the one checkpoint.
enum { SEG_GATES = 0, SEG_RLAYER = 1, SEG_DIAG = 2, SEG_PERM = 3, SEG_DIAGPERM = 4 };
struct Seg {
  int16_t kind;
  int16_t split;  // SEG_DIAGPERM: ops of the diagonal part; SEG_RLAYER: 1 = product layer
  int32_t first;  // first op
  int32_t count;  // number of ops
  int32_t ckpt;   // checkpoint slot of psi before the segment, or -1
};
static_assert(sizeof(Seg) == 16, "Seg layout");

// Gates of one permutation segment of the batched kernel.
constexpr int kMaxPerm = 32;
// Gradient slots per fused pass (and RZ gates per diagonal item).
constexpr int kMaxSlotsDev = 16;
// Lowest contiguous bits every fused tile includes (runs of 2^kMinLowBits amplitudes, 256 B),
// so that tiles of an HBM-resident state move in long DRAM bursts.  A state small enough for
// psi and lambda to stay in L2 (n <= kL2Qubits) needs only 32-byte sectors: its tiles include
// kMinLowBitsL2 low bits, which leaves more of the tile's bits for gate wires (fewer passes).
constexpr int kMinLowBits = 4;
constexpr int kMinLowBitsL2 = 2;
constexpr int kL2Qubits = 21;

// A fused pass of the single-state path: every item of the pass acts inside one "tile" of
// 2^m amplitudes (the basis-index bits in tile_mask, which always include the c lowest bits,
// so a tile is 2^(m-c) contiguous runs of 2^c amplitudes); the other bits (outer_mask) number
// the 2^(n-m) tiles.  A pass loads a tile into shared memory, applies its items in order and
// writes it back, so a whole run of gates costs one read and one write of the state.
struct FPass {
  uint64_t tile_mask;
  uint64_t outer_mask;
  int32_t m, c;
  int32_t first_item, n_items;
  int32_t n_slots;  // gradient slots used by the pass's parameterised items
  int32_t pad[3];
};
static_assert(sizeof(FPass) == 48, "FPass layout");

// One item of a fused pass: an op in tile-local bit coordinates (kind 0), or a run of RZ gates
// applied as one diagonal phase (kind 1: global ops [op, op + count); their bits may lie
// inside or outside the tile).  slot: first gradient slot of the item, or -1.
struct FItem {
  int32_t kind;
  int32_t op;
  int32_t count;
  int32_t slot;
  DOp local;
};
static_assert(sizeof(FItem) == 64, "FItem layout");

__host__ __device__ __forceinline__ bool is_param_type(int t) {
  return t == SV_GATE_RX || t == SV_GATE_RY || t == SV_GATE_RZ || t == SV_GATE_SINGLE_EXC ||
         t == SV_GATE_DOUBLE_EXC;
}

}  // namespace svqe
