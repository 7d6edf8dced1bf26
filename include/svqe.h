/*
 * svqe.h -- C ABI of libsvqe.so, the GB300 (sm_103a) state-vector VQE hot path.
 *
 * The paper (Malarchick & Steed, "Parallelizing the Variational Quantum Eigensolver", 2026)
 * poses the problem as: for each Hamiltonian H(d) (Sec. 2.2), prepare |psi(theta)> =
 * U(theta)|HF> (Sec. 3.3, Eq. 4-5), evaluate E(theta) = <psi|H|psi> (Sec. 3.1, Eq. 2) and
 * its gradient, and update theta (Algorithm 1; Sec. 3.4).  This header exposes exactly those
 * steps over complex128 amplitudes on one GPU.
 *
 * Conventions shared by every call
 *   - Amplitudes are complex128, stored interleaved (re, im) as 16-byte pairs; a state of
 *     n qubits has 2^n amplitudes (Table 3: 2^n x 16 bytes).
 *   - Qubit q is bit (n-1-q) of a basis index (qubit 0 is the most significant bit), so the
 *     Hartree-Fock state |1100> of Eq. 4 has basis index 12.
 *   - A Pauli string is a pair of masks over basis-index bits: x has the bits whose factor is
 *     X or Y, z the bits whose factor is Z or Y; the string is i^{popc(x&z)} X^x Z^z
 *     (Y = iXZ).  Coefficients are real (Sec. 3.2, Eq. 3 after Jordan-Wigner).
 *   - Gates: RX/RY/RZ(t) = exp(-i t/2 X/Y/Z); CNOT(control, target); CZ; X; H;
 *     SingleExcitation(t) on wires (a, b) rotates span{|01>, |10>} by t/2 and
 *     DoubleExcitation(t) on (a, b, c, d) rotates span{|0011>, |1100>} by t/2:
 *       |lo> -> cos(t/2)|lo> + sin(t/2)|hi>,  |hi> -> cos(t/2)|hi> - sin(t/2)|lo>
 *     (Eq. 5 read as exp(-t/2 (A - A^dag)), A = a0^dag a1^dag a2 a3 under Jordan-Wigner).
 *
 * Ownership: the caller owns every array it passes; the library copies what it keeps.
 * Handles (sv_ctx, sv_ham, sv_batch, sv_server) belong to the library until freed.
 * Pointers named *_dev are device pointers; all other array pointers are host pointers.
 *
 * Streams: every call is ordered on the stream of its context or batch.  Calls that return
 * host values (energies, gradients, states) synchronise that stream before returning.
 *
 * Errors: every call returns sv_status and never aborts the process.  SV_EINVAL reports a
 * malformed argument (bad wire, duplicate wire, qubit count outside [1, 31], mask bit >= n,
 * parameter index out of range, NULL pointer).  SV_ECUDA reports a CUDA failure; the handle
 * that saw it is then unusable ("sticky") and must be destroyed.  sv_last_error() gives the
 * calling thread's most recent message.
 *
 * Threading: a handle may be used by one host thread at a time.  Different handles may be
 * used concurrently from different threads.
 */
#ifndef SVQE_H
#define SVQE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SV_OK = 0,
  SV_EINVAL = 1,        /* malformed argument */
  SV_ENOMEM = 2,        /* device or host allocation failed, or an HBM budget is exceeded */
  SV_ECUDA = 3,         /* a CUDA call failed; the handle is now unusable */
  SV_ETIMEOUT = 4,      /* a bounded wait ran out */
  SV_EUNSUPPORTED = 5,  /* valid request the library does not implement */
  SV_EBUSY = 6          /* result not ready yet (serving poll) */
} sv_status;

/* Gate codes (the `type` field of sv_gate). */
enum {
  SV_GATE_X = 0,
  SV_GATE_H = 1,
  SV_GATE_RX = 2,
  SV_GATE_RY = 3,
  SV_GATE_RZ = 4,
  SV_GATE_CNOT = 5,
  SV_GATE_SINGLE_EXC = 6,
  SV_GATE_DOUBLE_EXC = 7,
  SV_GATE_CZ = 8
};

/* One gate record, 32 bytes.  wires: the first 1, 2 or 4 entries are used (others ignored);
 * param: index into theta, or -1 to use fixed_angle.  X, H, CNOT and CZ ignore the angle. */
typedef struct {
  int32_t type;
  int32_t wires[4];
  int32_t param;
  double fixed_angle;
} sv_gate;

/* A circuit U = U_{n_gates-1} ... U_0 (gates applied in array order) with n_params angles. */
typedef struct {
  int32_t n_qubits;
  int32_t n_gates;
  int32_t n_params;
  const sv_gate* gates;
} sv_circuit;

/* H = sum_t coeff[t] * P(x_mask[t], z_mask[t])  (Sec. 3.2). */
typedef struct {
  int32_t n_qubits;
  int32_t n_terms;
  const uint64_t* x_mask;
  const uint64_t* z_mask;
  const double* coeff;
} sv_paulisum;

typedef struct sv_ctx sv_ctx;        /* one n-qubit state: psi and lambda buffers + stream */
typedef struct sv_ham sv_ham;        /* device-resident grouped Pauli sum                  */
typedef struct sv_batch sv_batch;    /* many small instances, run by one persistent kernel */
typedef struct sv_server sv_server;  /* continuous-batching request loop                   */

/* ---------------------------------------------------------------- library information */

/* Human-readable name of a status code (static string). */
const char* sv_status_str(sv_status s);
/* The calling thread's most recent error message ("" if none); valid until its next call. */
const char* sv_last_error(void);
/* ABI version, currently 1. */
int32_t sv_abi_version(void);
/* Bytes of one n-qubit complex128 state, 2^n * 16 (Table 3); 0 if n is outside [0, 62]. */
uint64_t sv_state_bytes(int32_t n_qubits);
/* Device bytes a context of n qubits allocates: two state buffers (psi, lambda) plus
 * reduction scratch.  Unless checkpoints are enabled (sv_set_checkpoint_bytes), at most three
 * state-sized buffers are ever used (31 qubits fit). */
uint64_t sv_ctx_device_bytes(int32_t n_qubits);

/* ---------------------------------------------------------------- contexts */

/* Create a context for n_qubits in [1, 31].  cuda_stream is a cudaStream_t to order work on
 * (cudaStreamLegacy or cudaStreamPerThread for a default stream), or NULL for a stream the
 * context creates and owns.  Allocates psi and lambda (2 x 2^n x 16
 * bytes) and scratch on the current device; SV_ENOMEM if that fails. */
sv_status sv_create(sv_ctx** out, int32_t n_qubits, void* cuda_stream);
/* Free a context and everything it allocated (NULL is accepted). */
sv_status sv_destroy(sv_ctx* ctx);
/* Device memory (bytes) the context may add for psi checkpoints; the default is 0 (psi and
 * lambda only).  Applies to sv_adjoint_grad* and vqe_step.
 * A commuting layer is a run of RY (or RX) gates on distinct qubits.  For up to
 * bytes / (2^n * 16) such layers, the forward pass copies psi before the layer into its own
 * buffer.  The adjoint sweep then takes all of the layer's gradients at its end (the
 * layer's gates commute).  It un-applies the layer to lambda only and copies psi back:
 * 5 instead of 8 FP64 operations per amplitude per gate.  The paper's gradient (Algorithm 1)
 * is unchanged up to rounding.  Buffers are allocated when a circuit is staged, as far as
 * the device allows.  A smaller budget frees the buffers beyond it; SV_EINVAL for a NULL
 * handle. */
sv_status sv_set_checkpoint_bytes(sv_ctx* ctx, uint64_t bytes);
/* Autotuning of the fused-pass tile size; off by default
 * (tiles of 2^11 amplitudes).  When on, the first sv_adjoint_grad* / vqe_step call with a
 * circuit structure not seen before in the process does the following.  Gate types and wires
 * count as structure; angles do not.  It times the forward pass with tiles of 2^9, 2^10 and
 * 2^11 amplitudes and keeps the fastest.  That call therefore runs three extra forward passes
 * on psi, which the evaluation re-initialises.  Results are shared by every context of the
 * process.  If the environment variable SVQE_TUNE_CACHE names a file, results are read from
 * and appended to it as "n key bits" lines.  SV_EINVAL for a NULL handle. */
sv_status sv_set_autotune(sv_ctx* ctx, int32_t enable);
/* Tile size (bits) of the fused passes of the last circuit staged on the context. */
sv_status sv_tile_bits(const sv_ctx* ctx, int32_t* tile_bits);

/* ---------------------------------------------------------------- Hamiltonians */

/* Copy a Pauli sum to the device, grouped by X-flip mask: terms sharing x are one group
 * whose phase-and-sign function f_g(i) = sum_{t in g} c_t i^{popc(x&z_t)} (-1)^{popc(z_t&i)}
 * is tabulated over the bits its z masks touch, so each group reads psi once per amplitude.
 * Mask bits >= n_qubits are SV_EINVAL.  The handle may be used with any context of the same
 * qubit count on the same device. */
sv_status sv_ham_upload(sv_ctx* ctx, const sv_paulisum* h, sv_ham** out);
sv_status sv_ham_free(sv_ham* h);
/* Number of X-mask groups and device bytes of a handle (either pointer may be NULL). */
sv_status sv_ham_info(const sv_ham* h, int32_t* n_groups, uint64_t* device_bytes);

/* Host-only inspection of the grouping sv_ham_upload performs (no device work): with
 * kmax = largest number of z-bits a group table may span (a single term wider than kmax
 * gets a table of its own z-weight), fills n_groups and n_table and,
 * when the array pointers are non-NULL (sized from a first call with NULL arrays), the
 * groups (x, zu, cls, toff) and the tables as interleaved (re, im) doubles.  Group g maps
 * (H psi)[k] += f_g(k) * psi[k ^ x_g] with f_g(k) = table[toff_g + pext(k, zu_g)] and cls 0
 * (real table), 1 (imaginary) or 2 (complex); or, for a group of one term, cls 4 (real) or 5
 * (imaginary) and f_g(k) = table[toff_g] * (-1)^{popc(zu_g & k)}, zu_g being its z mask. */
sv_status sv_ham_lower(const sv_paulisum* h, int32_t kmax, int32_t* n_groups, int64_t* n_table,
                       uint64_t* x, uint64_t* zu, int32_t* cls, int64_t* toff, double* table);

/* Host-only inspection of the fused-pass plan the single-state path uses (no device work;
 * whole-state segments and checkpointed layers, which cut the plan into chunks on the device
 * path, are not applied here): *n_passes receives the number of shared-memory passes
 * over the state and, if pass_of_gate is not NULL, pass_of_gate[g] the pass that applies gate
 * g (n_gates entries).  Gates keep their relative order whenever they share a qubit.
 * tile_bits <= 0 selects the library's tile size (11 bits). */
sv_status sv_circuit_plan(const sv_circuit* circuit, int32_t tile_bits, int32_t* n_passes,
                          int32_t* pass_of_gate);

/* Host-only inspection of the segments the batched kernel runs a circuit as (no device work):
 * *n_segs receives their number and *n_ckpt the checkpoint slots they use.  If segs is not
 * NULL it receives cap rows of 5 int32 (kind, split, first gate, gate count, checkpoint slot
 * or -1), in forward order; cap smaller than the segment count is SV_EINVAL.  Kinds:
 *   0 plain gates, applied one at a time;
 *   1 RY (or RX) gates on distinct qubits (split 1: the first segment, all RY, acting on the
 *     reference state, written as a product state);
 *   2 a run of RZ and CZ gates with at least 3 RZ (at most 16 RZ and 16 CZ);
 *   3 a run of 2 to 32 CNOT/X gates;
 *   4 a kind-2 run directly followed by a kind-3 run (split = gates of the diagonal part).
 * Each checkpoint slot holds a state; a kind-4 segment also keeps its tables there.
 * *team_scratch_amps (if not NULL) receives the checkpoint scratch one instance needs, in
 * amplitudes.  Gates are numbered as in the circuit. */
sv_status sv_batch_segments(const sv_circuit* circuit, int32_t cap, int32_t* segs,
                            int32_t* n_segs, int32_t* n_ckpt, int64_t* team_scratch_amps);

/* ---------------------------------------------------------------- one state */

/* psi = |basis_index> (Eq. 4); also records it as the context's reference state, the
 * starting point of sv_adjoint_grad and vqe_step.  basis_index must be < 2^n. */
sv_status sv_init_reference(sv_ctx* ctx, uint64_t basis_index);
/* psi <- U(theta) psi, gates in list order (Sec. 3.3, Eq. 4-5: the ansatz acting on the
 * reference state).  theta: host array of circuit->n_params angles; a gate whose param is -1
 * uses its fixed_angle.  SV_EINVAL for a malformed gate record (unknown type, wire outside
 * [0, n), duplicate wire, parameter index out of range) or circuit->n_qubits != the
 * context's n; nothing is applied then. */
sv_status sv_apply_circuit(sv_ctx* ctx, const sv_circuit* circuit, const double* theta);
/* *energy_out = <psi|H|psi> for the context's current psi (Eq. 2). */
sv_status sv_expval_paulisum(sv_ctx* ctx, const sv_ham* h, double* energy_out);
/* Energy and gradient of E(theta) = <ref|U^dag H U|ref> (Sec. 3.1, Eq. 2 with the state of
 * Eq. 4; the gradient step of Algorithm 1, Sec. 4.3), with |ref> the reference state of the
 * last sv_init_reference (|0> if none).  The paper differentiates by parameter shift; this
 * call reaches the same gradient by the adjoint method.  Forward pass, lambda = H psi, then the adjoint sweep
 * over gates in reverse: g_p += 2 Im<lambda|G_l|psi> for each gate l with parameter p, then
 * psi <- U_l^dag psi and lambda <- U_l^dag lambda.  Uses psi and lambda only, unless
 * checkpoints are enabled (sv_set_checkpoint_bytes).  energy_out:
 * host double; grad_out: host array of n_params (gates sharing a parameter are summed). */
sv_status sv_adjoint_grad(sv_ctx* ctx, const sv_circuit* circuit, const double* theta,
                          const sv_ham* h, double* energy_out, double* grad_out);
/* As sv_adjoint_grad with device pointers (theta_dev: n_params doubles; energy_dev: 1
 * double; grad_dev: n_params doubles).  Stream-ordered; does not synchronise. */
sv_status sv_adjoint_grad_dev(sv_ctx* ctx, const sv_circuit* circuit, const double* theta_dev,
                              const sv_ham* h, double* energy_dev, double* grad_dev);
/* n_steps of gradient descent theta <- theta - lr * dE/dtheta from the reference state
 * (Algorithm 1's inner loop with a fixed step).  theta_inout: host, n_params, updated in
 * place.  energy_out: host array of n_steps (E before each update) or NULL. */
sv_status vqe_step(sv_ctx* ctx, const sv_circuit* circuit, const sv_ham* h, double* theta_inout,
                   double lr, int32_t n_steps, double* energy_out);
/* Copy psi to / from host memory (2^n interleaved complex128). */
sv_status sv_get_state(sv_ctx* ctx, void* host_out);
sv_status sv_set_state(sv_ctx* ctx, const void* host_in);
/* Device address of psi (valid until sv_destroy). */
sv_status sv_state_device_ptr(sv_ctx* ctx, void** psi_dev);

/* ---------------------------------------------------------------- batches */

/* One instance of a batch: its circuit, its Hamiltonian and its reference basis index.
 * circuit.n_qubits must equal ham.n_qubits and lie in [1, SV_BATCH_MAX_QUBITS]. */
typedef struct {
  sv_circuit circuit;
  sv_paulisum ham;
  uint64_t ref;
} sv_instance;

#define SV_BATCH_MAX_QUBITS 12

/* Compile and upload n instances (Sec. 4.1, Eq. 7: independent problems) for the persistent
 * batched kernel, which keeps each instance's psi and lambda in shared memory.  Theta and
 * gradients of all instances are concatenated in instance order (offsets = prefix sums of
 * n_params).  cuda_stream: NULL for an owned stream. */
sv_status sv_batch_create(const sv_instance* inst, int32_t n, void* cuda_stream,
                          sv_batch** out);
sv_status sv_batch_free(sv_batch* b);
/* Layout autotuner of the batched kernel (process-wide; off by default).  The kernel's layout
 * for the instances of one qubit count q is the number of warps that run each instance and the
 * widths at which runs of gates become segments: a run of RY/RX gates on distinct qubits is
 * one commuting-layer segment, and a run of RZ/CZ gates one diagonal segment, only when it is
 * long enough; shorter runs are applied gate by gate (see sv_batch_segments).  Off, every batch
 * uses a fixed rule (the smallest team that holds the instance; layers of >= 2 gates and
 * diagonal runs of >= 3 RZ gates become segments).  On, sv_batch_create first measures, for
 * each qubit count of the batch not measured before in this process, the candidate layouts
 * (that team and the one with twice its warps; layer segments on or off; diagonal segments on
 * or off) on a calibration batch made of that count's instances, and compiles the batch with
 * the fastest.  The results are cached for the process and, if the environment variable
 * SVQE_BATCH_TUNE_CACHE names a file, read from and appended to that file.  The tuning runs
 * on the batch's stream and synchronises it; call it outside any stream capture. */
sv_status sv_batch_set_autotune(int32_t enable);
/* Put a layout for n_qubits-qubit instances into the tuner's process-wide cache, so that
 * batches created while the tuner is on use it without measuring: team_warps (1, 2, 4 or 8;
 * 2^n_qubits <= 512 x team_warps), and the two segment widths (>= 1).  team_warps = 0 removes
 * the entry, so that the next tuned batch measures that size again.  SV_EINVAL for a layout
 * that cannot hold the instances.  Host-only. */
sv_status sv_batch_set_layout(int32_t n_qubits, int32_t team_warps, int32_t min_layer,
                              int32_t min_diag_rz);
/* The layout b was compiled with for n_qubits-qubit instances: warps per instance team and the
 * two segment widths (a width of 2^20 means that segment kind is not used).  All three are 0
 * when b holds no instance of that size.  Host-only.  Any output pointer may be NULL. */
sv_status sv_batch_layout(const sv_batch* b, int32_t n_qubits, int32_t* team_warps,
                          int32_t* min_layer, int32_t* min_diag_rz);
/* Sizes: instances, total parameters. */
sv_status sv_batch_info(const sv_batch* b, int32_t* n_instances, int64_t* n_params_total);
/* Algorithmic cost of one sv_batch_run, counted from the compiled segments exactly as the
 * kernel executes them: fp64_flops (FMA = 2) of the forward pass, lambda = H psi and the
 * adjoint sweep; hbm_bytes read and written (program, tables, parameters, results,
 * checkpoints).  Either pointer may be NULL.  Host-only. */
sv_status sv_batch_cost(const sv_batch* b, double* fp64_flops, double* hbm_bytes);
/* Energy and adjoint gradient of every instance, host buffers: theta (n_params_total) is
 * copied in, energy (n) and grad (n_params_total) are copied out; synchronises. */
sv_status sv_batch_run(sv_batch* b, const double* theta, double* energy, double* grad);
/* The same on device buffers; one persistent launch, replayed from a CUDA graph captured on
 * the first call for these pointers.  Stream-ordered; does not synchronise. */
sv_status sv_batch_run_dev(sv_batch* b, const double* theta_dev, double* energy_dev,
                           double* grad_dev);
/* n_steps of gradient descent on every instance inside one persistent launch:
 * theta_dev is updated in place; energy_traj_dev (n_steps x n, step-major) receives E before
 * each update, or may be NULL.  Stream-ordered. */
sv_status sv_batch_vqe_dev(sv_batch* b, double* theta_dev, double lr, int32_t n_steps,
                           double* energy_traj_dev);

/* n_steps of Adam, the paper's optimizer (Sec. 3.4; Algorithm 1's update), on every instance
 * inside one persistent launch: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
 * theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) with b1 = 0.9,
 * b2 = 0.999, eps = 1e-8 and t the update count.  The moments live in the batch; reset = 1
 * starts from zero moments and t = 0, reset = 0 continues from the previous call (the first
 * call always resets).  energy_traj_dev as for sv_batch_vqe_dev.  Stream-ordered. */
sv_status sv_batch_adam_dev(sv_batch* b, double* theta_dev, double lr, int32_t n_steps,
                            double* energy_traj_dev, int32_t reset);

/* ---------------------------------------------------------------- serving */

/* A request loop that serves many independent VQE optimisations (Sec. 4.1, Eq. 7: every
 * problem is independent) as they arrive.  A scheduler thread admits queued requests in
 * arrival order while their device footprint fits hbm_budget_bytes.  Requests of at most
 * SV_BATCH_MAX_QUBITS qubits become resident in a device arena (program, tables, parameters,
 * trajectory) and advance together, steps_per_tick gradient steps per persistent batched
 * launch; a request that arrives while a launch runs joins at the next launch, and one that
 * finishes leaves and frees its memory.  Larger requests get their own state buffers and
 * stream and run concurrently with the batched launches (at most max_active_large at once).
 * Each request runs n_steps of gradient descent theta <- theta - lr * dE/dtheta from theta0
 * (Algorithm 1's loop with a fixed step) and returns its final theta and the energies before
 * each update.  A request's results do not depend on which other requests shared its launches.
 * serial = 1 runs one request at a time, with no batching (the one-circuit-at-a-time baseline).
 * Large requests of at least heavy_qubits qubits (default 20) fill the GPU by themselves, so
 * at most max_active_heavy of them (default 2) run at once; the other large-request slots stay
 * free for mid-size requests, whose many short launches then overlap the heavy ones.  The
 * batched launches and mid-size requests run on streams of the device's greatest priority,
 * heavy requests on its least, so that the block scheduler starts short work first.
 * Zero fields take defaults: 4 GiB, 4096, 1, 8, 2, 20.  The server reserves a device arena of
 * min(hbm_budget_bytes, 6 GiB) for small requests at creation; a large request gets its own
 * buffers when admitted, and keeps them idle after it finishes for the next request of the same
 * qubit count (at most max_active_large idle sets), so that steady-state admission and
 * completion allocate and free nothing on the device.  The admitted requests' footprints and
 * the idle buffers together never exceed the budget; idle buffers are freed when an admission
 * needs their room. */
typedef struct {
  uint64_t hbm_budget_bytes;
  int32_t max_active_small;
  int32_t steps_per_tick;
  int32_t max_active_large;
  int32_t serial;
  int32_t max_active_heavy;
  int32_t heavy_qubits;
} sv_server_config;

/* Times are seconds since the server was created. */
typedef struct {
  uint64_t id;
  int32_t status;      /* SV_OK done; SV_EBUSY queued or running; otherwise the failure */
  int32_t n_qubits;
  int32_t n_params;
  int32_t n_steps;
  uint64_t footprint_bytes;
  double submit_s;
  double admit_s;
  double done_s;
} sv_request_info;

typedef struct {
  uint64_t submitted, completed, failed, cancelled;
  uint64_t launches;           /* batched launches issued */
  uint64_t bytes_in_use;       /* device bytes held by admitted requests now */
  uint64_t peak_bytes_in_use;  /* never above hbm_budget_bytes */
  int32_t queued, running;
} sv_server_stats;

/* Create a server on the current device (allocates its arena and scratch). */
sv_status sv_server_create(const sv_server_config* cfg, sv_server** out);
/* Queue a request.  The instance and theta0 (circuit.n_params angles) are copied; validation
 * errors and a footprint larger than the whole budget are returned here (SV_EINVAL /
 * SV_ENOMEM).  *id receives the request's id. */
sv_status sv_server_submit(sv_server* s, const sv_instance* inst, const double* theta0,
                           int32_t n_steps, double lr, uint64_t* id);
/* Wait up to timeout_ms (< 0: forever) for request id.  SV_ETIMEOUT if it has not finished;
 * otherwise its final status, with theta_out (n_params) and energy_out (n_steps) filled when
 * not NULL and info when not NULL.  A finished request is forgotten after this call. */
sv_status sv_server_wait(sv_server* s, uint64_t id, int32_t timeout_ms, double* theta_out,
                         double* energy_out, sv_request_info* info);
/* Cancel a request that is still queued (SV_EBUSY if it is already running). */
sv_status sv_server_cancel(sv_server* s, uint64_t id);
sv_status sv_server_get_stats(sv_server* s, sv_server_stats* out);
/* Cancel queued requests, finish running ones, free everything. */
sv_status sv_server_destroy(sv_server* s);

/* ---------------------------------------------------------------- measurement */

/* FP64 issue-rate probe, the denominator of the batched kernel's roofline (that kernel is
 * bound by double-precision arithmetic, not by memory).  It has no counterpart in the paper.
 * Launches `blocks` x `threads` threads, each running `chains` (1, 2, 4, 8 or 16)
 * independent chains of `iters` fused multiply-adds on doubles, on cuda_stream (NULL: the
 * legacy default stream), and writes one double per thread to out_dev (device,
 * blocks * threads doubles, caller-owned).  *dfma_out (host, may be NULL) receives the number
 * of FMAs the launch executes.  The caller times the launch (for example with events on the
 * same stream).  SV_EINVAL for threads not a multiple of 32 in [32, 1024], blocks < 1,
 * iters < 1, another chain count or a NULL out_dev. */
sv_status sv_fp64_probe(int32_t blocks, int32_t threads, int32_t chains, int32_t iters,
                        double* out_dev, void* cuda_stream, double* dfma_out);

/* ---------------------------------------------------------------- no device allocation */

/* This entry point has no counterpart in the paper; it exists for callers that cannot
 * allocate device memory.  Those are programs whose host application owns every byte of
 * device memory (a framework's caching allocator, or a fixed budget reserved at start-up) and
 * forbids allocations by anyone else, and latency-critical loops that must not pay for, or
 * risk the failure of, a cudaMalloc after start-up.  The caller brings every input and output
 * buffer; the working memory (psi, lambda, op records, rotation coefficients, reduction
 * partials) lives in one fixed array of SV_NOALLOC_SCRATCH_BYTES inside the library, which
 * every GPU that loads the library holds until the process exits.  The call allocates no
 * device memory and makes no allocating library call.
 *
 * sv_adjoint_grad_noalloc computes the same energy and gradient as sv_adjoint_grad_dev, for
 * states of at most SV_NOALLOC_MAX_QUBITS qubits and circuits of at most
 * SV_NOALLOC_MAX_GATES gates; larger requests are rejected with SV_EINVAL and a message
 * naming the limit.
 *   circuit      host gate records (validated as for sv_apply_circuit).
 *   ref          basis index of the reference state, < 2^n.
 *   ham_n_qubits the register width the group records were lowered for; it must equal
 *                circuit->n_qubits (SV_EINVAL otherwise), because a wire maps to bit n-1-wire
 *                and records lowered for another width describe another operator.
 *   groups_dev   device array (8-byte aligned) of n_groups sv_group records, and tables_dev
 *                the device array of n_table interleaved complex128 table entries, both as
 *                sv_ham_lower reports them for the Hamiltonian (x_mask, z_union,
 *                z_bits = popcount(z_union), cls, table_offset).  n_groups <= 2^n.
 *   theta_dev    device array of circuit->n_params angles.
 *   energy_dev   device address receiving E; grad_dev device array of n_params derivatives.
 *   cuda_stream  cudaStream_t to order the work on (NULL: the legacy default stream).
 * The records sit in device memory, so the host cannot read them: a kernel checks each one
 * (masks inside the register, a known class, its table range inside [0, n_table)) before
 * anything is read through it.  If any record fails, no out-of-range read happens and the
 * call writes NaN to energy_dev and grad_dev; the status is still SV_OK, since the call
 * returns before the check runs.
 * Stream-ordered; returns without synchronising.  The first call on a device looks up the
 * array's device address once (cudaGetSymbolAddress with that device current); make that
 * first call before any stream capture.  Every call on a device shares the one array and
 * leaves its contents behind; calls whose work overlaps on the GPU (other streams or other
 * threads) race on it, so the caller must order them. */
typedef struct {
  uint64_t x_mask;
  uint64_t z_union;
  int32_t z_bits;
  int32_t cls;
  int64_t table_offset;
} sv_group;

#define SV_NOALLOC_MAX_QUBITS 14
#define SV_NOALLOC_MAX_GATES 256
#define SV_NOALLOC_SCRATCH_BYTES (4u << 20)

sv_status sv_adjoint_grad_noalloc(const sv_circuit* circuit, uint64_t ref,
                                  int32_t ham_n_qubits, const sv_group* groups_dev,
                                  int32_t n_groups, const double* tables_dev, int64_t n_table,
                                  const double* theta_dev, double* energy_dev,
                                  double* grad_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SVQE_H */
