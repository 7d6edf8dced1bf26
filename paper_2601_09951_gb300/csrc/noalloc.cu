// noalloc.cu -- energy and adjoint gradient of one small state without allocating device
// memory (sv_adjoint_grad_noalloc).
//
// Who needs this: code that runs inside a host application which owns every byte of device
// memory (a framework's caching allocator, or a fixed memory budget reserved at start-up) and
// forbids any other allocation, and latency-critical loops that must not pay for, or risk the
// failure of, a cudaMalloc after start-up.  Such callers bring their own input and output
// buffers; the working memory the computation needs (psi, lambda, op records, rotation
// coefficients, reduction partials) lives here, in one file-scope __device__ array that every
// GPU which loads this library holds until the process exits.
//
// The array is shared by every call on a device and keeps the previous call's contents.  No
// part of it needs to start at zero: each call writes every region before reading it.  Calls
// whose work overlaps on the GPU (different streams, or different host threads) race on the
// array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/svqe.h"
#include "host_compile.h"
#include "launch.h"
#include "svqe_types.h"

namespace svqe {
namespace {

static_assert(sizeof(sv_group) == sizeof(DGroup), "sv_group must match the device group record");

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Layout of the scratch array (byte offsets).
constexpr size_t kStateBytes = (size_t)16 << SV_NOALLOC_MAX_QUBITS;
constexpr size_t kOffPsi = 0;
constexpr size_t kOffLam = kOffPsi + align256(kStateBytes);
constexpr size_t kOffOps = kOffLam + align256(kStateBytes);
constexpr size_t kOffCoef = kOffOps + align256(sizeof(DOp) * SV_NOALLOC_MAX_GATES);
constexpr size_t kOffContrib = kOffCoef + align256(sizeof(Rot) * SV_NOALLOC_MAX_GATES);
constexpr size_t kOffGpart = kOffContrib + align256(sizeof(double) * SV_NOALLOC_MAX_GATES);
constexpr size_t kOffEpart =
    kOffGpart + align256(sizeof(double) * (size_t)kRedBlocks * SV_NOALLOC_MAX_GATES);
constexpr size_t kScratchBytes = kOffEpart + align256(sizeof(double) * kRedBlocks);
static_assert(kScratchBytes <= SV_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds its stated size");

// The scratch itself.  In host code this name is only a host-side stand-in: its device address
// comes from cudaGetSymbolAddress (see scratch_address).
static __device__ __align__(256) unsigned char g_scratch[SV_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device.
sv_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("cudaGetDevice: %s", cudaGetErrorString(e));
    return SV_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device index %d out of range", dev);
    return SV_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress(scratch) on device %d: %s", dev, cudaGetErrorString(e));
      return SV_ECUDA;
    }
    g_addr[dev] = (unsigned char*)p;
  }
  *out = g_addr[dev];
  return SV_OK;
}

#define NA_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      set_error("%s: %s", #call, cudaGetErrorString(e_));                                \
      return SV_ECUDA;                                                                   \
    }                                                                                    \
  } while (0)

}  // namespace
}  // namespace svqe

using namespace svqe;

extern "C" sv_status sv_adjoint_grad_noalloc(const sv_circuit* circuit, uint64_t ref,
                                             const sv_group* groups_dev, int32_t n_groups,
                                             const double* tables_dev, const double* theta_dev,
                                             double* energy_dev, double* grad_dev,
                                             void* cuda_stream) {
  clear_error();
  if (!circuit || !energy_dev || (n_groups > 0 && (!groups_dev || !tables_dev)) ||
      n_groups < 0) {
    set_error("NULL or negative argument");
    return SV_EINVAL;
  }
  if (circuit->n_qubits < 1 || circuit->n_qubits > SV_NOALLOC_MAX_QUBITS) {
    set_error("n_qubits %d outside [1, %d]: the scratch array holds states of at most %d "
              "qubits", circuit->n_qubits, SV_NOALLOC_MAX_QUBITS, SV_NOALLOC_MAX_QUBITS);
    return SV_EINVAL;
  }
  if (circuit->n_gates > SV_NOALLOC_MAX_GATES) {
    set_error("%d gates exceed the scratch array's limit of %d", circuit->n_gates,
              SV_NOALLOC_MAX_GATES);
    return SV_EINVAL;
  }
  HostCircuit hc;
  sv_status st = lower_circuit(circuit, circuit->n_qubits, hc);
  if (st != SV_OK) return st;
  if (hc.n_params > 0 && (!theta_dev || !grad_dev)) {
    set_error("theta/grad is NULL");
    return SV_EINVAL;
  }
  const int n = hc.n;
  if (ref >= (1ull << n)) {
    set_error("reference index %llu >= 2^%d", (unsigned long long)ref, n);
    return SV_EINVAL;
  }
  unsigned char* base = nullptr;
  if ((st = scratch_address(&base)) != SV_OK) return st;
  double2* psi = (double2*)(base + kOffPsi);
  double2* lam = (double2*)(base + kOffLam);
  DOp* ops = (DOp*)(base + kOffOps);
  Rot* coef = (Rot*)(base + kOffCoef);
  double* contrib = (double*)(base + kOffContrib);
  double* gpart = (double*)(base + kOffGpart);
  double* epart = (double*)(base + kOffEpart);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int n_ops = (int)hc.ops.size();
  if (n_ops)
    NA_CUDA(cudaMemcpyAsync(ops, hc.ops.data(), n_ops * sizeof(DOp), cudaMemcpyHostToDevice, s));
  NA_CUDA(launch_init_basis(psi, n, ref, s));
  NA_CUDA(launch_prep_coefs(ops, n_ops, theta_dev, coef, s));
  for (int l = 0; l < n_ops; ++l) NA_CUDA(launch_apply_op(psi, n, hc.ops[l], coef + l, false, s));
  NA_CUDA(launch_hpsi(psi, lam, n, (const DGroup*)groups_dev, n_groups,
                      (const double2*)tables_dev, epart, s));
  NA_CUDA(launch_sum(epart, kRedBlocks, energy_dev, s));
  for (int l = n_ops - 1; l >= 0; --l) {
    double* part = hc.ops[l].param >= 0 ? gpart + (size_t)l * kRedBlocks : nullptr;
    NA_CUDA(launch_adjoint_op(psi, lam, n, hc.ops[l], coef + l, part, s));
  }
  if (n_ops || hc.n_params)
    NA_CUDA(launch_reduce_grads(ops, n_ops, gpart, hc.n_params, contrib, grad_dev, s));
  return SV_OK;
}
