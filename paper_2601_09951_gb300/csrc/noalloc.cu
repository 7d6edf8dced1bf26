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
// The array is shared by every call on a device and keeps the previous call's contents.  The
// one word that must start at zero, the bad-record flag, is cleared by the first kernel of each
// call; every other region is written before it is read.  Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array and must be serialised by
// the caller.
//
// The Hamiltonian's group records live in the caller's device memory, where the host cannot
// inspect them.  A one-block kernel therefore checks each record against the declared register
// width and table size before any kernel reads the state through it, and copies it into the
// array; a record that fails is replaced by one that reads only table entry 0 and psi[k], and
// the call's outputs are then overwritten with NaN.  No record can make a kernel read outside
// psi, lambda or the caller's table.
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
// A register of n qubits has at most 2^n distinct X masks, hence at most 2^n groups.
constexpr int kMaxGroups = 1 << SV_NOALLOC_MAX_QUBITS;
constexpr size_t kOffGroups = kOffEpart + align256(sizeof(double) * kRedBlocks);
constexpr size_t kOffFlag = kOffGroups + align256(sizeof(DGroup) * (size_t)kMaxGroups);
constexpr size_t kScratchBytes = kOffFlag + 256;
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

// Op records travel to the device as kernel parameters (by value, copied at launch), so the
// upload reads no host memory after the call returns.
constexpr int kOpChunk = 64;
struct OpChunk {
  DOp op[kOpChunk];
};
static_assert(sizeof(OpChunk) <= 4096, "op chunk must stay a small kernel parameter");

__global__ void k_na_put_ops(OpChunk c, DOp* __restrict__ dst, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = c.op[i];
}

// Checks every caller record (x_mask and z_union inside the n-qubit register, a known class,
// and a table range inside [0, n_table): 2^popcount(z_union) entries for a table group, one for
// a single-term group) and copies it to `out`.  A failing record becomes {x 0, z 0, single
// real term at entry 0}, which reads only psi[k] and table entry 0 (n_table >= 1 is checked
// on the host), and sets *flag.  One block; the flag is cleared first.
__global__ void k_na_check_groups(const sv_group* __restrict__ in, int n_groups, int n,
                                  long long n_table, DGroup* __restrict__ out,
                                  unsigned* __restrict__ flag) {
  __shared__ unsigned bad;
  if (threadIdx.x == 0) bad = 0u;
  __syncthreads();
  const uint64_t outside = ~((n >= 64) ? ~0ull : ((1ull << n) - 1ull));
  for (int g = threadIdx.x; g < n_groups; g += blockDim.x) {
    const sv_group r = in[g];
    bool ok = ((r.x_mask | r.z_union) & outside) == 0 && r.table_offset >= 0 &&
              (r.cls == 0 || r.cls == 1 || r.cls == 2 || r.cls == 4 || r.cls == 5);
    if (ok) {
      // popcount(z_union) <= n <= 14 here, so the shift is in range
      const long long entries = r.cls >= 4 ? 1ll : (1ll << __popcll(r.z_union));
      ok = r.table_offset <= n_table - entries;
    }
    DGroup d;
    if (ok) {
      d.x = r.x_mask;
      d.zu = r.z_union;
      d.kz = __popcll(r.z_union);
      d.cls = r.cls;
      d.toff = r.table_offset;
    } else {
      d.x = 0;
      d.zu = 0;
      d.kz = 0;
      d.cls = 4;
      d.toff = 0;
      atomicOr(&bad, 1u);
    }
    out[g] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) *flag = bad;
}

// After a call that met a failing record: energy and every gradient entry become NaN.
__global__ void k_na_poison(const unsigned* __restrict__ flag, double* __restrict__ energy,
                            double* __restrict__ grad, int n_params) {
  if (*flag == 0u) return;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (threadIdx.x == 0) *energy = nan;
  for (int p = threadIdx.x; p < n_params; p += blockDim.x) grad[p] = nan;
}

}  // namespace
}  // namespace svqe

using namespace svqe;

extern "C" sv_status sv_adjoint_grad_noalloc(const sv_circuit* circuit, uint64_t ref,
                                             int32_t ham_n_qubits, const sv_group* groups_dev,
                                             int32_t n_groups, const double* tables_dev,
                                             int64_t n_table, const double* theta_dev,
                                             double* energy_dev, double* grad_dev,
                                             void* cuda_stream) {
  clear_error();
  if (!circuit || !energy_dev || (n_groups > 0 && (!groups_dev || !tables_dev)) ||
      n_groups < 0 || n_table < 0) {
    set_error("NULL or negative argument");
    return SV_EINVAL;
  }
  if (circuit->n_qubits < 1 || circuit->n_qubits > SV_NOALLOC_MAX_QUBITS) {
    set_error("n_qubits %d outside [1, %d]: the scratch array holds states of at most %d "
              "qubits", circuit->n_qubits, SV_NOALLOC_MAX_QUBITS, SV_NOALLOC_MAX_QUBITS);
    return SV_EINVAL;
  }
  if (ham_n_qubits != circuit->n_qubits) {
    set_error("the Hamiltonian's records were lowered for %d qubits, the circuit has %d",
              ham_n_qubits, circuit->n_qubits);
    return SV_EINVAL;
  }
  if (circuit->n_gates > SV_NOALLOC_MAX_GATES) {
    set_error("%d gates exceed the scratch array's limit of %d", circuit->n_gates,
              SV_NOALLOC_MAX_GATES);
    return SV_EINVAL;
  }
  if (n_groups > kMaxGroups) {
    set_error("%d groups: a %d-qubit register has at most %d distinct X masks", n_groups,
              circuit->n_qubits, 1 << circuit->n_qubits);
    return SV_EINVAL;
  }
  if (n_groups > 0 && n_table < 1) {
    set_error("%d groups but an empty table", n_groups);
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
  DGroup* groups = (DGroup*)(base + kOffGroups);
  unsigned* flag = (unsigned*)(base + kOffFlag);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int n_ops = (int)hc.ops.size();
  for (int i0 = 0; i0 < n_ops; i0 += kOpChunk) {
    OpChunk c;
    const int cnt = n_ops - i0 < kOpChunk ? n_ops - i0 : kOpChunk;
    for (int i = 0; i < cnt; ++i) c.op[i] = hc.ops[i0 + i];
    k_na_put_ops<<<1, kOpChunk, 0, s>>>(c, ops + i0, cnt);
    NA_CUDA(cudaGetLastError());
  }
  k_na_check_groups<<<1, 1024, 0, s>>>(groups_dev, n_groups, n, (long long)n_table, groups,
                                       flag);
  NA_CUDA(cudaGetLastError());
  NA_CUDA(launch_init_basis(psi, n, ref, s));
  NA_CUDA(launch_prep_coefs(ops, n_ops, theta_dev, coef, s));
  for (int l = 0; l < n_ops; ++l) NA_CUDA(launch_apply_op(psi, n, hc.ops[l], coef + l, false, s));
  NA_CUDA(launch_hpsi(psi, lam, n, groups, n_groups, (const double2*)tables_dev, epart, s));
  NA_CUDA(launch_sum(epart, kRedBlocks, energy_dev, s));
  for (int l = n_ops - 1; l >= 0; --l) {
    double* part = hc.ops[l].param >= 0 ? gpart + (size_t)l * kRedBlocks : nullptr;
    NA_CUDA(launch_adjoint_op(psi, lam, n, hc.ops[l], coef + l, part, s));
  }
  if (n_ops || hc.n_params)
    NA_CUDA(launch_reduce_grads(ops, n_ops, gpart, hc.n_params, contrib, grad_dev, s));
  k_na_poison<<<1, 256, 0, s>>>(flag, energy_dev, grad_dev, hc.n_params);
  NA_CUDA(cudaGetLastError());
  return SV_OK;
}
