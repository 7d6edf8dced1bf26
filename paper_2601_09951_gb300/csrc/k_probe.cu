// k_probe.cu -- FP64 issue-rate probe (sv_fp64_probe).
//
// The batched kernel is bound by the FP64 pipe, not by HBM, so its roofline denominator is
// the rate at which the SMs retire double-precision fused multiply-adds.  This kernel
// measures that rate: every thread runs CHAINS independent dependency chains
// x <- fma(x, a, b), so that with enough chains and warps the pipe, not the FMA latency,
// limits it.  a and b are kernel arguments (the compiler cannot fold the chains), and
// multipliers below 1 keep every value finite and normal: each chain converges to
// c / (1 - m).
#include <cuda_runtime.h>

#include "../../include/svqe.h"
#include "api_internal.h"

namespace svqe {
namespace {

template <int CHAINS>
__global__ void k_fp64_probe(int iters, double a, double b, double* __restrict__ out) {
  // Each chain has its own multiplier and addend in registers (derived from the thread index,
  // so the compiler cannot take them from the constant bank or share them), the form the
  // state-vector kernels' FMAs take.
  double x[CHAINS], m[CHAINS], c[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) {
    const double t = (double)((threadIdx.x + 3 * k) & 15);
    x[k] = t * 1e-3;
    m[k] = a - t * 1e-12;
    c[k] = b + t * 1e-12;
  }
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], m[k], c[k]);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  // one store per thread keeps the chains live; it is not part of the count
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace svqe

using namespace svqe;

extern "C" sv_status sv_fp64_probe(int32_t blocks, int32_t threads, int32_t chains,
                                   int32_t iters, double* out_dev, void* cuda_stream,
                                   double* dfma_out) {
  clear_error();
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1 ||
      !out_dev || (chains != 1 && chains != 2 && chains != 4 && chains != 8 && chains != 16)) {
    set_error("bad probe shape (blocks %d, threads %d, chains %d, iters %d) or NULL output",
              blocks, threads, chains, iters);
    return SV_EINVAL;
  }
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  const double a = 0.9999999, b = 1e-7;
  switch (chains) {
    case 1: k_fp64_probe<1><<<blocks, threads, 0, s>>>(iters, a, b, out_dev); break;
    case 2: k_fp64_probe<2><<<blocks, threads, 0, s>>>(iters, a, b, out_dev); break;
    case 4: k_fp64_probe<4><<<blocks, threads, 0, s>>>(iters, a, b, out_dev); break;
    case 8: k_fp64_probe<8><<<blocks, threads, 0, s>>>(iters, a, b, out_dev); break;
    default: k_fp64_probe<16><<<blocks, threads, 0, s>>>(iters, a, b, out_dev); break;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("k_fp64_probe: %s", cudaGetErrorString(e));
    return SV_ECUDA;
  }
  if (dfma_out) *dfma_out = (double)blocks * threads * (double)chains * iters;
  return SV_OK;
}
