// svqe_internal.cuh -- types and device arithmetic shared by the CUDA translation units.
//
// Design rule for GB300: FP64 issue rate is ~2 DFMA/clk/SM (measured 598 G DFMA/s on the
// whole chip) against ~64 integer and ~110 FP32 lane-ops/clk/SM.  Every kernel here is
// therefore written to minimise FP64 instructions per amplitude:
//   * sign flips and multiplications by +-1, +-i are integer bit operations or swaps;
//   * a real 2x2 rotation is applied as three shears ("lifting", x += a*y; y += b*x;
//     x += a*y), 3 DFMA per real pair instead of 2 DMUL + 2 DFMA, after reducing the angle
//     to [-pi/4, pi/4] with an exact quarter-turn (a swap and sign flips);
//   * Pauli groups are applied through tabulated f_g(i), one complex or real multiply-add
//     per amplitude per group whatever the number of terms in the group.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/svqe.h"
#include "svqe_types.h"

namespace svqe {

// Negation by flipping the sign bit (an integer op: never issued to the FP64 pipe).
__device__ __forceinline__ double dneg(double v) {
  return __hiloint2double(__double2hiint(v) ^ 0x80000000, __double2loint(v));
}

// Insert zero bits at the sorted positions sb[0..k) of counter p.
__device__ __forceinline__ uint64_t insert_zeros(uint64_t p, const uint8_t* sb, int k) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t < k) {
      const uint64_t low = p & ((1ull << sb[t]) - 1ull);
      p = ((p >> sb[t]) << (sb[t] + 1)) | low;
    }
  }
  return p;
}

// Gather the bits of i selected by mask m into the low bits (software pext).
__device__ __forceinline__ uint32_t pext64(uint64_t i, uint64_t m) {
  uint32_t r = 0;
  int k = 0;
  while (m) {
    const int pos = __ffsll((long long)m) - 1;
    r |= (uint32_t)((i >> pos) & 1ull) << k;
    ++k;
    m &= m - 1;
  }
  return r;
}

// Rotation coefficients for R(phi), computed once per gate (not per amplitude).
__device__ __forceinline__ Rot make_rot(double phi) {
  double s, c;
  sincos(phi, &s, &c);
  Rot r;
  double cr, sr;
  if (fabs(c) >= fabs(s)) {
    if (c >= 0) { r.k = 0; cr = c; sr = s; } else { r.k = 2; cr = -c; sr = -s; }
  } else {
    if (s > 0) { r.k = 1; cr = s; sr = -c; } else { r.k = 3; cr = -s; sr = c; }
  }
  r.a = -sr / (1.0 + cr);
  r.b = sr;
  r.pad = 0;
  return r;
}

// Coefficients of R(-phi) from those of R(phi).
__device__ __forceinline__ Rot rot_inverse(const Rot& r) {
  Rot q;
  q.k = (4 - r.k) & 3;
  q.a = dneg(r.a);
  q.b = dneg(r.b);
  q.pad = 0;
  return q;
}

// (x, y) <- R(phi) (x, y): an exact quarter turn, then three shears (3 DFMA).
__device__ __forceinline__ void rot_apply(const Rot& r, double& x, double& y) {
  double u = x, v = y;
  switch (r.k) {
    case 1: u = dneg(y); v = x; break;
    case 2: u = dneg(x); v = dneg(y); break;
    case 3: u = y; v = dneg(x); break;
    default: break;
  }
  u = fma(r.a, v, u);
  v = fma(r.b, u, v);
  u = fma(r.a, v, u);
  x = u;
  y = v;
}

// ------------------------------------------------------------------------------ gate math
// Coefficients of a compiled op: rotation ops store Rot(theta/2).
struct Coef {
  Rot r;
};

__device__ __forceinline__ Coef make_coef(const DOp& op, const double* theta) {
  Coef c;
  const double t = op.param >= 0 ? theta[op.param] : op.fixed;
  if (is_param_type(op.type)) {
    c.r = make_rot(0.5 * t);
  } else {
    c.r.a = c.r.b = 0.0;
    c.r.k = 0;
    c.r.pad = 0;
  }
  return c;
}

// Apply (inv = false) or un-apply (inv = true) a pair gate to (x, y) = (psi[i], psi[j]).
__device__ __forceinline__ void pair_apply(int type, const Rot& rf, bool inv, double2& x,
                                           double2& y) {
  switch (type) {
    case SV_GATE_X:
    case SV_GATE_CNOT: {
      const double2 t = x; x = y; y = t;
    } break;
    case SV_GATE_H: {
      const double r = 0.70710678118654752440;
      const double2 a = x, b = y;
      x.x = r * (a.x + b.x); x.y = r * (a.y + b.y);
      y.x = r * (a.x - b.x); y.y = r * (a.y - b.y);
    } break;
    case SV_GATE_RY:
    case SV_GATE_SINGLE_EXC:
    case SV_GATE_DOUBLE_EXC: {
      const Rot r = inv ? rot_inverse(rf) : rf;
      rot_apply(r, x.x, y.x);
      rot_apply(r, x.y, y.y);
    } break;
    case SV_GATE_RX: {
      // x' = c x - i s y ; y' = -i s x + c y : R(-phi) on (x.re, y.im), R(phi) on (x.im, y.re)
      const Rot r = inv ? rot_inverse(rf) : rf;
      const Rot m = rot_inverse(r);
      rot_apply(m, x.x, y.y);
      rot_apply(r, x.y, y.x);
    } break;
    case SV_GATE_RZ: {
      // x *= e^{-i phi}: R(-phi) on (x.re, x.im); y *= e^{+i phi}: R(phi) on (y.re, y.im)
      const Rot r = inv ? rot_inverse(rf) : rf;
      const Rot m = rot_inverse(r);
      rot_apply(m, x.x, x.y);
      rot_apply(r, y.x, y.y);
    } break;
    default: break;
  }
}

// 2 Im<lambda|G|psi> restricted to one pair, for the generator G of a parameterised gate
// (U = exp(-i t G)): G = X/2, Y/2, Z/2 for RX/RY/RZ, sigma_y/2 on (lo, hi) for excitations.
__device__ __forceinline__ double pair_grad(int type, const double2& lx, const double2& ly,
                                            const double2& px, const double2& py) {
  switch (type) {
    case SV_GATE_RY:
    case SV_GATE_SINGLE_EXC:
    case SV_GATE_DOUBLE_EXC: {
      // Re(conj(ly) px) - Re(conj(lx) py)
      double v = ly.x * px.x;
      v = fma(ly.y, px.y, v);
      v = fma(dneg(lx.x), py.x, v);
      v = fma(dneg(lx.y), py.y, v);
      return v;
    }
    case SV_GATE_RX: {
      // Im(conj(lx) py) + Im(conj(ly) px)
      double v = lx.x * py.y;
      v = fma(dneg(lx.y), py.x, v);
      v = fma(ly.x, px.y, v);
      v = fma(dneg(ly.y), px.x, v);
      return v;
    }
    case SV_GATE_RZ: {
      // Im(conj(lx) px) - Im(conj(ly) py)
      double v = lx.x * px.y;
      v = fma(dneg(lx.y), px.x, v);
      v = fma(dneg(ly.x), py.y, v);
      v = fma(ly.y, py.x, v);
      return v;
    }
    default:
      return 0.0;
  }
}

// acc += f * v for a group table value f of class cls (0 real, 1 imaginary, 2 complex).
__device__ __forceinline__ void group_madd(int cls, const double2& f, const double2& v,
                                           double2& acc) {
  if (cls == 0) {
    acc.x = fma(f.x, v.x, acc.x);
    acc.y = fma(f.x, v.y, acc.y);
  } else if (cls == 1) {
    // (i fi) v = (-fi v.im, fi v.re)
    acc.x = fma(dneg(f.y), v.y, acc.x);
    acc.y = fma(f.y, v.x, acc.y);
  } else {
    acc.x = fma(f.x, v.x, acc.x);
    acc.x = fma(dneg(f.y), v.y, acc.x);
    acc.y = fma(f.x, v.y, acc.y);
    acc.y = fma(f.y, v.x, acc.y);
  }
}

// f_g(k) of a group (see DGroup); returns the class of the value (0 real, 1 imag, 2 complex).
__device__ __forceinline__ int group_value(const DGroup& G, uint64_t k, const double2* tables,
                                           double2& f) {
  if (G.cls >= 4) {
    f = tables[G.toff];
    if (__popcll(k & G.zu) & 1) f = make_double2(dneg(f.x), dneg(f.y));
    return G.cls - 4;
  }
  f = tables[G.toff + pext64(k, G.zu)];
  return G.cls;
}

// ------------------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace svqe
