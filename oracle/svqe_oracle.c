/*
 * svqe_oracle.c -- plain, slow, obviously-correct CPU oracle for the VQE hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline / reference legs load this library.  It shares no code, header or constant
 * table with the CUDA library; both sides read the same instance arrays produced by the
 * seeded generator and nothing else.
 *
 * Paper: Malarchick & Steed, "Parallelizing the Variational Quantum Eigensolver: From JIT
 * Compilation to Multi-GPU Scaling" (2026).  What is computed, and where it is defined:
 *   |psi(theta)> = U(theta) |HF>              Sec. 3.3, Eq. 4 (reference state, ansatz)
 *   U = DoubleExcitation(theta)               Sec. 3.3, Eq. 5 (read as a real Givens rotation)
 *   E(theta) = <psi|H|psi>                    Sec. 3.1, Eq. 2
 *   H = sum_t c_t P_t  (Jordan-Wigner sum)    Sec. 3.2, Eq. 3
 *   dE/dtheta by parameter shift              Algorithm 1 (gradient step); Sec. 4.3
 * All arithmetic is IEEE binary64 (double / double complex), one gate at a time over the
 * whole vector, one Pauli term at a time, with no grouping, fusion or adjoint.
 *
 * Conventions (the paper is silent; these are the readings used on both sides):
 *   - qubit q is bit (n-1-q) of the basis index (qubit 0 is the most significant bit),
 *     so |1100> = 12;
 *   - Pauli masks are over basis-index bits; the term with masks (x, z) is
 *     P = i^{popc(x&z)} X^x Z^z, i.e. P|i> = i^{popc(x&z)} (-1)^{popc(z&i)} |i xor x>;
 *   - RX/RY/RZ(t) = exp(-i t/2 X/Y/Z);
 *   - SingleExcitation(t) on wires (a,b) rotates span{|01>,|10>}:
 *       |01> -> cos(t/2)|01> + sin(t/2)|10>,  |10> -> cos(t/2)|10> - sin(t/2)|01>;
 *     DoubleExcitation(t) on wires (a,b,c,d) rotates span{|0011>,|1100>} the same way;
 *   - gradient: two-term shift (+-pi/2) for RX/RY/RZ, whose generators have eigenvalues
 *     +-1/2; four-term shift (+-pi/2, +-3pi/2) for the excitation gates, whose generators
 *     have eigenvalues {-1/2, 0, +1/2} (two frequencies, 1/2 and 1).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Gate codes of the instance format (the same integers the generator writes). */
enum { ORC_X = 0, ORC_H = 1, ORC_RX = 2, ORC_RY = 3, ORC_RZ = 4, ORC_CNOT = 5,
       ORC_SINGLE_EXC = 6, ORC_DOUBLE_EXC = 7, ORC_CZ = 8 };

static int n_wires_of(int type) {
  switch (type) {
    case ORC_X: case ORC_H: case ORC_RX: case ORC_RY: case ORC_RZ: return 1;
    case ORC_CNOT: case ORC_SINGLE_EXC: case ORC_CZ: return 2;
    case ORC_DOUBLE_EXC: return 4;
    default: return -1;
  }
}

static int is_param_gate(int type) {
  return type == ORC_RX || type == ORC_RY || type == ORC_RZ ||
         type == ORC_SINGLE_EXC || type == ORC_DOUBLE_EXC;
}

/* Mask of basis-index bit for qubit q. */
static inline uint64_t bit_of(int n, int q) { return (uint64_t)1 << (n - 1 - q); }

/* Apply a 2x2 matrix [[u00,u01],[u10,u11]] to qubit q: for every index i whose bit is 0,
 * the pair (psi[i], psi[i | bit]) is (|0>, |1>) of that qubit. */
static void apply_1q(int n, double complex* psi, int q, double complex u00, double complex u01,
                     double complex u10, double complex u11) {
  const uint64_t N = (uint64_t)1 << n, b = bit_of(n, q);
  for (uint64_t i = 0; i < N; ++i) {
    if (i & b) continue;
    const double complex a0 = psi[i], a1 = psi[i | b];
    psi[i] = u00 * a0 + u01 * a1;
    psi[i | b] = u10 * a0 + u11 * a1;
  }
}

/* Real rotation by t/2 inside the two-dimensional span {|lo>, |hi>} selected by `pattern_lo`
 * (the bits of the wires that are 1 in the "from" pattern) inside `wmask` (all wires of the
 * gate):  |lo> -> c|lo> + s|hi>,  |hi> -> c|hi> - s|lo>.  All other amplitudes unchanged. */
static void apply_givens(int n, double complex* psi, uint64_t wmask, uint64_t pattern_lo,
                         double t) {
  const uint64_t N = (uint64_t)1 << n, flip = wmask;
  const double c = cos(0.5 * t), s = sin(0.5 * t);
  for (uint64_t i = 0; i < N; ++i) {
    if ((i & wmask) != pattern_lo) continue;
    const uint64_t j = i ^ flip;                 /* the |hi> partner */
    const double complex lo = psi[i], hi = psi[j];
    psi[i] = c * lo - s * hi;
    psi[j] = s * lo + c * hi;
  }
}

/* Apply one gate.  Returns 0, or -1 on a malformed record. */
int orc_apply_gate(int n, double complex* psi, int type, const int* w, double t) {
  const int k = n_wires_of(type);
  if (k < 0) return -1;
  for (int a = 0; a < k; ++a) {
    if (w[a] < 0 || w[a] >= n) return -1;
    for (int b = 0; b < a; ++b) if (w[a] == w[b]) return -1;
  }
  const double c = cos(0.5 * t), s = sin(0.5 * t);
  switch (type) {
    case ORC_X: apply_1q(n, psi, w[0], 0, 1, 1, 0); break;
    case ORC_H: { const double r = 1.0 / sqrt(2.0); apply_1q(n, psi, w[0], r, r, r, -r); } break;
    case ORC_RX: apply_1q(n, psi, w[0], c, -I * s, -I * s, c); break;
    case ORC_RY: apply_1q(n, psi, w[0], c, -s, s, c); break;
    case ORC_RZ: apply_1q(n, psi, w[0], cexp(-I * 0.5 * t), 0, 0, cexp(I * 0.5 * t)); break;
    case ORC_CNOT: {
      const uint64_t N = (uint64_t)1 << n, bc = bit_of(n, w[0]), bt = bit_of(n, w[1]);
      for (uint64_t i = 0; i < N; ++i) {
        if ((i & bc) && !(i & bt)) {
          const double complex tmp = psi[i]; psi[i] = psi[i | bt]; psi[i | bt] = tmp;
        }
      }
    } break;
    case ORC_CZ: {
      const uint64_t N = (uint64_t)1 << n, b0 = bit_of(n, w[0]), b1 = bit_of(n, w[1]);
      for (uint64_t i = 0; i < N; ++i) if ((i & b0) && (i & b1)) psi[i] = -psi[i];
    } break;
    case ORC_SINGLE_EXC: {
      /* span{|01>,|10>} on (w0, w1): "lo" pattern = w0 empty, w1 occupied. */
      const uint64_t m = bit_of(n, w[0]) | bit_of(n, w[1]);
      apply_givens(n, psi, m, bit_of(n, w[1]), t);
    } break;
    case ORC_DOUBLE_EXC: {
      /* span{|0011>,|1100>} on (w0..w3): "lo" pattern = w0,w1 empty, w2,w3 occupied. */
      const uint64_t m = bit_of(n, w[0]) | bit_of(n, w[1]) | bit_of(n, w[2]) | bit_of(n, w[3]);
      apply_givens(n, psi, m, bit_of(n, w[2]) | bit_of(n, w[3]), t);
    } break;
    default: return -1;
  }
  return 0;
}

/* psi = |b>  (Eq. 4: the reference state is a computational-basis product state). */
void orc_init_basis(int n, double complex* psi, uint64_t b) {
  const uint64_t N = (uint64_t)1 << n;
  for (uint64_t i = 0; i < N; ++i) psi[i] = 0;
  psi[b & (N - 1)] = 1;
}

/* Angle of gate g: theta[param] if the gate is parameterised, else its fixed angle; plus
 * `shift` when g == shift_gate (used by the parameter-shift rule). */
static double gate_angle(int g, const int* params, const double* fixed, const double* theta,
                         int shift_gate, double shift) {
  double t = params[g] >= 0 ? theta[params[g]] : fixed[g];
  if (g == shift_gate) t += shift;
  return t;
}

/* psi <- U_L ... U_1 psi, gates in list order. */
int orc_apply_circuit(int n, double complex* psi, int n_gates, const int* types, const int* wires,
                      const int* params, const double* fixed, const double* theta,
                      int shift_gate, double shift) {
  for (int g = 0; g < n_gates; ++g) {
    const double t = gate_angle(g, params, fixed, theta, shift_gate, shift);
    if (orc_apply_gate(n, psi, types[g], wires + 4 * g, t) != 0) return -1;
  }
  return 0;
}

/* Neumaier compensated sum, so that the oracle's own rounding stays far below the
 * tolerances it is used to check. */
typedef struct { double s, c; } nsum;
static inline void nsum_add(nsum* a, double v) {
  const double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v; else a->c += (v - t) + a->s;
  a->s = t;
}
static inline double nsum_get(const nsum* a) { return a->s + a->c; }

static int popcount64(uint64_t v) { return __builtin_popcountll(v); }

/* <psi|P|psi> for one Pauli string, summed over i of conj(psi[i^x]) * (P|i> coefficient) *
 * psi[i].  Sec. 3.2: H is a real-weighted sum of Pauli strings. */
static void pauli_expval(int n, const double complex* psi, uint64_t x, uint64_t z,
                         double* re, double* im) {
  const uint64_t N = (uint64_t)1 << n;
  static const double complex ipow[4] = {1, I, -1, -I};
  const double complex ph = ipow[popcount64(x & z) & 3];
  nsum sr = {0, 0}, si = {0, 0};
  for (uint64_t i = 0; i < N; ++i) {
    const double sign = (popcount64(z & i) & 1) ? -1.0 : 1.0;
    const double complex v = conj(psi[i ^ x]) * (ph * sign) * psi[i];
    nsum_add(&sr, creal(v));
    nsum_add(&si, cimag(v));
  }
  *re = nsum_get(&sr);
  *im = nsum_get(&si);
}

/* E = sum_t c_t <psi|P_t|psi>  (Eq. 2).  The imaginary part is returned too; it is zero up
 * to rounding for a Hermitian H and is checked, then discarded, by the caller. */
void orc_expval(int n, const double complex* psi, int n_terms, const uint64_t* x,
                const uint64_t* z, const double* coeff, double* e_re, double* e_im) {
  nsum er = {0, 0}, ei = {0, 0};
  for (int t = 0; t < n_terms; ++t) {
    double r, i;
    pauli_expval(n, psi, x[t], z[t], &r, &i);
    nsum_add(&er, coeff[t] * r);
    nsum_add(&ei, coeff[t] * i);
  }
  *e_re = nsum_get(&er);
  *e_im = nsum_get(&ei);
}

/* E(theta) with an optional shift of one gate's angle; `work` holds 2^n amplitudes. */
static int energy_into(int n, uint64_t ref, int n_gates, const int* types, const int* wires,
                       const int* params, const double* fixed, const double* theta,
                       int shift_gate, double shift, int n_terms, const uint64_t* x,
                       const uint64_t* z, const double* coeff, double complex* work,
                       double* e) {
  orc_init_basis(n, work, ref);
  if (orc_apply_circuit(n, work, n_gates, types, wires, params, fixed, theta, shift_gate,
                        shift) != 0)
    return -1;
  double im;
  orc_expval(n, work, n_terms, x, z, coeff, e, &im);
  return 0;
}

/* E(theta) = <ref| U^dag H U |ref>  (Eq. 2, Eq. 4). */
int orc_energy(int n, uint64_t ref, int n_gates, const int* types, const int* wires,
               const int* params, const double* fixed, const double* theta, int n_terms,
               const uint64_t* x, const uint64_t* z, const double* coeff, double* e) {
  double complex* work = (double complex*)malloc(sizeof(double complex) << n);
  if (!work) return -2;
  const int rc = energy_into(n, ref, n_gates, types, wires, params, fixed, theta, -1, 0.0,
                             n_terms, x, z, coeff, work, e);
  free(work);
  return rc;
}

static int g_threads = 1;
void orc_set_threads(int k) { g_threads = k > 0 ? k : 1; }
int orc_get_threads(void) { return g_threads; }

/* Energy and gradient.  The gradient is the parameter-shift rule (Algorithm 1's gradient
 * step; Sec. 4.3: two circuit evaluations per parameter for the rotation gates), applied to
 * every occurrence of a parameter and summed over occurrences:
 *   RX/RY/RZ:   dE/dt = [E(t+pi/2) - E(t-pi/2)] / 2
 *   excitation: dE/dt = d1 [E(t+pi/2) - E(t-pi/2)] - d2 [E(t+3pi/2) - E(t-3pi/2)],
 *               d1 = (sqrt2+1)/(4 sqrt2), d2 = (sqrt2-1)/(4 sqrt2),
 * the second being the shift rule for a generator with eigenvalues {-1/2, 0, 1/2}.  The
 * shifted energies are independent circuit evaluations; they run in parallel (one state
 * buffer per thread) and are summed afterwards in a fixed order. */
static int energy_grad_impl(int n, uint64_t ref, int n_gates, const int* types,
                            const int* wires, const int* params, const double* fixed,
                            const double* theta, int n_params, int n_terms, const uint64_t* x,
                            const uint64_t* z, const double* coeff, const char* want,
                            double* e, double* grad);

int orc_energy_grad(int n, uint64_t ref, int n_gates, const int* types, const int* wires,
                    const int* params, const double* fixed, const double* theta, int n_params,
                    int n_terms, const uint64_t* x, const uint64_t* z, const double* coeff,
                    double* e, double* grad) {
  return energy_grad_impl(n, ref, n_gates, types, wires, params, fixed, theta, n_params,
                          n_terms, x, z, coeff, NULL, e, grad);
}

/* As orc_energy_grad, for the parameters listed in `which` only (n_which entries); grad has
 * n_params entries, the others are left at zero.  Used to sample gradients of circuits too
 * large for the full parameter-shift sweep. */
int orc_energy_grad_subset(int n, uint64_t ref, int n_gates, const int* types, const int* wires,
                           const int* params, const double* fixed, const double* theta,
                           int n_params, int n_terms, const uint64_t* x, const uint64_t* z,
                           const double* coeff, const int* which, int n_which, double* e,
                           double* grad) {
  char* want = (char*)calloc(n_params > 0 ? n_params : 1, 1);
  if (!want) return -2;
  for (int k = 0; k < n_which; ++k)
    if (which[k] >= 0 && which[k] < n_params) want[which[k]] = 1;
  const int rc = energy_grad_impl(n, ref, n_gates, types, wires, params, fixed, theta, n_params,
                                  n_terms, x, z, coeff, want, e, grad);
  free(want);
  return rc;
}

static int energy_grad_impl(int n, uint64_t ref, int n_gates, const int* types,
                            const int* wires, const int* params, const double* fixed,
                            const double* theta, int n_params, int n_terms, const uint64_t* x,
                            const uint64_t* z, const double* coeff, const char* want,
                            double* e, double* grad) {
  const double PI = 3.14159265358979323846;
  const double d1 = (sqrt(2.0) + 1.0) / (4.0 * sqrt(2.0));
  const double d2 = (sqrt(2.0) - 1.0) / (4.0 * sqrt(2.0));
  int n_jobs = 1;  /* job 0: the unshifted energy */
  for (int g = 0; g < n_gates; ++g) {
    if (params[g] < 0 || !is_param_gate(types[g])) continue;
    if (params[g] >= n_params) return -1;
    if (want && !want[params[g]]) continue;
    n_jobs += (types[g] == ORC_SINGLE_EXC || types[g] == ORC_DOUBLE_EXC) ? 4 : 2;
  }
  int* jg = (int*)malloc(sizeof(int) * n_jobs);
  double* js = (double*)malloc(sizeof(double) * n_jobs);
  double* jw = (double*)malloc(sizeof(double) * n_jobs);
  double* je = (double*)malloc(sizeof(double) * n_jobs);
  if (!jg || !js || !jw || !je) { free(jg); free(js); free(jw); free(je); return -2; }
  int k = 0;
  jg[k] = -1; js[k] = 0; jw[k] = 0; ++k;
  for (int g = 0; g < n_gates; ++g) {
    if (params[g] < 0 || !is_param_gate(types[g])) continue;
    if (want && !want[params[g]]) continue;
    if (types[g] == ORC_SINGLE_EXC || types[g] == ORC_DOUBLE_EXC) {
      jg[k] = g; js[k] = +0.5 * PI; jw[k] = +d1; ++k;
      jg[k] = g; js[k] = -0.5 * PI; jw[k] = -d1; ++k;
      jg[k] = g; js[k] = +1.5 * PI; jw[k] = -d2; ++k;
      jg[k] = g; js[k] = -1.5 * PI; jw[k] = +d2; ++k;
    } else {
      jg[k] = g; js[k] = +0.5 * PI; jw[k] = +0.5; ++k;
      jg[k] = g; js[k] = -0.5 * PI; jw[k] = -0.5; ++k;
    }
  }
  int failed = 0;
#pragma omp parallel num_threads(g_threads) reduction(| : failed)
  {
    double complex* work = (double complex*)malloc(sizeof(double complex) << n);
    if (!work) failed = 1;
#pragma omp for schedule(dynamic, 1)
    for (int j = 0; j < n_jobs; ++j) {
      if (!work) continue;
      if (energy_into(n, ref, n_gates, types, wires, params, fixed, theta, jg[j], js[j],
                      n_terms, x, z, coeff, work, &je[j]) != 0)
        failed = 1;
    }
    free(work);
  }
  if (!failed) {
    *e = je[0];
    for (int p = 0; p < n_params; ++p) grad[p] = 0.0;
    for (int j = 1; j < n_jobs; ++j) grad[params[jg[j]]] += jw[j] * je[j];
  }
  free(jg); free(js); free(jw); free(je);
  return failed ? -1 : 0;
}

/* The final state U(theta)|ref>, written to `psi` (2^n amplitudes). */
int orc_state(int n, uint64_t ref, int n_gates, const int* types, const int* wires,
              const int* params, const double* fixed, const double* theta, double complex* psi) {
  orc_init_basis(n, psi, ref);
  return orc_apply_circuit(n, psi, n_gates, types, wires, params, fixed, theta, -1, 0.0);
}
