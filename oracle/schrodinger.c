/*
 * Plain FP64 Schroedinger-style simulation in C (oracle O1, Sec. II-A and Example 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check, the scripts that write
 * stored expected values under tests/golden/ and the CPU-baseline leg of the benchmark
 * may load this library.  It shares no code, header or table with the CUDA path.
 *
 * What it computes: psi = G_T ... G_2 G_1 |0...0> on the full 2^n statevector, one gate
 * at a time, by the definition of a gate acting on a subset of the qubits: for every
 * assignment of the qubits the gate does not touch, the 2^k amplitudes that differ only
 * on the gate's k qubits are multiplied by the gate's 2^k x 2^k matrix.  No fusion, no
 * reordering, no special cases for diagonal gates.
 *
 * Conventions (Sec. II-A): bit q of a basis index is qubit q; a gate on the ordered
 * qubits (q[0], q[1], ...) has its matrix row/column index in Kronecker order with q[0]
 * the most significant factor (so CNOT with the control listed first is
 * P0 (x) I + P1 (x) X, Example 2).  Matrices are row-major complex128, re/im interleaved.
 *
 * The loop over the untouched qubits runs in parallel with OpenMP; every iteration
 * reads and writes its own 2^k amplitudes, so the result does not depend on the thread
 * count.
 */
#include <stdint.h>
#include <stdlib.h>

#define MAXQ 4

/* Insert a zero bit at each of the k positions in pos (ascending) into t. */
static uint64_t spread(uint64_t t, const int *pos_sorted, int k) {
  for (int j = 0; j < k; ++j) {
    const int p = pos_sorted[j];
    const uint64_t low = t & ((1ull << p) - 1ull);
    t = ((t >> p) << (p + 1)) | low;
  }
  return t;
}

/* psi <- (M on qubits q[0..k)) psi for one gate. */
static void apply_gate(double *psi, int n, int k, const int *q, const double *m) {
  const int dim = 1 << k;
  int sorted[MAXQ];
  for (int j = 0; j < k; ++j) sorted[j] = q[j];
  for (int a = 1; a < k; ++a)               /* insertion sort, ascending */
    for (int b = a; b > 0 && sorted[b - 1] > sorted[b]; --b) {
      const int t = sorted[b];
      sorted[b] = sorted[b - 1];
      sorted[b - 1] = t;
    }
  /* offset of matrix index s: qubit q[x] carries bit (k-1-x) of s */
  uint64_t off[1 << MAXQ];
  for (int s = 0; s < dim; ++s) {
    uint64_t o = 0;
    for (int x = 0; x < k; ++x)
      if ((s >> (k - 1 - x)) & 1) o |= 1ull << q[x];
    off[s] = o;
  }
  const int64_t bases = (int64_t)1 << (n - k);
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < bases; ++t) {
    const uint64_t base = spread((uint64_t)t, sorted, k);
    double in_re[1 << MAXQ], in_im[1 << MAXQ];
    for (int s = 0; s < dim; ++s) {
      in_re[s] = psi[2 * (base | off[s])];
      in_im[s] = psi[2 * (base | off[s]) + 1];
    }
    for (int r = 0; r < dim; ++r) {
      double re = 0.0, im = 0.0;
      for (int s = 0; s < dim; ++s) {
        const double mr = m[2 * (r * dim + s)], mi = m[2 * (r * dim + s) + 1];
        re += mr * in_re[s] - mi * in_im[s];
        im += mr * in_im[s] + mi * in_re[s];
      }
      psi[2 * (base | off[r])] = re;
      psi[2 * (base | off[r]) + 1] = im;
    }
  }
}

/*
 * oracle_schrodinger: psi (2^n complex128, caller-owned) <- the circuit applied to
 * |0...0>.  Gate g acts on nq[g] qubits qubits[4g .. 4g+nq[g]) with the matrix at
 * mats + 2 * mat_off[g] (complex elements, row-major).  Returns 0, or -1 for bad input.
 */
int oracle_schrodinger(int n, int num_gates, const int32_t *nq, const int32_t *qubits,
                       const double *mats, const int64_t *mat_off, double *psi) {
  if (n < 1 || n > 40 || num_gates < 0 || !psi) return -1;
  for (int g = 0; g < num_gates; ++g) {
    if (nq[g] < 1 || nq[g] > MAXQ) return -1;
    for (int x = 0; x < nq[g]; ++x) {
      const int qx = qubits[4 * g + x];
      if (qx < 0 || qx >= n) return -1;
      for (int y = 0; y < x; ++y)
        if (qubits[4 * g + y] == qx) return -1;
    }
  }
  const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < 2 * dim; ++i) psi[i] = 0.0;
  psi[0] = 1.0;
  for (int g = 0; g < num_gates; ++g)
    apply_gate(psi, n, nq[g], qubits + 4 * g, mats + 2 * mat_off[g]);
  return 0;
}

/* Apply gates [g0, g1) of the same description to an existing state (CPU-baseline timing
 * of a bounded sample of a circuit). */
int oracle_apply_gates(int n, int g0, int g1, const int32_t *nq, const int32_t *qubits,
                       const double *mats, const int64_t *mat_off, double *psi) {
  if (n < 1 || n > 40 || g0 < 0 || g1 < g0 || !psi) return -1;
  for (int g = g0; g < g1; ++g) {
    if (nq[g] < 1 || nq[g] > MAXQ) return -1;
    apply_gate(psi, n, nq[g], qubits + 4 * g, mats + 2 * mat_off[g]);
  }
  return 0;
}
