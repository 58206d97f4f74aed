/* Fused multiply-add for the CPU oracle (test infrastructure only).
 *
 * IEEE 754-2008 fusedMultiplyAdd: out[i] = a[i] * b[i] + c[i] computed exactly
 * and rounded once to nearest-even binary64.  C99's fma() is specified to do
 * exactly this (correctly rounded, no intermediate rounding), so the loop
 * below is the whole definition.  Compiled without -ffast-math and with
 * -ffp-contract=off so the compiler adds no other fused operations. */
#include <math.h>
#include <stdint.h>

void oracle_fma(const double* a, const double* b, const double* c, double* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = fma(a[i], b[i], c[i]);
}
