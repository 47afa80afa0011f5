/* Brute force over every spin configuration of an Ising instance (Eq. 2 of
 * the paper), in plain C with OpenMP across the host's cores.
 *
 * Test infrastructure only: part of the FP64 CPU oracle, never linked into
 * the library.  For every configuration index c (bit i = spin i, s = 2b - 1)
 * the energy E = sum_e J_e s_i s_j + sum_i h_i s_i is evaluated directly
 * (integers in units of 2^-shift).  Two passes: the ground energy, then the
 * degeneracy and Z' = sum_c exp(-beta_u (E_c - E_min)) (every term <= 1),
 * giving log Z = -beta_u E_min + log Z'.  Returns 0, or -1 for n outside
 * 1..30. */
#include <math.h>
#include <stdint.h>

static int64_t energy_of(uint64_t c, int m, const int32_t* ei, const int32_t* ej, const int64_t* J, int n,
                         const int64_t* h) {
  int64_t E = 0;
  for (int e = 0; e < m; ++e) {
    const int64_t si = ((c >> ei[e]) & 1u) ? 1 : -1, sj = ((c >> ej[e]) & 1u) ? 1 : -1;
    E += J[e] * si * sj;
  }
  for (int i = 0; i < n; ++i) E += h[i] * (((c >> i) & 1u) ? 1 : -1);
  return E;
}

int oracle_brute_force(int n, int m, const int32_t* ei, const int32_t* ej, const int64_t* J, const int64_t* h,
                       double beta_u, int64_t* emin_out, int64_t* degeneracy_out, double* logz_out) {
  if (n < 1 || n > 30) return -1;
  const int64_t total = (int64_t)1 << n;
  int64_t emin = INT64_MAX;
#pragma omp parallel for reduction(min : emin) schedule(static)
  for (int64_t c = 0; c < total; ++c) {
    const int64_t E = energy_of((uint64_t)c, m, ei, ej, J, n, h);
    if (E < emin) emin = E;
  }
  int64_t deg = 0;
  double z = 0.0;
#pragma omp parallel for reduction(+ : deg, z) schedule(static)
  for (int64_t c = 0; c < total; ++c) {
    const int64_t E = energy_of((uint64_t)c, m, ei, ej, J, n, h);
    if (E == emin) ++deg;
    z += exp(-beta_u * (double)(E - emin));
  }
  *emin_out = emin;
  *degeneracy_out = deg;
  *logz_out = -beta_u * (double)emin + log(z);
  return 0;
}
