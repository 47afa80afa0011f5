// Diversity of a set of solutions (include/spg.h spg_diversity; Fig. 3 (c),
// (f) of the paper): the solutions within approximation ratio a_r of the
// best energy, taken in ascending (energy, lexicographic variables, index)
// order, each counted when it differs in more than N/2 variables from every
// one counted before it.  Host only.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <numeric>
#include <vector>

#include "spg.h"

extern "C" int spg_diversity(int32_t n, int32_t N, const int32_t* vars, const int64_t* energies, int64_t e_best,
                             double a_r, int32_t* count, int32_t* chosen) {
  if (n < 0 || N < 1 || !(a_r >= 0.0) || (n > 0 && (!vars || !energies))) return SPG_EINVAL;
  // E - E_best < 2 a_r |E_best| (the printed test read with |E_best|)
  const double bound = 2.0 * a_r * std::fabs((double)e_best);
  std::vector<int32_t> order;
  for (int32_t k = 0; k < n; ++k)
    if ((double)(energies[k] - e_best) < bound) order.push_back(k);
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (energies[a] != energies[b]) return energies[a] < energies[b];
    const int32_t *va = vars + (size_t)a * N, *vb = vars + (size_t)b * N;
    if (!std::equal(va, va + N, vb)) return std::lexicographical_compare(va, va + N, vb, vb + N);
    return a < b;  // a solution given twice: the first copy first
  });
  std::vector<int32_t> picked;
  for (int32_t k : order) {
    const int32_t* vk = vars + (size_t)k * N;
    bool far = true;
    for (int32_t c : picked) {
      const int32_t* vc = vars + (size_t)c * N;
      int32_t d = 0;
      for (int32_t q = 0; q < N; ++q) d += vk[q] != vc[q];
      if (2 * (int64_t)d <= N) {
        far = false;
        break;
      }
    }
    if (far) picked.push_back(k);
  }
  if (count) *count = (int32_t)picked.size();
  if (chosen) std::copy(picked.begin(), picked.end(), chosen);
  return SPG_OK;
}
