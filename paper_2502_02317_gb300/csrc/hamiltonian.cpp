// Clustered Hamiltonian on the host (include/spg.h spg_potts_hamiltonian):
// Sec. 2 of the paper, Eq. 2 -> Eq. 1 (spins grouped into clusters on a grid
// of cells, every cluster a Potts variable over all its 2^k states), with the
// pairwise interaction of two clusters reduced to its distinct rows and
// columns through projectors (Sec. 3.1 Sparsity).  For the large clusters of
// Sec. 3.1.1 (Pegasus 24 spins, Zephyr 16) the d_m x d_n table of an edge is
// never formed: it is a function of the configurations of the spins its
// couplers touch, E_e[x, y] = T[a(x)][b(y)], every configuration occurs, so
// rows of E_e are equal exactly when rows of T are, and the first state with
// configuration a (only a's spins set) grows with a; the reduced table and
// the projectors, first-occurrence order included, are computed over the
// configurations and read off for every state.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "spg.h"

struct spg_hamiltonian {
  int rows = 0, cols = 0, shift = 0;
  std::vector<int> k;                      // spins per site
  std::vector<std::vector<int64_t>> E;     // local tables
  struct Edge {
    int m = 0, n = 0, Dm = 0, Dn = 0;
    std::vector<int64_t> R;
    std::vector<int32_t> Pm, Pn;
    std::vector<int> Sm, Sn;               // positions of the coupled spins in m and n
    std::vector<int64_t> T;                // energy over their configurations [2^|Sm|][2^|Sn|]
  };
  std::vector<Edge> edges;
  std::map<std::pair<int, int>, int> edge_of;  // (m, n) -> index in edges
};

namespace {

// Configuration index of the spins at positions S (ascending) in state x.
inline int64_t sub_of(int64_t x, const std::vector<int>& S) {
  int64_t a = 0;
  for (size_t q = 0; q < S.size(); ++q) a |= ((x >> S[q]) & 1) << q;
  return a;
}

// First-occurrence classes of the rows of T [na][nb] (row-major); returns
// the class of every row and the first row of every class.
void classes_of_rows(const std::vector<int64_t>& T, int64_t na, int64_t nb, std::vector<int32_t>& cls,
                     std::vector<int64_t>& first) {
  std::map<std::vector<int64_t>, int32_t> index;
  cls.assign((size_t)na, 0);
  first.clear();
  for (int64_t a = 0; a < na; ++a) {
    std::vector<int64_t> row(T.begin() + a * nb, T.begin() + (a + 1) * nb);
    auto it = index.find(row);
    if (it == index.end()) {
      it = index.emplace(std::move(row), (int32_t)first.size()).first;
      first.push_back(a);
    }
    cls[(size_t)a] = it->second;
  }
}

bool on_grid(double v, double scale, int64_t* out) {
  const double x = v * scale;
  if (!std::isfinite(x) || std::rint(x) != x || std::fabs(x) >= 4503599627370496.0) return false;
  *out = (int64_t)x;
  return true;
}

}  // namespace

extern "C" int spg_potts_hamiltonian(int32_t n_spins, int32_t n_edges, const int32_t* ei, const int32_t* ej,
                                     const double* J, const double* h, const int32_t* cluster_of_spin,
                                     int32_t grid_rows, int32_t grid_cols, const int32_t* cluster_row,
                                     const int32_t* cluster_col, int32_t energy_shift, int32_t node_type,
                                     spg_hamiltonian** out) {
  if (!out) return SPG_EINVAL;
  *out = nullptr;
  if (n_spins <= 0 || n_edges < 0 || grid_rows <= 0 || grid_cols <= 0 || !cluster_of_spin || !cluster_row ||
      !cluster_col || (n_edges > 0 && (!ei || !ej || !J)))
    return SPG_EINVAL;
  if (energy_shift < 0 || energy_shift > 52 || (node_type != SPG_SQUARE && node_type != SPG_KING)) return SPG_EINVAL;
  if ((int64_t)grid_rows * grid_cols > (1 << 24)) return SPG_EUNSUPPORTED;
  const int n = grid_rows * grid_cols;
  const double scale = std::ldexp(1.0, energy_shift);
  spg_hamiltonian* H = new (std::nothrow) spg_hamiltonian();
  if (!H) return SPG_ENOMEM;
  int rc = SPG_OK;
  try {
    std::vector<int> site_of_cluster(n, -1), used(n, 0);
    for (int c = 0; c < n && rc == SPG_OK; ++c) {
      const int r = cluster_row[c], cc = cluster_col[c];
      if (r < 0 || r >= grid_rows || cc < 0 || cc >= grid_cols || used[r * grid_cols + cc]) {
        rc = SPG_EINVAL;
        break;
      }
      used[r * grid_cols + cc] = 1;
      site_of_cluster[c] = r * grid_cols + cc;
    }
    std::vector<int> site_of_spin(n_spins), pos(n_spins);
    std::vector<std::vector<int>> spins(n);
    for (int i = 0; i < n_spins && rc == SPG_OK; ++i) {
      const int c = cluster_of_spin[i];
      if (c < 0 || c >= n) {
        rc = SPG_EINVAL;
        break;
      }
      site_of_spin[i] = site_of_cluster[c];
      pos[i] = (int)spins[site_of_spin[i]].size();  // spins visited in ascending index
      spins[site_of_spin[i]].push_back(i);
    }
    H->rows = grid_rows;
    H->cols = grid_cols;
    H->shift = energy_shift;
    H->k.resize(n);
    H->E.resize(n);
    for (int s = 0; s < n && rc == SPG_OK; ++s) {
      H->k[s] = (int)spins[s].size();
      if (H->k[s] > SPG_MAX_HAMILTONIAN_SPINS) rc = SPG_EUNSUPPORTED;
      else H->E[s].assign((size_t)1 << H->k[s], 0);
    }
    auto spin = [](int64_t x, int q) -> int64_t { return ((x >> q) & 1) ? 1 : -1; };
    for (int i = 0; i < n_spins && rc == SPG_OK && h; ++i) {
      int64_t hv = 0;
      if (!on_grid(h[i], scale, &hv)) {
        rc = SPG_EINEXACT;
        break;
      }
      std::vector<int64_t>& E = H->E[site_of_spin[i]];
      if (hv != 0)
        for (int64_t x = 0; x < (int64_t)E.size(); ++x) E[x] += hv * spin(x, pos[i]);
    }
    struct Coupler {
      int pa, pb;
      int64_t J;
    };
    std::map<std::pair<int, int>, std::vector<Coupler>> inter;  // ascending (m, n)
    for (int e = 0; e < n_edges && rc == SPG_OK; ++e) {
      const int a = ei[e], b = ej[e];
      int64_t Jv = 0;
      if (a < 0 || a >= n_spins || b < 0 || b >= n_spins || a == b) {
        rc = SPG_EINVAL;
        break;
      }
      if (!on_grid(J[e], scale, &Jv)) {
        rc = SPG_EINEXACT;
        break;
      }
      int sa = site_of_spin[a], sb = site_of_spin[b], pa = pos[a], pb = pos[b];
      if (sa == sb) {
        std::vector<int64_t>& E = H->E[sa];
        for (int64_t x = 0; x < (int64_t)E.size(); ++x) E[x] += Jv * spin(x, pa) * spin(x, pb);
        continue;
      }
      if (sa > sb) {
        std::swap(sa, sb);
        std::swap(pa, pb);
      }
      const int dr = std::abs(sa / grid_cols - sb / grid_cols), dc = std::abs(sa % grid_cols - sb % grid_cols);
      if (!(node_type == SPG_SQUARE ? (dr + dc == 1) : (std::max(dr, dc) == 1))) {
        rc = SPG_EINVAL;
        break;
      }
      inter[{sa, sb}].push_back({pa, pb, Jv});
    }
    for (auto it = inter.begin(); it != inter.end() && rc == SPG_OK; ++it) {
      std::vector<int> Sm, Sn;
      for (const Coupler& c : it->second) {
        Sm.push_back(c.pa);
        Sn.push_back(c.pb);
      }
      std::sort(Sm.begin(), Sm.end());
      Sm.erase(std::unique(Sm.begin(), Sm.end()), Sm.end());
      std::sort(Sn.begin(), Sn.end());
      Sn.erase(std::unique(Sn.begin(), Sn.end()), Sn.end());
      if ((int)Sm.size() > SPG_MAX_HAMILTONIAN_COUPLED || (int)Sn.size() > SPG_MAX_HAMILTONIAN_COUPLED) {
        rc = SPG_EUNSUPPORTED;
        break;
      }
      const int64_t na = (int64_t)1 << Sm.size(), nb = (int64_t)1 << Sn.size();
      // the edge's energy over the configurations (a, b) of its coupled spins
      std::vector<int64_t> T((size_t)(na * nb), 0), Tt((size_t)(na * nb));
      for (const Coupler& c : it->second) {
        const int qa = (int)(std::lower_bound(Sm.begin(), Sm.end(), c.pa) - Sm.begin());
        const int qb = (int)(std::lower_bound(Sn.begin(), Sn.end(), c.pb) - Sn.begin());
        for (int64_t a = 0; a < na; ++a)
          for (int64_t b = 0; b < nb; ++b) T[a * nb + b] += c.J * spin(a, qa) * spin(b, qb);
      }
      for (int64_t a = 0; a < na; ++a)
        for (int64_t b = 0; b < nb; ++b) Tt[b * na + a] = T[a * nb + b];
      std::vector<int32_t> cm, cn;
      std::vector<int64_t> fa, fb;
      classes_of_rows(T, na, nb, cm, fa);
      classes_of_rows(Tt, nb, na, cn, fb);
      spg_hamiltonian::Edge e;
      e.m = it->first.first;
      e.n = it->first.second;
      e.Dm = (int)fa.size();
      e.Dn = (int)fb.size();
      e.R.resize((size_t)e.Dm * e.Dn);
      for (int i = 0; i < e.Dm; ++i)
        for (int j = 0; j < e.Dn; ++j) e.R[(size_t)i * e.Dn + j] = T[fa[i] * nb + fb[j]];
      e.Pm.resize(H->E[e.m].size());
      e.Pn.resize(H->E[e.n].size());
      for (int64_t x = 0; x < (int64_t)e.Pm.size(); ++x) e.Pm[x] = cm[sub_of(x, Sm)];
      for (int64_t y = 0; y < (int64_t)e.Pn.size(); ++y) e.Pn[y] = cn[sub_of(y, Sn)];
      e.Sm = Sm;
      e.Sn = Sn;
      e.T.swap(T);
      H->edge_of[{e.m, e.n}] = (int)H->edges.size();
      H->edges.push_back(std::move(e));
    }
  } catch (const std::bad_alloc&) {
    rc = SPG_ENOMEM;
  }
  if (rc != SPG_OK) {
    delete H;
    return rc;
  }
  *out = H;
  return SPG_OK;
}

extern "C" int spg_hamiltonian_size(const spg_hamiltonian* H, int32_t* n_sites, int32_t* n_edges) {
  if (!H) return SPG_EINVAL;
  if (n_sites) *n_sites = (int32_t)H->E.size();
  if (n_edges) *n_edges = (int32_t)H->edges.size();
  return SPG_OK;
}

extern "C" int spg_hamiltonian_local(const spg_hamiltonian* H, int32_t site, int64_t* n_states, int64_t* E) {
  if (!H || site < 0 || site >= (int32_t)H->E.size()) return SPG_EINVAL;
  const std::vector<int64_t>& v = H->E[site];
  if (n_states) *n_states = (int64_t)v.size();
  if (E) std::memcpy(E, v.data(), sizeof(int64_t) * v.size());
  return SPG_OK;
}

extern "C" int spg_hamiltonian_edge(const spg_hamiltonian* H, int32_t k, int32_t* m, int32_t* n, int32_t* Dm,
                                    int32_t* Dn, int64_t* R, int32_t* Pm, int32_t* Pn) {
  if (!H || k < 0 || k >= (int32_t)H->edges.size()) return SPG_EINVAL;
  const spg_hamiltonian::Edge& e = H->edges[k];
  if (m) *m = e.m;
  if (n) *n = e.n;
  if (Dm) *Dm = e.Dm;
  if (Dn) *Dn = e.Dn;
  if (R) std::memcpy(R, e.R.data(), sizeof(int64_t) * e.R.size());
  if (Pm) std::memcpy(Pm, e.Pm.data(), sizeof(int32_t) * e.Pm.size());
  if (Pn) std::memcpy(Pn, e.Pn.data(), sizeof(int32_t) * e.Pn.size());
  return SPG_OK;
}

extern "C" void spg_hamiltonian_destroy(spg_hamiltonian* H) { delete H; }

namespace {

// Joint projection `which` of site s (include/spg.h spg_hamiltonian_classes):
// the class of every state and the first state of every class.  The key of
// an interface configuration c (the spins coupled by the projection's edges,
// ascending) is the tuple of its rows of the edges' configuration tables;
// classes in order of c ascending, which is the order of first occurrence
// over the states (the first state carrying c grows with c).
int site_classes(const spg_hamiltonian* H, int s, int which, std::vector<int32_t>& P, std::vector<int32_t>& reps) {
  const int cols = H->cols, rows = H->rows, i = s / cols, j = s % cols;
  auto at = [&](int ii, int jj) { return (ii >= 0 && ii < rows && jj >= 0 && jj < cols) ? ii * cols + jj : -1; };
  std::vector<int> nb;
  switch (which) {
    case SPG_CLASS_L: nb = {at(i, j - 1), at(i - 1, j - 1)}; break;
    case SPG_CLASS_U: nb = {at(i - 1, j)}; break;
    case SPG_CLASS_R: nb = {at(i, j + 1), at(i - 1, j + 1)}; break;
    case SPG_CLASS_D: nb = {at(i + 1, j - 1), at(i + 1, j), at(i + 1, j + 1)}; break;
    case SPG_CLASS_G: nb = {at(i + 1, j + 1)}; break;
    default: return SPG_EINVAL;
  }
  struct Part {
    const spg_hamiltonian::Edge* e;
    bool row;  // s is the edge's row variable (m)
  };
  std::vector<Part> parts;
  std::vector<int> U;
  for (int t : nb) {
    if (t < 0) continue;
    auto it = H->edge_of.find({std::min(s, t), std::max(s, t)});
    if (it == H->edge_of.end()) continue;
    const spg_hamiltonian::Edge& e = H->edges[it->second];
    parts.push_back({&e, s == e.m});
    const std::vector<int>& S = s == e.m ? e.Sm : e.Sn;
    U.insert(U.end(), S.begin(), S.end());
  }
  std::sort(U.begin(), U.end());
  U.erase(std::unique(U.begin(), U.end()), U.end());
  if (U.size() > 20) return SPG_EUNSUPPORTED;
  const int64_t nc = (int64_t)1 << U.size();
  int64_t key_len = 0;  // entries of one configuration's key
  for (const Part& p : parts) key_len += (int64_t)1 << (p.row ? p.e->Sn.size() : p.e->Sm.size());
  if (nc * std::max<int64_t>(key_len, 1) > ((int64_t)1 << 24)) return SPG_EUNSUPPORTED;  // keys beyond 128 MB
  std::vector<int32_t> cls((size_t)nc);
  std::vector<int64_t> first;
  std::map<std::vector<int64_t>, int32_t> index;
  for (int64_t c = 0; c < nc; ++c) {
    int64_t x = 0;  // the first state carrying configuration c
    for (size_t q = 0; q < U.size(); ++q) x |= ((c >> q) & 1) << U[q];
    std::vector<int64_t> key;
    for (const Part& p : parts) {
      const spg_hamiltonian::Edge& e = *p.e;
      const int64_t na = (int64_t)1 << e.Sm.size(), nbb = (int64_t)1 << e.Sn.size();
      if (p.row) {
        const int64_t a = sub_of(x, e.Sm);
        key.insert(key.end(), e.T.begin() + a * nbb, e.T.begin() + (a + 1) * nbb);
      } else {
        const int64_t b = sub_of(x, e.Sn);
        for (int64_t a = 0; a < na; ++a) key.push_back(e.T[a * nbb + b]);
      }
    }
    auto it = index.find(key);
    if (it == index.end()) {
      it = index.emplace(std::move(key), (int32_t)first.size()).first;
      first.push_back(x);
    }
    cls[(size_t)c] = it->second;
  }
  const int64_t d = (int64_t)H->E[s].size();
  P.resize((size_t)d);
  for (int64_t x = 0; x < d; ++x) P[(size_t)x] = cls[(size_t)sub_of(x, U)];
  reps.assign(first.begin(), first.end());
  return SPG_OK;
}

}  // namespace

extern "C" int spg_hamiltonian_classes(const spg_hamiltonian* H, int32_t site, int32_t which, int32_t* n_classes,
                                       int32_t* P, int32_t* reps) {
  if (!H || site < 0 || site >= (int32_t)H->E.size()) return SPG_EINVAL;
  std::vector<int32_t> Pv, rv;
  try {
    const int rc = site_classes(H, site, which, Pv, rv);
    if (rc != SPG_OK) return rc;
  } catch (const std::bad_alloc&) {
    return SPG_ENOMEM;
  }
  if (n_classes) *n_classes = (int32_t)rv.size();
  if (P) std::memcpy(P, Pv.data(), sizeof(int32_t) * Pv.size());
  if (reps) std::memcpy(reps, rv.data(), sizeof(int32_t) * rv.size());
  return SPG_OK;
}

extern "C" int spg_hamiltonian_class_weights(const spg_hamiltonian* H, int32_t site, double beta, double* C) {
  if (!H || site < 0 || site >= (int32_t)H->E.size() || !C || !(beta > 0.0)) return SPG_EINVAL;
  try {
    std::vector<int32_t> P[4], reps;
    for (int w = 0; w < 4; ++w) {
      const int rc = site_classes(H, site, w, P[w], reps);
      if (rc != SPG_OK) return rc;
    }
    int64_t N[4];
    for (int w = 0; w < 4; ++w) N[w] = 1 + *std::max_element(P[w].begin(), P[w].end());
    const std::vector<int64_t>& E = H->E[site];
    const int64_t mn = *std::min_element(E.begin(), E.end());
    const double bu = beta * std::ldexp(1.0, -H->shift);
    std::fill(C, C + N[0] * N[1] * N[2] * N[3], 0.0);
    for (size_t x = 0; x < E.size(); ++x)
      C[((P[0][x] * N[1] + P[1][x]) * N[2] + P[2][x]) * N[3] + P[3][x]] += std::exp(-bu * (double)(E[x] - mn));
  } catch (const std::bad_alloc&) {
    return SPG_ENOMEM;
  }
  return SPG_OK;
}

namespace {

const spg_hamiltonian::Edge* edge_between(const spg_hamiltonian* H, int s, int t) {
  if (s < 0 || t < 0) return nullptr;
  auto it = H->edge_of.find({std::min(s, t), std::max(s, t)});
  return it == H->edge_of.end() ? nullptr : &H->edges[it->second];
}

// Boltzmann factors exp(-bu (E_e[xs][xt] - min E_e)) of the edge between s
// and t (seen from s) at the states rs x rt; ones without an edge.
std::vector<double> boltz(const spg_hamiltonian* H, int s, int t, const std::vector<int32_t>& rs,
                          const std::vector<int32_t>& rt, double bu) {
  std::vector<double> out(rs.size() * rt.size(), 1.0);
  const spg_hamiltonian::Edge* e = edge_between(H, s, t);
  if (!e) return out;
  const int64_t nb = (int64_t)1 << e->Sn.size();
  const int64_t mn = *std::min_element(e->T.begin(), e->T.end());
  for (size_t a = 0; a < rs.size(); ++a)
    for (size_t b = 0; b < rt.size(); ++b) {
      const int64_t xm = s == e->m ? rs[a] : rt[b], xn = s == e->m ? rt[b] : rs[a];
      const int64_t v = e->T[sub_of(xm, e->Sm) * nb + sub_of(xn, e->Sn)];
      out[a * rt.size() + b] = std::exp(-bu * (double)(v - mn));
    }
  return out;
}

}  // namespace

extern "C" int spg_hamiltonian_site_tensor(const spg_hamiltonian* H, int32_t site, double beta, int32_t* dims,
                                           double* W) {
  if (!H || site < 0 || site >= (int32_t)H->E.size() || !(beta > 0.0)) return SPG_EINVAL;
  try {
    const int cols = H->cols, rows = H->rows, i = site / cols, j = site % cols;
    auto at = [&](int ii, int jj) { return (ii >= 0 && ii < rows && jj >= 0 && jj < cols) ? ii * cols + jj : -1; };
    const int left = at(i, j - 1), upleft = at(i - 1, j - 1), up = at(i - 1, j);
    const double bu = beta * std::ldexp(1.0, -H->shift);
    std::vector<int32_t> P[4], rep[4], tmp, repRl{0}, repGul{0}, repDu{0}, PGu, repGu{0};
    for (int w = 0; w < 4; ++w) {
      const int rc = site_classes(H, site, w, P[w], rep[w]);
      if (rc != SPG_OK) return rc;
    }
    int rc = SPG_OK;
    if (left >= 0 && (rc = site_classes(H, left, SPG_CLASS_R, tmp, repRl)) != SPG_OK) return rc;
    if (upleft >= 0 && (rc = site_classes(H, upleft, SPG_CLASS_G, tmp, repGul)) != SPG_OK) return rc;
    if (up >= 0 && (rc = site_classes(H, up, SPG_CLASS_D, tmp, repDu)) != SPG_OK) return rc;
    if (up >= 0 && (rc = site_classes(H, up, SPG_CLASS_G, PGu, repGu)) != SPG_OK) return rc;
    const int NL = (int)rep[0].size(), NU = (int)rep[1].size(), NR = (int)rep[2].size(), ND = (int)rep[3].size();
    const int NRl = (int)repRl.size(), Gin = (int)repGul.size(), DU = (int)repDu.size(), Gout = (int)repGu.size();
    const int DL = NRl * Gin, DR = NR * Gout;
    // the sums cost DL DU NR ND NL NU multiply-adds
    if ((double)DL * DU * NR * ND * NL * NU > 4e9) return SPG_EUNSUPPORTED;
    if (dims) {
      dims[0] = DL;
      dims[1] = DR;
      dims[2] = DU;
      dims[3] = ND;
    }
    if (!W) return SPG_OK;
    const std::vector<double> bh = boltz(H, left, site, repRl, rep[0], bu);     // [NRl][NL]
    const std::vector<double> bd = boltz(H, upleft, site, repGul, rep[0], bu);  // [Gin][NL]
    const std::vector<double> bup = boltz(H, up, site, repDu, rep[1], bu);      // [DU][NU]
    const std::vector<double> bad = boltz(H, up, left, repDu, repRl, bu);       // [DU][NRl]
    std::vector<double> C((size_t)NL * NU * NR * ND);
    if ((rc = spg_hamiltonian_class_weights(H, site, beta, C.data())) != SPG_OK) return rc;
    std::fill(W, W + (size_t)DL * DR * DU * ND, 0.0);
    for (int l = 0; l < DL; ++l) {
      const int a = l / Gin, g = l % Gin;
      for (int u = 0; u < DU; ++u) {
        const int gu = up >= 0 ? PGu[repDu[u]] : 0;
        const double f = bad[(size_t)u * NRl + a];
        for (int ap = 0; ap < NR; ++ap)
          for (int d = 0; d < ND; ++d) {
            double acc = 0.0;
            for (int h = 0; h < NL; ++h)
              for (int v = 0; v < NU; ++v)
                acc += bh[(size_t)a * NL + h] * bd[(size_t)g * NL + h] * bup[(size_t)u * NU + v] *
                       C[(((size_t)h * NU + v) * NR + ap) * ND + d];
            W[(((size_t)l * DR + ap * Gout + gu) * DU + u) * ND + d] = f * acc;
          }
      }
    }
  } catch (const std::bad_alloc&) {
    return SPG_ENOMEM;
  }
  return SPG_OK;
}
