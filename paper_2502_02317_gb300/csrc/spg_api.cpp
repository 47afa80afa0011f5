// C ABI of libspg (include/spg.h): problem construction (S1: cluster factor
// graph, integer local and pairwise tables, projectors), the device
// workspace, and the orchestration of the boundary-MPS (S2-S4) and search
// (S5-S8) kernels.
//
// Paper: Eq. 1 and Eq. 2 (generalised Potts and Ising energies), Sec. 2
// (clusters of spins as Potts variables; PEPS of the Boltzmann distribution;
// branch and bound with merging), Sec. 3.1 (the solver's parameters).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/spg.h"
#include "spg_internal.h"

using namespace spg;

// The worker streams of spg_solve_batch need as many hardware work queues as
// there are streams in flight; CUDA gives a process 8 unless
// CUDA_DEVICE_MAX_CONNECTIONS asks for more (up to 32), and streams beyond
// the queue count share a queue and run one after another.  The variable is
// read when the process creates its CUDA context, so it is set (unless the
// user set it) when the library is loaded.
__attribute__((constructor)) static void spg_default_connections() {
  setenv("CUDA_DEVICE_MAX_CONNECTIONS", "32", 0);
}

struct spg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  // grow-only device arena, bump-allocated per solve
  char* arena = nullptr;
  size_t arena_bytes = 0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  // worker contexts (own stream and workspace) of spg_solve_batch
  std::vector<spg_ctx*> workers;
  // captured solves (see solve_impl)
  struct Graph {
    const void* problem = nullptr;
    spg_params prm{};
    int tsize = 0;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    int uses = 0;
    int group_n = 1;  // instances of the lockstep group (P: instance 0's problem)
    cudaGraphExec_t exec = nullptr;  // the whole solve, one launch
    long long launches = 0;
  };
  std::vector<Graph> graphs;
  spg_mlp* warm = nullptr;  // warm-start network (not owned)
  // live handles made through this context, and whether spg_destroy was
  // called (the context is then released with its last handle)
  std::mutex life_mu;
  int children = 0;
  bool closing = false;
};

struct spg_problem {
  spg_ctx* ctx = nullptr;
  int rows = 0, cols = 0, n = 0, dmax = 0, node_type = 0, shift = 0;
  std::vector<int> d;
  std::vector<int64_t> E;  // [n][dmax]
  std::vector<uint8_t> PL, PR, PU, PD, PG;
  std::vector<int> dims;  // [n][DIMW]
  std::vector<int64_t> RL;      // [n][lstride]
  std::vector<int64_t> RU, RA;  // [n][256]
  std::vector<uint8_t> gD;      // [n][MAXP]
  int bmax = 1, lstride = MAXP;
  bool ucpl = false;  // some site's MPO tensor depends on its up index beyond b_up (king's graph)
  size_t dev_bytes = 0;
  std::vector<int16_t> xsL;
  std::vector<int> xoffL;  // [n][MAXP+1]
  std::vector<int> keys;   // [n][MAXKEY+1]
  int kbits = 1;
  double min_sum = 0.0;  // sum of the minima of all local and reduced tables
  // largest span over sites of the site's weight factors (local, left, up,
  // anti-diagonal tables: max - min, summed), units of 2^-shift
  double wspan = 0.0;
  void* dev = nullptr;
  size_t o_E = 0, o_RL = 0, o_RU = 0, o_RA = 0;  // device offsets of the value tables
  DevTables tb{};
  // Ising problems: per site the SPG_WS_PER_CLUSTER coupling numbers of the
  // warm-start features (empty for Potts problems)
  std::vector<double> wsblk;
  bool counted = false;  // counted as a handle of ctx
  // the caller's inputs, kept to build the problem on transformed lattices
  struct Raw {
    bool potts = false;
    int n_spins = 0;
    std::vector<int32_t> ei, ej, cos, crow, ccol;  // Ising
    std::vector<double> J, h;                      // Ising (h empty: no fields)
    std::vector<int32_t> d, em, en;                // Potts
    std::vector<int64_t> local, pair;              // Potts
  } raw;
};

struct spg_result {
  spg_ctx* ctx = nullptr;
  int N = 0, cap = 0;
  // the result's device buffers, one block laid out as the solve's staged
  // outputs (carve_out), so that one copy fills it
  void* blk = nullptr;
  size_t blk_used = 0;
  int group_size = 1;  // instances of the lockstep group this solve ran in
  uint16_t* d_states = nullptr;
  int64_t* d_E = nullptr;
  double* d_logp = nullptr;
  int* d_n = nullptr;
  // diagnostics copied at the end of the solve
  int* d_diag = nullptr;  // near_ties, err, deg_cuts
  double* d_cand = nullptr;
  unsigned long long* d_stamp = nullptr;  // GPU timer at start, phase boundary, end (ns)
  double* d_err = nullptr;                // log-marginal error against FP64 (check_fp64)
  int fp64_rows = 0;
  int precision_used = 0;
  int* d_dn = nullptr;        // droplets of the best state: count, overflow
  int64_t* d_dE = nullptr;    // [MAXDROP]
  uint16_t* d_dst = nullptr;  // [MAXDROP][N]
  float ms_boundary = 0.f, ms_search = 0.f;
  double lognorm = 0.0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool fetched = false;
  int n = 0;
  long long launches = 0;
};

namespace {

int fail(spg_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, SPG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

}  // namespace
std::atomic<int>& spg::alloc_failure_countdown() {
  static std::atomic<int> c{-1};
  return c;
}
namespace {

// A device allocation, or the injected failure of the test hook.
cudaError_t device_alloc(void** p, size_t bytes) {
  int c = alloc_failure_countdown().load();
  while (c >= 0 && !alloc_failure_countdown().compare_exchange_weak(c, c - 1)) {
  }
  if (c == 0) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

// ---------------------------------------------------------------- warm-start inputs
// Index of the pair q1 < q2 of 8 spin positions in lexicographic order.
int ws_pair_slot(int q1, int q2) { return q1 * 8 - q1 * (q1 + 1) / 2 + (q2 - q1 - 1); }

// Inputs of the sites of boundary row r (include/spg.h spg_warm_features):
// the coupling blocks of the clusters in rows r .. r+2, columns j-2 .. j+2,
// then five position features, then zeros.
void ws_features(const spg_problem* P, int r, float* out) {
  const int rows = P->rows, cols = P->cols;
  for (int j = 0; j < cols; ++j) {
    float* x = out + (size_t)j * SPG_WS_FEATURES;
    std::fill(x, x + SPG_WS_FEATURES, 0.f);
    int o = 0;
    for (int i = r; i < r + 3; ++i)
      for (int k = j - 2; k <= j + 2; ++k, o += SPG_WS_PER_CLUSTER)
        if (i >= 0 && i < rows && k >= 0 && k < cols)
          for (int f = 0; f < SPG_WS_PER_CLUSTER; ++f)
            x[o + f] = (float)P->wsblk[(size_t)(i * cols + k) * SPG_WS_PER_CLUSTER + f];
    x[o + 0] = j == 0 ? 1.f : 0.f;
    x[o + 1] = j == cols - 1 ? 1.f : 0.f;
    x[o + 2] = j == 1 ? 1.f : 0.f;
    x[o + 3] = j == cols - 2 ? 1.f : 0.f;
    x[o + 4] = (float)(std::min(rows - r, 8) / 8.0);
  }
}

// The attached network when a solve with these parameters starts its rows
// from it: warm_start set, an Ising problem, and sites of this chi.
const spg_mlp* warm_of(const spg_ctx* ctx, const spg_problem* P, const spg_params* prm) {
  const spg_mlp* m = ctx->warm;
  if (!prm->warm_start || !m || P->wsblk.empty()) return nullptr;
  if (m->n_in != SPG_WS_FEATURES || m->n_out != MAXP * prm->chi * prm->chi) return nullptr;
  return m;
}

// ---------------------------------------------------------------- S1 helpers
struct EdgeTab {
  int Dm = 1, Dn = 1;
  std::vector<int64_t> R;       // Dm x Dn
  std::vector<uint8_t> Pm, Pn;  // d_m, d_n
};

// Distinct rows / columns of a full table T (dm x dn) in order of first
// occurrence; projectors and reduced table.  Returns false if > MAXP.
bool reduce_full(const std::vector<int64_t>& T, int dm, int dn, EdgeTab& out) {
  std::map<std::vector<int64_t>, int> rows, colsm;
  std::vector<int> firstr, firstc;
  out.Pm.assign(dm, 0);
  out.Pn.assign(dn, 0);
  for (int x = 0; x < dm; ++x) {
    std::vector<int64_t> r(T.begin() + (size_t)x * dn, T.begin() + (size_t)(x + 1) * dn);
    auto it = rows.find(r);
    if (it == rows.end()) {
      it = rows.emplace(r, (int)rows.size()).first;
      firstr.push_back(x);
    }
    if (it->second >= MAXP) return false;
    out.Pm[x] = (uint8_t)it->second;
  }
  for (int y = 0; y < dn; ++y) {
    std::vector<int64_t> c(dm);
    for (int x = 0; x < dm; ++x) c[x] = T[(size_t)x * dn + y];
    auto it = colsm.find(c);
    if (it == colsm.end()) {
      it = colsm.emplace(c, (int)colsm.size()).first;
      firstc.push_back(y);
    }
    if (it->second >= MAXP) return false;
    out.Pn[y] = (uint8_t)it->second;
  }
  out.Dm = (int)firstr.size();
  out.Dn = (int)firstc.size();
  out.R.assign((size_t)out.Dm * out.Dn, 0);
  for (int a = 0; a < out.Dm; ++a)
    for (int b = 0; b < out.Dn; ++b) out.R[(size_t)a * out.Dn + b] = T[(size_t)firstr[a] * dn + firstc[b]];
  return true;
}

// Joint projections, bond tables and device upload (S1).  The class of a
// state on a set of edges is its tuple of per-edge projections, numbered in
// order of first occurrence (x ascending); the pairwise energy between class
// representatives (first states) is exact because classes only merge states
// with equal table rows.
int finish_problem(spg_ctx* ctx, spg_problem* P, std::map<std::pair<int, int>, EdgeTab>& edges,
                   bool upload = true) {
  const int n = P->n, dmax = P->dmax, rows = P->rows, cols = P->cols;
  auto at = [&](int i, int j) { return (i >= 0 && i < rows && j >= 0 && j < cols) ? i * cols + j : -1; };
  auto edge = [&](int s, int t) -> const EdgeTab* {
    if (s < 0 || t < 0) return nullptr;
    auto it = edges.find({std::min(s, t), std::max(s, t)});
    return it == edges.end() ? nullptr : &it->second;
  };
  // projection of state x of s on its edge to t
  auto proj = [&](const EdgeTab* e, int s, int t, int x) { return s < t ? (int)e->Pm[x] : (int)e->Pn[x]; };
  // pairwise energy between state xs of s and xt of t (0 without an edge)
  auto pairE = [&](int s, int xs, int t, int xt) -> int64_t {
    const EdgeTab* e = edge(s, t);
    if (!e) return 0;
    if (s > t) {
      std::swap(s, t);
      std::swap(xs, xt);
    }
    return e->R[(size_t)e->Pm[xs] * e->Dn + e->Pn[xt]];
  };
  struct Cls {
    std::vector<uint8_t> P;
    std::vector<int> rep;
  };
  auto joint = [&](int s, std::initializer_list<int> nbrs, Cls& c) -> bool {
    std::map<std::vector<int>, int> idx;
    c.P.assign(dmax, 0);
    c.rep.clear();
    for (int x = 0; x < P->d[s]; ++x) {
      std::vector<int> key;
      for (int t : nbrs) {
        const EdgeTab* e = edge(s, t);
        if (e) key.push_back(proj(e, s, t, x));
      }
      auto it = idx.find(key);
      if (it == idx.end()) {
        if ((int)idx.size() >= MAXP) return false;
        it = idx.emplace(key, (int)idx.size()).first;
        c.rep.push_back(x);
      }
      c.P[x] = (uint8_t)it->second;
    }
    return true;
  };
  std::vector<Cls> L(n), U(n), R(n), D(n), G(n);
  for (int s = 0; s < n; ++s) {
    const int i = s / cols, j = s % cols;
    if (!joint(s, {at(i, j - 1), at(i - 1, j - 1)}, L[s]) || !joint(s, {at(i - 1, j)}, U[s]) ||
        !joint(s, {at(i, j + 1), at(i - 1, j + 1)}, R[s]) ||
        !joint(s, {at(i + 1, j - 1), at(i + 1, j), at(i + 1, j + 1)}, D[s]) || !joint(s, {at(i + 1, j + 1)}, G[s]))
      return fail(ctx, SPG_EUNSUPPORTED, "a joint projection has more than 16 classes");
  }
  auto ncls = [&](std::vector<Cls>& c, int s) { return s < 0 ? 1 : (int)c[s].rep.size(); };
  P->PL.assign((size_t)n * dmax, 0);
  P->PR.assign((size_t)n * dmax, 0);
  P->PU.assign((size_t)n * dmax, 0);
  P->PD.assign((size_t)n * dmax, 0);
  P->PG.assign((size_t)n * dmax, 0);
  P->dims.assign((size_t)n * DIMW, 0);
  int bmax = 1;
  for (int s = 0; s < n; ++s) {
    const int i = s / cols, j = s % cols;
    const int left = at(i, j - 1), upleft = at(i - 1, j - 1), up = at(i - 1, j);
    int* dm = &P->dims[(size_t)s * DIMW];
    dm[D_NRL] = ncls(R, left);
    dm[D_GIN] = ncls(G, upleft);
    dm[D_GOUT] = ncls(G, up);
    dm[D_NR] = ncls(R, s);
    dm[D_DL] = dm[D_NRL] * dm[D_GIN];
    dm[D_DR] = dm[D_NR] * dm[D_GOUT];
    dm[D_DU] = ncls(D, up);
    dm[D_DD] = ncls(D, s);
    dm[D_NL] = ncls(L, s);
    dm[D_NU] = ncls(U, s);
    dm[D_UCPL] = (dm[D_GOUT] > 1 || (edge(up, left) != nullptr)) ? 1 : 0;
    bmax = std::max(bmax, std::max(dm[D_DL], dm[D_DR]));
    std::copy(L[s].P.begin(), L[s].P.end(), P->PL.begin() + (size_t)s * dmax);
    std::copy(U[s].P.begin(), U[s].P.end(), P->PU.begin() + (size_t)s * dmax);
    std::copy(R[s].P.begin(), R[s].P.end(), P->PR.begin() + (size_t)s * dmax);
    std::copy(D[s].P.begin(), D[s].P.end(), P->PD.begin() + (size_t)s * dmax);
    std::copy(G[s].P.begin(), G[s].P.end(), P->PG.begin() + (size_t)s * dmax);
  }
  P->bmax = bmax;
  P->lstride = bmax * MAXP;
  P->ucpl = false;
  for (int s = 0; s < n; ++s) P->ucpl = P->ucpl || P->dims[(size_t)s * DIMW + D_UCPL] != 0;
  P->RL.assign((size_t)n * P->lstride, 0);
  P->RU.assign((size_t)n * 256, 0);
  P->RA.assign((size_t)n * 256, 0);
  P->gD.assign((size_t)n * MAXP, 0);
  double mins = 0.0;
  for (int s = 0; s < n; ++s) {
    const int i = s / cols, j = s % cols;
    const int left = at(i, j - 1), upleft = at(i - 1, j - 1), up = at(i - 1, j);
    const int* dm = &P->dims[(size_t)s * DIMW];
    int64_t mn = INT64_MAX;
    for (int x = 0; x < P->d[s]; ++x) mn = std::min(mn, P->E[(size_t)s * dmax + x]);
    mins += (double)mn;
    // left and up-left edges
    int64_t mnL = INT64_MAX;
    for (int l = 0; l < dm[D_DL]; ++l) {
      const int a = l / dm[D_GIN], g = l % dm[D_GIN];
      for (int h = 0; h < dm[D_NL]; ++h) {
        const int xh = L[s].rep[h];
        int64_t v = 0;
        if (left >= 0) v += pairE(left, R[left].rep[a], s, xh);
        if (upleft >= 0) v += pairE(upleft, G[upleft].rep[g], s, xh);
        P->RL[(size_t)s * P->lstride + (size_t)l * MAXP + h] = v;
        mnL = std::min(mnL, v);
      }
    }
    mins += (double)mnL;
    // up edge
    int64_t mnU = INT64_MAX;
    for (int u = 0; u < dm[D_DU]; ++u)
      for (int h = 0; h < dm[D_NU]; ++h) {
        const int64_t v = up >= 0 ? pairE(up, D[up].rep[u], s, U[s].rep[h]) : 0;
        P->RU[(size_t)s * 256 + u * 16 + h] = v;
        mnU = std::min(mnU, v);
      }
    mins += (double)mnU;
    // anti-diagonal edge (i-1, j)-(i, j-1)
    int64_t mnA = INT64_MAX;
    for (int a = 0; a < dm[D_NRL]; ++a)
      for (int u = 0; u < dm[D_DU]; ++u) {
        const int64_t v = (up >= 0 && left >= 0) ? pairE(up, D[up].rep[u], left, R[left].rep[a]) : 0;
        P->RA[(size_t)s * 256 + a * 16 + u] = v;
        mnA = std::min(mnA, v);
      }
    mins += (double)mnA;
    for (int u = 0; u < dm[D_DD]; ++u) P->gD[(size_t)s * MAXP + u] = G[s].P[D[s].rep[u]];
  }
  P->min_sum = mins;
  double wspan = 0.0;
  for (int s = 0; s < n; ++s) {
    const int* dm = &P->dims[(size_t)s * DIMW];
    auto span = [](int64_t lo, int64_t hi) { return hi >= lo ? (double)(hi - lo) : 0.0; };
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    for (int x = 0; x < P->d[s]; ++x) {
      lo = std::min(lo, P->E[(size_t)s * dmax + x]);
      hi = std::max(hi, P->E[(size_t)s * dmax + x]);
    }
    double t = span(lo, hi);
    lo = INT64_MAX, hi = INT64_MIN;
    for (int l = 0; l < dm[D_DL]; ++l)
      for (int h = 0; h < dm[D_NL]; ++h) {
        const int64_t v = P->RL[(size_t)s * P->lstride + (size_t)l * MAXP + h];
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
    t += span(lo, hi);
    lo = INT64_MAX, hi = INT64_MIN;
    for (int u = 0; u < dm[D_DU]; ++u)
      for (int h = 0; h < dm[D_NU]; ++h) {
        const int64_t v = P->RU[(size_t)s * 256 + u * 16 + h];
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
    t += span(lo, hi);
    lo = INT64_MAX, hi = INT64_MIN;
    for (int a = 0; a < dm[D_NRL]; ++a)
      for (int u = 0; u < dm[D_DU]; ++u) {
        const int64_t v = P->RA[(size_t)s * 256 + a * 16 + u];
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
    t += span(lo, hi);
    wspan = std::max(wspan, t);
  }
  P->wspan = wspan;
  // states grouped by PL
  P->xsL.assign((size_t)n * dmax, 0);
  P->xoffL.assign((size_t)n * (MAXP + 1), 0);
  for (int s = 0; s < n; ++s) {
    const int NL = P->dims[(size_t)s * DIMW + D_NL];
    int pos = 0;
    for (int h = 0; h < NL; ++h) {
      P->xoffL[s * (MAXP + 1) + h] = pos;
      for (int x = 0; x < P->d[s]; ++x)
        if (P->PL[(size_t)s * dmax + x] == h) P->xsL[(size_t)s * dmax + pos++] = (int16_t)x;
    }
    for (int h = NL; h <= MAXP; ++h) P->xoffL[s * (MAXP + 1) + h] = pos;
  }
  // merge keys: sites t <= s (t != s) with an edge to a site > s
  int bits = 1;
  while ((1 << bits) < dmax) ++bits;
  int kb = 1;
  while (kb < bits) kb <<= 1;
  P->kbits = kb;
  P->keys.assign((size_t)n * (MAXKEY + 1), 0);
  std::vector<int> far(n, -1);  // largest neighbour index of each site
  for (auto& kv : edges) {
    const int a = kv.first.first, b = kv.first.second;
    far[a] = std::max(far[a], b);
    far[b] = std::max(far[b], a);
  }
  for (int s = 0; s < n; ++s) {
    std::vector<int> ks;
    for (int t = 0; t < s; ++t)
      if (far[t] > s) ks.push_back(t);
    P->dims[(size_t)s * DIMW + D_XIN] = far[s] > s ? 1 : 0;  // the site's own state is part of its key
    if ((int)ks.size() > MAXKEY || (int)ks.size() * kb > KEYW * 64)
      return fail(ctx, SPG_EUNSUPPORTED, "merge key longer than the built limit");
    P->keys[(size_t)s * (MAXKEY + 1)] = (int)ks.size();
    for (size_t q = 0; q < ks.size(); ++q) P->keys[(size_t)s * (MAXKEY + 1) + 1 + q] = ks[q];
  }
  if (!upload) return SPG_OK;  // host tables only (spg_problem_update_ising)
  // upload
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t nd = (size_t)n * dmax;
  const size_t o_d = take(sizeof(int) * n), o_E = take(sizeof(int64_t) * nd), o_PL = take(nd), o_PR = take(nd),
               o_PU = take(nd), o_PD = take(nd), o_PG = take(nd), o_dims = take(sizeof(int) * n * DIMW),
               o_RL = take(sizeof(int64_t) * P->RL.size()), o_RU = take(sizeof(int64_t) * n * 256),
               o_RA = take(sizeof(int64_t) * n * 256), o_gD = take((size_t)n * MAXP),
               o_xs = take(sizeof(int16_t) * nd), o_xo = take(sizeof(int) * n * (MAXP + 1)),
               o_k = take(sizeof(int) * n * (MAXKEY + 1)), o_kb = take(sizeof(int));
  P->o_E = o_E;
  P->o_RL = o_RL;
  P->o_RU = o_RU;
  P->o_RA = o_RA;
  CK(cudaSetDevice(ctx->device));
  if (device_alloc(&P->dev, off) != cudaSuccess) {
    cudaGetLastError();
    P->dev = nullptr;
    return fail(ctx, SPG_ENOMEM, "problem tables: device allocation failed");
  }
  P->dev_bytes = off;
  char* base = (char*)P->dev;
  cudaStream_t st = ctx->stream;
  auto up = [&](size_t o, const void* src, size_t bytes) {
    return cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, st);
  };
  CK(up(o_d, P->d.data(), sizeof(int) * n));
  CK(up(o_E, P->E.data(), sizeof(int64_t) * nd));
  CK(up(o_PL, P->PL.data(), nd));
  CK(up(o_PR, P->PR.data(), nd));
  CK(up(o_PU, P->PU.data(), nd));
  CK(up(o_PD, P->PD.data(), nd));
  CK(up(o_PG, P->PG.data(), nd));
  CK(up(o_dims, P->dims.data(), sizeof(int) * n * DIMW));
  CK(up(o_RL, P->RL.data(), sizeof(int64_t) * P->RL.size()));
  CK(up(o_RU, P->RU.data(), sizeof(int64_t) * n * 256));
  CK(up(o_RA, P->RA.data(), sizeof(int64_t) * n * 256));
  CK(up(o_gD, P->gD.data(), (size_t)n * MAXP));
  CK(up(o_xs, P->xsL.data(), sizeof(int16_t) * nd));
  CK(up(o_xo, P->xoffL.data(), sizeof(int) * n * (MAXP + 1)));
  CK(up(o_k, P->keys.data(), sizeof(int) * n * (MAXKEY + 1)));
  CK(up(o_kb, &P->kbits, sizeof(int)));
  CK(cudaStreamSynchronize(st));
  DevTables& tb = P->tb;
  tb.rows = P->rows;
  tb.cols = P->cols;
  tb.n = n;
  tb.dmax = dmax;
  tb.lstride = P->lstride;
  tb.bmax = P->bmax;
  tb.d = (const int*)(base + o_d);
  tb.E = (const int64_t*)(base + o_E);
  tb.PL = (const uint8_t*)(base + o_PL);
  tb.PR = (const uint8_t*)(base + o_PR);
  tb.PU = (const uint8_t*)(base + o_PU);
  tb.PD = (const uint8_t*)(base + o_PD);
  tb.PG = (const uint8_t*)(base + o_PG);
  tb.dims = (const int*)(base + o_dims);
  tb.RL = (const int64_t*)(base + o_RL);
  tb.RU = (const int64_t*)(base + o_RU);
  tb.RA = (const int64_t*)(base + o_RA);
  tb.gD = (const uint8_t*)(base + o_gD);
  tb.xsL = (const int16_t*)(base + o_xs);
  tb.xoffL = (const int*)(base + o_xo);
  tb.keys = (const int*)(base + o_k);
  tb.kshift = (const int*)(base + o_kb);
  return SPG_OK;
}

// ---------------------------------------------------------------- workspace
struct Arena {
  char* base;
  size_t off = 0, cap;
  template <typename T>
  T* get(size_t count) {
    size_t o = off;
    off += (sizeof(T) * count + 255) & ~size_t(255);
    return off <= cap ? reinterpret_cast<T*>(base + o) : nullptr;
  }
};

void drop_graphs(spg_ctx* ctx, const void* problem);

int ensure_arena(spg_ctx* ctx, size_t bytes) {
  if (ctx->arena_bytes >= bytes) return SPG_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  drop_graphs(ctx, nullptr);  // captured solves address the old workspace
  if (ctx->arena) CK(cudaFree(ctx->arena));
  ctx->arena = nullptr;
  ctx->arena_bytes = 0;
  cudaError_t e = device_alloc((void**)&ctx->arena, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SPG_ENOMEM, "device workspace allocation failed");
  }
  ctx->arena_bytes = bytes;
  return SPG_OK;
}

// Host-side bond dimensions of every boundary MPS (structural: they depend
// only on the tables' dimensions, chi, and the zipper's keep rule).
struct Plan {
  int rows, cols, chi;
  std::vector<int> dimA;  // [(rows+1)*cols][3] p, chiL, chiR
  size_t stride;
};

Plan make_plan(const spg_problem* P, int chi, int down_to) {
  Plan pl;
  pl.rows = P->rows;
  pl.cols = P->cols;
  pl.chi = chi;
  const int cols = P->cols;
  pl.dimA.assign((size_t)(P->rows + 1) * cols * 3, 1);
  for (int r = P->rows - 1; r >= down_to; --r) {
    int K = 1;
    for (int j = cols - 1; j >= 0; --j) {
      const int s = r * cols + j;
      const int DL = P->dims[(size_t)s * DIMW + D_DL], DU = P->dims[(size_t)s * DIMW + D_DU];
      const int chiL_in = pl.dimA[(((size_t)(r + 1) * cols + j) * 3) + 1];
      int* o = &pl.dimA[((size_t)r * cols + j) * 3];
      if (j == 0) {
        o[0] = DU;
        o[1] = 1;
        o[2] = K;
      } else {
        const int m = DL * chiL_in, n = DU * K;
        const int keep = std::min(chi, std::min(m, n));
        o[0] = DU;
        o[1] = keep;
        o[2] = K;
        K = keep;
      }
    }
  }
  pl.stride = (size_t)MAXP * chi * chi;
  return pl;
}

template <typename T>
struct BoundaryBufs {
  DevMPS<T> mps;
  int* dimA_dev;
  DevWeights<T> wt;
  DevWeights<double> wd;
  T* T1;
  T* M;
  T* V;
  T* US;
  T* carry[2];
  T* svdw;
  size_t svdw_elems;
  double* s1;
  int* degc;
  T* swork;
  double* sdbl;
  float* tcw;  // tensor-core product workspace (FP32 solves on large zipper matrices)
  size_t tcw_elems;
  // FP64 truncation of the final rows in the mixed mode (fp64 > 0, T = float):
  // the zipper matrix, V, US, the truncation's work, one MPS row and the
  // left-canonical scratch, all in FP64
  int fp64 = 0;
  double *Md = nullptr, *Vd = nullptr, *USd = nullptr, *svdwd = nullptr, *rowd = nullptr, *lcd = nullptr;
  size_t svdwd_elems = 0;
  // warm start: the network, its inputs [cols][SPG_WS_FEATURES], outputs
  // [cols][16 chi chi] and inference scratch
  const spg_mlp* ws = nullptr;
  float *wsX = nullptr, *wsY = nullptr, *wswork = nullptr;
  // export of every row as it is finished (rows 1 ..): padded sites
  // [rows-1][cols][16][chi][chi], sign gauge when exp_fix
  T* exp_out = nullptr;
  int exp_fix = 0;
};

// Boundary rows whose truncations run in FP64 in the mixed mode: rows 1 ..
// fp64 (and row 0 when fp64 >= 1); none in the FP64 mode, where every row is.
template <typename T>
int fp64_rows_of(const spg_params* prm, const spg_problem* P) {
  if (sizeof(T) == sizeof(double)) return 0;
  if (prm->fp64_rows >= 0) return prm->fp64_rows;
  return P->n <= SPG_FP64_ROWS_AUTO_SITES ? P->rows : 0;
}

bool fp64_row(int fp64, int r) { return fp64 >= 1 && r <= fp64; }

// Whether a solve in SPG_MIXED runs the FP64 path instead: when the weight
// factors of one site may multiply down to e^-SPG_FP32_WEIGHT_SPAN, states
// that matter can get FP32 weights below the normal range (e^-87) and their
// conditionals come out as zero.
bool fp32_range_exceeded(const spg_problem* P, const spg_params* prm) {
  return prm->precision == SPG_MIXED && prm->beta * std::ldexp(P->wspan, -P->shift) > SPG_FP32_WEIGHT_SPAN;
}

// Tensor-core workspace of a problem's largest zipper matrix (FP32 only).
template <typename T>
size_t tc_work(const spg_problem* P, int chi) {
  if (sizeof(T) != sizeof(float)) return 0;
  const int mmax = P->bmax * chi, nmax = MAXP * chi;
  const int s = std::min(SMAX, (chi + 16 + 15) / 16 * 16);
  return tc_gemm_eligible(mmax, nmax, s) ? tc_gemm_elems(mmax, nmax, s) : 0;
}

template <typename T>
size_t boundary_bytes(const spg_problem* P, const Plan& pl, int fp64 = 0, const spg_mlp* ws = nullptr) {
  const int chi = pl.chi;
  const size_t sites = (size_t)(P->rows + 1) * P->cols;
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~size_t(255); };
  add(sizeof(T) * sites * pl.stride);
  add(sizeof(int) * sites * 3);
  add(sizeof(double) * (P->rows + 1));
  add(sizeof(T) * P->n * P->dmax);
  add(sizeof(T) * P->n * P->lstride);
  add(sizeof(T) * P->n * 256 * 2);
  add(sizeof(double) * P->n * P->dmax);
  add(sizeof(double) * P->n * P->lstride);
  add(sizeof(double) * P->n * 256 * 2);
  const size_t mmax = (size_t)P->bmax * chi, nmax = (size_t)MAXP * chi;
  add(sizeof(T) * (size_t)chi * MAXP * P->bmax * chi);  // T1
  add(sizeof(T) * mmax * nmax);                        // M
  add(sizeof(T) * nmax * chi);                         // V
  add(sizeof(T) * mmax * chi);                         // US
  add(sizeof(T) * P->bmax * chi * chi * 2);            // carries
  add(sizeof(T) * truncated_svd_work((int)mmax, (int)nmax, chi));
  add(sizeof(double) * 4);
  add(sizeof(int) * 4);
  add(sizeof(T) * sweep_work_elems<T>(P->cols, chi, P->bmax));
  add(sizeof(double) * 4);
  add(sizeof(float) * tc_work<T>(P, chi));
  if (fp64 > 0 && sizeof(T) == sizeof(float)) {
    add(sizeof(double) * mmax * nmax);
    add(sizeof(double) * nmax * chi);
    add(sizeof(double) * mmax * chi);
    add(sizeof(double) * truncated_svd_work((int)mmax, (int)nmax, chi));
    add(sizeof(double) * P->cols * pl.stride);
    add(sizeof(double) * (size_t)MAXP * chi * chi);
  }
  if (ws) {
    add(sizeof(float) * P->cols * SPG_WS_FEATURES);
    add(sizeof(float) * P->cols * (size_t)MAXP * chi * chi);
    add(sizeof(float) * mlp_infer_elems(ws, P->cols));
  }
  return b + 4096;
}

template <typename T>
int carve_boundary(spg_ctx* ctx, const spg_problem* P, const Plan& pl, Arena& ar, BoundaryBufs<T>& bb,
                   bool init = true, int fp64 = 0, const spg_mlp* ws = nullptr) {
  const int chi = pl.chi;
  const size_t sites = (size_t)(P->rows + 1) * P->cols;
  bb.mps.A = ar.get<T>(sites * pl.stride);
  bb.mps.site_stride = pl.stride;
  bb.dimA_dev = ar.get<int>(sites * 3);
  bb.mps.dimA = bb.dimA_dev;
  bb.mps.lognorm = ar.get<double>(P->rows + 1);
  bb.wt.w = ar.get<T>((size_t)P->n * P->dmax);
  bb.wt.bL = ar.get<T>((size_t)P->n * P->lstride);
  bb.wt.bU = ar.get<T>((size_t)P->n * 256);
  bb.wt.bA = ar.get<T>((size_t)P->n * 256);
  bb.wd.w = ar.get<double>((size_t)P->n * P->dmax);
  bb.wd.bL = ar.get<double>((size_t)P->n * P->lstride);
  bb.wd.bU = ar.get<double>((size_t)P->n * 256);
  bb.wd.bA = ar.get<double>((size_t)P->n * 256);
  const size_t mmax = (size_t)P->bmax * chi, nmax = (size_t)MAXP * chi;
  bb.T1 = ar.get<T>((size_t)chi * MAXP * P->bmax * chi);
  bb.M = ar.get<T>(mmax * nmax);
  bb.V = ar.get<T>(nmax * chi);
  bb.US = ar.get<T>(mmax * chi);
  bb.carry[0] = ar.get<T>((size_t)P->bmax * chi * chi);
  bb.carry[1] = ar.get<T>((size_t)P->bmax * chi * chi);
  bb.svdw_elems = truncated_svd_work((int)mmax, (int)nmax, chi);
  bb.svdw = ar.get<T>(bb.svdw_elems);
  bb.s1 = ar.get<double>(4);
  bb.degc = ar.get<int>(4);
  bb.swork = ar.get<T>(sweep_work_elems<T>(P->cols, chi, P->bmax));
  bb.sdbl = ar.get<double>(4);
  bb.tcw_elems = tc_work<T>(P, chi);
  bb.tcw = bb.tcw_elems ? ar.get<float>(bb.tcw_elems) : nullptr;
  if (!bb.sdbl || (bb.tcw_elems && !bb.tcw)) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  bb.fp64 = sizeof(T) == sizeof(float) ? fp64 : 0;
  if (bb.fp64 > 0) {
    bb.Md = ar.get<double>(mmax * nmax);
    bb.Vd = ar.get<double>(nmax * chi);
    bb.USd = ar.get<double>(mmax * chi);
    bb.svdwd_elems = truncated_svd_work((int)mmax, (int)nmax, chi);
    bb.svdwd = ar.get<double>(bb.svdwd_elems);
    bb.rowd = ar.get<double>((size_t)P->cols * pl.stride);
    bb.lcd = ar.get<double>((size_t)MAXP * chi * chi);
    if (!bb.lcd) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  }
  bb.ws = ws;
  if (ws) {
    bb.wsX = ar.get<float>((size_t)P->cols * SPG_WS_FEATURES);
    bb.wsY = ar.get<float>((size_t)P->cols * MAXP * chi * chi);
    bb.wswork = ar.get<float>(mlp_infer_elems(ws, P->cols));
    if (!bb.wswork) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  }
  if (!init) return SPG_OK;
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(bb.dimA_dev, pl.dimA.data(), sizeof(int) * sites * 3, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(bb.mps.lognorm, 0, sizeof(double) * (P->rows + 1), st));
  CK(cudaMemsetAsync(bb.degc, 0, sizeof(int) * 4, st));
  return SPG_OK;
}

// Row r of the boundary MPSs from B_{r+1} (S3): the left-canonical QR of
// B_{r+1}, then either the zipper (MPO site by MPO site, right to left, with
// the truncated SVD of each zipper matrix) or, with `warm`, the sites the
// network predicts from the couplings near the row (the starting point of
// the variational compression that follows).
template <typename T>
int build_row(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, const Plan& pl, BoundaryBufs<T>& bb, int r,
              bool warm) {
  cudaStream_t st = ctx->stream;
  const int cols = P->cols;
  const bool f64 = bb.fp64 > 0 && fp64_row(bb.fp64, r);
  if constexpr (std::is_same<T, float>::value) {
    if (f64) {
      // left-canonical QR of B_{r+1} in FP64 (the row seen as row 0 of a
      // one-row MPS with the same dims and log-norm slot)
      T* row = bb.mps.A + (size_t)(r + 1) * cols * pl.stride;
      const size_t cnt = (size_t)cols * pl.stride;
      DevMPS<double> md{bb.rowd, pl.stride, bb.dimA_dev + (size_t)(r + 1) * cols * 3, bb.mps.lognorm + r + 1};
      CK((launch_convert<float, double>(row, bb.rowd, cnt, st)));
      CK(launch_left_canonical<double>(md, 0, cols, nullptr, bb.lcd, st));
      CK((launch_convert<double, float>(bb.rowd, row, cnt, st)));
    }
  }
  if (!f64) CK(launch_left_canonical<T>(bb.mps, r + 1, cols, nullptr, bb.T1, st));
  CK(zcopy(bb.mps.lognorm + r, bb.mps.lognorm + r + 1, sizeof(double), st));
  if (warm) {
    std::vector<float> X((size_t)cols * SPG_WS_FEATURES);
    ws_features(P, r, X.data());
    CK(cudaMemcpyAsync(bb.wsX, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, st));
    CK(mlp_infer_bf16(bb.ws, bb.wsX, cols, bb.wswork, bb.wsY, st));
    CK(launch_ws_scatter<T>(bb.wsY, pl.chi, cols, bb.mps, r, st));
    CK(cudaStreamSynchronize(st));  // X is released on return
    return SPG_OK;
  }
  CK(launch_set_strided<T>(bb.carry[0], 1, 1, T(1), st));
  int K = 1, cur = 0;
  for (int j = cols - 1; j >= 0; --j) {
    const int s = r * cols + j;
    const int* dm = &P->dims[(size_t)s * DIMW];
    const int DL = dm[D_DL], DR = dm[D_DR], DU = dm[D_DU];
    const int* din = &pl.dimA[((size_t)(r + 1) * cols + j) * 3];
    const int p = din[0], chiL = din[1], chiR = din[2];
    const T* Bsite = bb.mps.A + (size_t)((r + 1) * cols + j) * pl.stride;
    T* out = bb.mps.A + (size_t)(r * cols + j) * pl.stride;
    CK(launch_zip_matrix<T>(P->tb, bb.wt, Bsite, chiL, p, chiR, bb.carry[cur], DR, K, s, DL, DU, bb.T1, bb.M, st));
    if (j == 0) {
      CK(launch_zip_site0<T>(bb.M, DU, K, out, bb.mps.lognorm + r, st));
    } else {
      const int m = DL * chiL, n = DU * K;
      const int keep = pl.dimA[((size_t)r * cols + j) * 3 + 1];
      const int iters = prm->svd_iters >= 0 ? prm->svd_iters : (sizeof(T) == 8 ? 6 : 2);
      const uint64_t seed = prm->seed + (uint64_t)s * 7919u;
      if constexpr (std::is_same<T, float>::value) {
        if (f64) {
          // the FP32 zipper matrix truncated in FP64, V and US rounded back
          CK((launch_convert<float, double>(bb.M, bb.Md, (size_t)m * n, st)));
          CK(truncated_svd<double>(bb.Md, m, n, keep, iters, seed, bb.Vd, bb.USd, bb.svdwd, bb.svdwd_elems, bb.s1,
                                   bb.degc, st));
          CK((launch_convert<double, float>(bb.Vd, bb.V, (size_t)n * keep, st)));
          CK((launch_convert<double, float>(bb.USd, bb.US, (size_t)m * keep, st)));
        }
      }
      if (!f64)
        CK(truncated_svd<T>(bb.M, m, n, keep, iters, seed, bb.V, bb.US, bb.svdw, bb.svdw_elems, bb.s1, bb.degc, st,
                            bb.tcw, bb.tcw_elems));
      CK(launch_zip_write<T>(bb.V, bb.US, DL, chiL, DU, K, keep, out, bb.carry[cur ^ 1], bb.s1, bb.mps.lognorm + r,
                             st));
      cur ^= 1;
      K = keep;
    }
  }
  return SPG_OK;
}

// Boundary MPSs B_r for r = rows-1 .. down_to (S2-S4): weights, the trivial
// B_L, then row by row the zipper (or the network's start when bb.ws is
// set) and num_sweeps variational sweeps.
template <typename T>
int run_boundary(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, const Plan& pl, BoundaryBufs<T>& bb,
                 int down_to) {
  cudaStream_t st = ctx->stream;
  const int cols = P->cols;
  const double beta_u = prm->beta * std::ldexp(1.0, -P->shift);
  CK(launch_weights<T>(P->tb, bb.wt, beta_u, st));
  if (sizeof(T) != sizeof(double)) CK(launch_weights<double>(P->tb, bb.wd, beta_u, st));
  // B_L: trivial sites (value 1)
  CK(launch_set_strided<T>(bb.mps.A + (size_t)P->rows * cols * pl.stride, pl.stride, cols, T(1), st));
  for (int r = P->rows - 1; r >= down_to; --r) {
    int rc = build_row<T>(ctx, P, prm, pl, bb, r, bb.ws != nullptr);
    if (rc) return rc;
    if (prm->num_sweeps > 0)
      CK(variational_sweeps<T>(P->tb, bb.wt, bb.mps, r, cols, pl.dimA.data(), P->dims.data(), P->d.data(),
                               P->gD.data(), prm->num_sweeps, bb.swork, bb.sdbl, st));
    // the row as finished, before the next row's left-canonical QR changes its gauge
    if (bb.exp_out && r >= 1)
      CK(launch_export_row<T>(bb.mps, r, cols, pl.chi, bb.exp_out + (size_t)(r - 1) * cols * MAXP * pl.chi * pl.chi,
                              bb.dimA_dev + (size_t)r * cols * 3, bb.exp_fix, st));
  }
  return SPG_OK;
}

template <typename T>
struct SearchBufs {
  DevSearch ds;
  DevBeamT<T> bt;
  float* rtw = nullptr;         // tensor-core right environments' work (FP32)
  std::vector<char> tc_rows;    // rows whose right environments take that path
  std::vector<double> mflops;   // per site: algorithmic flops of one beam element's marginals
};

// Algorithmic flops of one beam element's conditionals at each site
// (profiling): v = lenv B (2 p chiL chiR), Z = v R (2 p NR chiR), the
// weights and their sum (4 d).
std::vector<double> marginal_flops(const spg_problem* P, const Plan& pl) {
  std::vector<double> f(P->n, 0.0);
  for (int s = 0; s < P->n; ++s) {
    const int i = s / P->cols, j = s % P->cols;
    if ((size_t)((i + 1) * P->cols + j) * 3 + 2 >= pl.dimA.size()) continue;
    const int* dA = &pl.dimA[((size_t)(i + 1) * P->cols + j) * 3];
    const double p = dA[0], chiL = dA[1], chiR = dA[2], NR = P->dims[(size_t)s * DIMW + D_NR];
    f[s] = 2.0 * p * chiL * chiR + 2.0 * p * NR * chiR + 4.0 * P->d[s];
  }
  return f;
}

// Whether a problem's right environments may run on the tensor cores at
// bond chi (renv_tc.cu): bonds of at most 32, environment bond <= 16.
bool renv_tc_problem(const spg_problem* P, int chi) { return chi <= 32 && P->bmax <= 16 && P->cols >= 3; }

// The rows whose sites satisfy the conditions of renv_tc.cu (Gout = 1, no
// up-index coupling, DL, DR, NL <= 16, B_{i+1}'s sites within 16 x 32 x 32,
// and, but at the rightmost column, every right class of a site's states
// with one left class, distinct for distinct right classes).
std::vector<char> renv_tc_rows(const spg_problem* P, const Plan& pl) {
  std::vector<char> ok(P->rows, 0);
  if (!renv_tc_problem(P, pl.chi)) return ok;
  const int cols = P->cols;
  for (int i = 0; i < P->rows; ++i) {
    bool good = true;
    for (int j = 1; j < cols && good; ++j) {
      const int s = i * cols + j;
      const int* dm = &P->dims[(size_t)s * DIMW];
      good = dm[D_DR] <= 16 && dm[D_DL] <= 16 && dm[D_NL] <= 16 && dm[D_GOUT] == 1 && dm[D_UCPL] == 0;
      const int* dA = &pl.dimA[((size_t)(i + 1) * cols + j) * 3];
      good = good && dA[0] <= 16 && dA[1] <= 32 && dA[2] <= 32;
      int h_of[MAXP], r_of[MAXP];
      for (int q = 0; q < MAXP; ++q) h_of[q] = r_of[q] = -1;
      for (int x = 0; x < P->d[s] && good && j < cols - 1; ++x) {
        const int r = P->PR[(size_t)s * P->dmax + x], h = P->PL[(size_t)s * P->dmax + x];
        if (r >= MAXP || h >= MAXP) {
          good = false;
        } else if (h_of[r] < 0) {
          good = r_of[h] < 0;  // distinct right classes keep distinct left classes
          h_of[r] = h;
          r_of[h] = r;
        } else {
          good = h_of[r] == h;
        }
      }
    }
    ok[i] = good ? 1 : 0;
  }
  return ok;
}

template <typename T>
size_t search_bytes(const spg_problem* P, int cap, int chi, bool drops = false) {
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~size_t(255); };
  const size_t N = P->n, dmax = P->dmax;
  for (int k = 0; k < 2; ++k) {
    add(sizeof(uint16_t) * cap * N);
    add(sizeof(int64_t) * cap);
    add(sizeof(double) * cap);
    add(sizeof(int) * cap);
    add(sizeof(T) * cap * chi);
  }
  add(sizeof(int) * 2);
  add(sizeof(double) * cap * dmax);
  add(sizeof(int64_t) * cap * dmax);
  add(sizeof(int) * cap * dmax);
  add(sizeof(unsigned long long) * cap * dmax);
  add(sizeof(int) * cap);
  add(sizeof(unsigned long long) * cap * KEYW);
  add(sizeof(int) * cap * 3);
  add(sizeof(int) * 4 * (size_t)cap * 2 + 1024);  // class hash table and minima
  add(sizeof(int) * cap * dmax);
  add(sizeof(unsigned) * 65536);
  add(sizeof(unsigned long long) * 16);
  add(sizeof(int) * 8);
  add(sizeof(double) * 2);
  add(sizeof(T) * cap * (P->cols + 1) * chi * P->bmax);
  if (sizeof(T) == sizeof(float) && renv_tc_problem(P, chi)) add(sizeof(float) * renv_tc_elems(P->cols, cap));
  if (drops)
    for (int k = 0; k < 2; ++k) {
      add(sizeof(int) * cap);
      add(sizeof(int64_t) * cap * MAXDROP);
      add(sizeof(uint16_t) * (size_t)cap * MAXDROP * N);
    }
  add(sizeof(int) * 4);
  return b + 4096;
}

template <typename T>
int carve_search(spg_ctx* ctx, const spg_problem* P, int cap, int chi, Arena& ar, SearchBufs<T>& sb,
                 bool init = true, bool drops = false) {
  DevSearch& ds = sb.ds;
  ds.cap = cap;
  ds.N = P->n;
  ds.dmax = P->dmax;
  for (int k = 0; k < 2; ++k) {
    ds.states[k] = ar.get<uint16_t>((size_t)cap * P->n);
    ds.E[k] = ar.get<int64_t>(cap);
    ds.logp[k] = ar.get<double>(cap);
    ds.rid[k] = ar.get<int>(cap);
    sb.bt.lenv[k] = ar.get<T>((size_t)cap * chi);
  }
  ds.n_beam = ar.get<int>(2);
  ds.logc = ar.get<double>((size_t)cap * P->dmax);
  ds.candE = ar.get<int64_t>((size_t)cap * P->dmax);
  ds.win = ar.get<int>((size_t)cap * P->dmax);
  ds.wmin = ar.get<unsigned long long>((size_t)cap * P->dmax);
  ds.wkey = ar.get<int>(cap);
  ds.key = ar.get<unsigned long long>((size_t)cap * KEYW);
  ds.rep = ar.get<int>(cap);
  ds.nxt = ar.get<int>(cap);
  ds.hsize = 1;
  while (ds.hsize < 2 * cap) ds.hsize <<= 1;
  ds.htab = ar.get<int>(ds.hsize);
  ds.hmin = ar.get<int>(ds.hsize);
  ds.sel_list = ar.get<int>(cap);
  ds.pend = ar.get<int>((size_t)cap * P->dmax);
  ds.hist = ar.get<unsigned>(65536);
  ds.sel_state = ar.get<unsigned long long>(16);
  int* misc = ar.get<int>(8);
  ds.sel_count = misc;
  ds.done_ctr = (unsigned*)(misc + 1);
  ds.near_ties = misc + 2;
  ds.err = misc + 3;
  ds.deg_cuts = misc + 4;
  ds.pend_n = misc + 5;
  ds.candidates = ar.get<double>(2);
  sb.bt.R = ar.get<T>((size_t)cap * (P->cols + 1) * chi * P->bmax);
  sb.bt.rs = P->bmax;
  sb.bt.chi = chi;
  if (sizeof(T) == sizeof(float) && renv_tc_problem(P, chi)) sb.rtw = ar.get<float>(renv_tc_elems(P->cols, cap));
  if (drops)
    for (int k = 0; k < 2; ++k) {
      ds.dn[k] = ar.get<int>(cap);
      ds.dE[k] = ar.get<int64_t>((size_t)cap * MAXDROP);
      ds.dst[k] = ar.get<uint16_t>((size_t)cap * MAXDROP * P->n);
    }
  ds.dflow = ar.get<int>(4);
  if (!ds.dflow) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  if (!init) return SPG_OK;
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(ds.hist, 0, sizeof(unsigned) * 65536, st));
  CK(cudaMemsetAsync(misc, 0, sizeof(int) * 8, st));
  CK(cudaMemsetAsync(sb.bt.R, 0, sizeof(T) * (size_t)cap * (P->cols + 1) * chi * P->bmax, st));
  CK(cudaMemsetAsync(sb.bt.lenv[0], 0, sizeof(T) * (size_t)cap * chi, st));
  CK(cudaMemsetAsync(sb.bt.lenv[1], 0, sizeof(T) * (size_t)cap * chi, st));
  return SPG_OK;
}

int check_params(spg_ctx* ctx, const spg_problem* P, const spg_params* prm) {
  if (!prm) return fail(ctx, SPG_EINVAL, "params is NULL");
  if (!(prm->beta >= 0.0) || !std::isfinite(prm->beta)) return fail(ctx, SPG_EINVAL, "beta must be finite, >= 0");
  if (prm->chi < 1 || prm->chi > SPG_MAX_CHI) return fail(ctx, SPG_EUNSUPPORTED, "chi outside 1..64");
  if (prm->beam < 1 || prm->beam > SPG_MAX_BEAM) return fail(ctx, SPG_EUNSUPPORTED, "beam outside 1..4096");
  if (prm->num_sweeps < 0 || prm->num_sweeps > 16) return fail(ctx, SPG_EINVAL, "num_sweeps outside 0..16");
  if (prm->precision != SPG_FP64 && prm->precision != SPG_MIXED) return fail(ctx, SPG_EINVAL, "bad precision");
  if (prm->svd_iters < -1 || prm->svd_iters > 64) return fail(ctx, SPG_EINVAL, "svd_iters outside -1..64");
  if (prm->warm_start != 0 && prm->warm_start != 1) return fail(ctx, SPG_EINVAL, "warm_start must be 0 or 1");
  if (prm->warm_start && prm->num_sweeps < 1)
    return fail(ctx, SPG_EINVAL, "warm_start needs num_sweeps >= 1 (the sweeps refine the network's start)");
  if (!(prm->cut_off_prob >= 0.0 && prm->cut_off_prob < 1.0)) return fail(ctx, SPG_EINVAL, "cut_off_prob in [0,1)");
  if (prm->fp64_rows < -1) return fail(ctx, SPG_EINVAL, "fp64_rows must be >= -1");
  if (prm->check_fp64 != 0 && prm->check_fp64 != 1) return fail(ctx, SPG_EINVAL, "check_fp64 must be 0 or 1");
  if (prm->group_max < 0) return fail(ctx, SPG_EINVAL, "group_max must be >= 0");
  if (prm->droplet_hamming < 0 || !std::isfinite(prm->droplet_energy))
    return fail(ctx, SPG_EINVAL, "droplet_hamming must be >= 0 and droplet_energy finite");
  if (prm->droplet_energy >= 0.0 && std::ldexp(prm->droplet_energy, P->shift) > 4.0e18)
    return fail(ctx, SPG_EINVAL, "droplet_energy too large for the integer energies");
  if (P->n > 65535) return fail(ctx, SPG_EUNSUPPORTED, "too many sites");
  return SPG_OK;
}

// Output staging at fixed workspace addresses, so that a captured solve can
// be replayed; copied into the result's own buffers after each run.
struct OutStage {
  uint16_t* states;
  int64_t* E;
  double* logp;
  int* n;
  int* diag;  // near_ties, err, degenerate cuts, Jacobi sweeps
  double* cand;  // candidates, log-norm of B_1
  unsigned long long* stamp;  // GPU timer at start, phase boundary, end
  double* err;  // log-marginal error against FP64 (NaN unless checked)
  int* dn;               // droplets of the best state: count,
  int64_t* dE;           // energies [MAXDROP],
  uint16_t* dst;         // states [MAXDROP][N]
};

// The staged outputs carved from `ar` (the same sequence for the workspace
// and for a result's block, so that both have one layout); returns the bytes
// taken, 0 when the arena is too small.
size_t carve_out(Arena& ar, const spg_problem* P, int cap, OutStage& o) {
  const size_t off0 = ar.off;
  o.states = ar.get<uint16_t>((size_t)cap * P->n);
  o.E = ar.get<int64_t>(cap);
  o.logp = ar.get<double>(cap);
  o.n = ar.get<int>(4);
  o.diag = ar.get<int>(4);
  o.cand = ar.get<double>(2);
  o.stamp = ar.get<unsigned long long>(4);
  o.err = ar.get<double>(1);
  o.dn = ar.get<int>(4);
  o.dE = ar.get<int64_t>(MAXDROP);
  o.dst = ar.get<uint16_t>((size_t)MAXDROP * P->n);
  return o.dst ? ar.off - off0 : 0;
}

size_t out_stage_bytes(const spg_problem* P, int cap) {
  auto r = [](size_t x) { return (x + 255) & ~size_t(255); };
  return r(sizeof(uint16_t) * (size_t)cap * P->n) + 2 * r(8 * (size_t)cap) + 7 * 256 + r(8 * MAXDROP) +
         r(sizeof(uint16_t) * MAXDROP * (size_t)P->n);
}

template <typename T>
int enqueue_boundary(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, const Plan& pl,
                     BoundaryBufs<T>& bb) {
  cudaStream_t st = ctx->stream;
  CK(zfill(bb.mps.lognorm, 0, sizeof(double) * (P->rows + 1), st));
  CK(zfill(bb.degc, 0, sizeof(int) * 4, st));
  return run_boundary<T>(ctx, P, prm, pl, bb, 1);
}

// Right environments of row i for beam buffer cur: on the tensor cores
// where the row allows it (FP32), else k_right_envs.
template <typename T>
cudaError_t right_envs(const spg_problem* P, BoundaryBufs<T>& bb, SearchBufs<T>& sb, int i, int cur,
                       cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value)
    if (sb.rtw && i < (int)sb.tc_rows.size() && sb.tc_rows[i])
      return launch_right_envs_tc(P->tb, bb.wt, bb.mps, i, sb.ds, sb.bt, cur, sb.rtw, st);
  return launch_right_envs<T>(P->tb, bb.wt, bb.mps, i, sb.ds, sb.bt, cur, st);
}

template <typename T>
int enqueue_search(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, BoundaryBufs<T>& bb,
                   SearchBufs<T>& sb, const OutStage& o) {
  cudaStream_t st = ctx->stream;
  DevSearch& ds = sb.ds;
  ds.deg_cuts = bb.degc;
  const int cols = P->cols;
  const double log_cut = prm->cut_off_prob > 0 ? std::log(prm->cut_off_prob) : -INFINITY;
  int cur = 0;
  CK(launch_reset_beam(ds, cur, st));
  for (int s = 0; s < P->n; ++s) {
    const int i = s / cols, j = s % cols;
    if (j == 0) CK(right_envs<T>(P, bb, sb, i, cur, st));
    CK(launch_marginals<T>(P->tb, bb.wt, bb.wd, bb.mps, s, ds, sb.bt, cur, st,
                           s < (int)sb.mflops.size() ? sb.mflops[s] * ds.cap : 0.0));
    CK(launch_merge(P->tb, s, ds, cur, prm->merge, st));
    CK(launch_select(P->tb, s, ds, cur, log_cut, st));
    CK(launch_update<T>(P->tb, bb.mps, s, ds, sb.bt, cur, st));
    if (ds.dcut >= 0) CK(launch_droplets(P->tb, s, ds, cur, prm->merge, st));
    cur ^= 1;
  }
  CK(launch_final(P->tb, ds, cur, o.states, o.E, o.logp, o.n, st));
  if (ds.dcut >= 0)
    CK(launch_final_droplets(ds, cur, o.dn, o.dE, o.dst, st));
  else
    CK(zfill(o.dn, 0, sizeof(int), st));
  CK(zcopy(o.dn + 1, ds.dflow, sizeof(int), st));
  CK(zcopy(o.diag + 0, ds.near_ties, sizeof(int), st));
  CK(zcopy(o.diag + 1, ds.err, sizeof(int), st));
  CK(zcopy(o.diag + 2, bb.degc, sizeof(int) * 2, st));
  CK(launch_or_flag(o.diag + 1, bb.degc + 2, st));  // truncation kernels' error flags
  CK(zcopy(o.cand, ds.candidates, sizeof(double), st));
  CK(zcopy(o.cand + 1, bb.mps.lognorm + 1, sizeof(double), st));
  return SPG_OK;
}

// Teacher-forced log-conditionals of the n (= *o.n) returned states along
// their paths, site by site, written to out[b][site] (the per-result check
// against FP64): the search's own right-environment, marginal and update
// kernels with the selection replaced by each state's own next variable.
template <typename T>
int enqueue_forced(spg_ctx* ctx, const spg_problem* P, BoundaryBufs<T>& bb, SearchBufs<T>& sb, const OutStage& o,
                   double* out) {
  cudaStream_t st = ctx->stream;
  DevSearch& ds = sb.ds;
  const int cols = P->cols;
  CK(launch_force_init(ds, o.n, 0, st));
  int cur = 0;
  for (int s = 0; s < P->n; ++s) {
    const int i = s / cols, j = s % cols;
    if (j == 0) CK(right_envs<T>(P, bb, sb, i, cur, st));
    CK(launch_marginals<T>(P->tb, bb.wt, bb.wd, bb.mps, s, ds, sb.bt, cur, st,
                           s < (int)sb.mflops.size() ? sb.mflops[s] * ds.cap : 0.0));
    CK(launch_force(s, ds, cur, o.states, out, st));
    CK(launch_update<T>(P->tb, bb.mps, s, ds, sb.bt, cur, st));
    cur ^= 1;
  }
  return SPG_OK;
}

// A solve is a fixed sequence of stream operations given the problem, the
// parameters and the workspace (everything data-dependent lives on the
// device), so it is captured into one CUDA graph on its second occurrence and
// replayed from then on: one graph launch instead of tens of thousands of
// kernel launches from the host.  One graph, not one per phase: a second graph
// launch on the same stream can hold the host until the first graph has run,
// which serialises the worker threads of spg_solve_batch.  The phase times
// come from GPU timer stamps inside the sequence.  The first occurrence runs
// uncaptured (it also performs the one-time kernel set-up).
// Host structure that a solve's launch sequence depends on: problems equal
// in it can be solved in lockstep (their device tables have one layout and
// every host decision is the same).
bool same_structure(const spg_problem* a, const spg_problem* b) {
  return a->rows == b->rows && a->cols == b->cols && a->n == b->n && a->dmax == b->dmax &&
         a->node_type == b->node_type && a->shift == b->shift && a->bmax == b->bmax && a->lstride == b->lstride &&
         a->ucpl == b->ucpl && a->dev_bytes == b->dev_bytes && a->kbits == b->kbits && a->o_E == b->o_E &&
         a->o_RL == b->o_RL && a->o_RU == b->o_RU && a->o_RA == b->o_RA && a->d == b->d && a->dims == b->dims &&
         a->gD == b->gD && a->keys == b->keys;
}

// The problem as the enqueue functions see it inside a group: instance 0's
// structure with its tables at `tables` (a copy in the group's block).
spg_problem group_view(const spg_problem* P, char* tables) {
  spg_problem V;
  V.ctx = P->ctx;
  V.rows = P->rows;
  V.cols = P->cols;
  V.n = P->n;
  V.dmax = P->dmax;
  V.node_type = P->node_type;
  V.shift = P->shift;
  V.d = P->d;
  V.dims = P->dims;
  V.gD = P->gD;
  V.PL = P->PL;  // host projections read by the choice of right-environment kernel
  V.PR = P->PR;
  V.bmax = P->bmax;
  V.lstride = P->lstride;
  V.ucpl = P->ucpl;
  V.dev_bytes = P->dev_bytes;
  V.kbits = P->kbits;
  V.wspan = P->wspan;
  V.dev = tables;
  V.tb = P->tb;
  const char* from = static_cast<const char*>(P->dev);
  auto re = [&](auto* q) { return reinterpret_cast<decltype(q)>(tables + (reinterpret_cast<const char*>(q) - from)); };
  DevTables& t = V.tb;
  t.d = re(t.d);
  t.E = re(t.E);
  t.PL = re(t.PL);
  t.PR = re(t.PR);
  t.PU = re(t.PU);
  t.PD = re(t.PD);
  t.PG = re(t.PG);
  t.dims = re(t.dims);
  t.RL = re(t.RL);
  t.RU = re(t.RU);
  t.RA = re(t.RA);
  t.gD = re(t.gD);
  t.xsL = re(t.xsL);
  t.xoffL = re(t.xoffL);
  t.keys = re(t.keys);
  t.kshift = re(t.kshift);
  return V;
}

// Sets the calling thread's lockstep group for its lifetime.
struct GroupScope {
  explicit GroupScope(int n, size_t zs, const char* lo) {
    Group& g = group();
    g.n = n;
    g.zs = zs;
    g.lo = lo;
    g.bad = false;
  }
  ~GroupScope() { group() = Group{}; }
};

// Bytes of one instance's block in a lockstep group: the problem's tables,
// then the solve's workspace (1024-byte multiple: the tensor maps of the
// tensor-core products step over instances by it).
template <typename T>
size_t group_stride(const spg_problem* P, const spg_params* prm) {
  Plan pl = make_plan(P, prm->chi, 1);
  const bool drops = prm->merge && prm->droplet_energy >= 0.0;
  const size_t tab = (P->dev_bytes + 1023) & ~size_t(1023);
  const size_t need = boundary_bytes<T>(P, pl, fp64_rows_of<T>(prm, P)) +
                      search_bytes<T>(P, prm->beam, prm->chi, drops) + out_stage_bytes(P, prm->beam);
  return (tab + need + 1023) & ~size_t(1023);
}

// A solve is a fixed sequence of stream operations given the problem, the
// parameters and the workspace (everything data-dependent lives on the
// device), so it is captured into one CUDA graph on its second occurrence and
// replayed from then on: one graph launch instead of tens of thousands of
// kernel launches from the host.  One graph, not one per phase: a second graph
// launch on the same stream can hold the host until the first graph has run,
// which serialises the worker threads of spg_solve_batch.  The phase times
// come from GPU timer stamps inside the sequence.  The first occurrence runs
// uncaptured (it also performs the one-time kernel set-up).
//
// With ng > 1 the problems probs[0 .. ng) (one structure, same_structure)
// are solved in lockstep: instance g's tables (copied from its problem) and
// workspace sit at g * zs in one block, and every launch of the sequence
// covers all ng instances (blockIdx.z), so the group costs the launches of
// one solve and its one-CTA kernels fill ng SMs at once.
template <typename T>
int solve_impl(spg_ctx* ctx, const spg_problem* const* probs, int ng, const spg_params* prm, spg_result* const* Rs) {
  cudaStream_t st = ctx->stream;
  const spg_problem* P0 = probs[0];
  const int chi = prm->chi, cap = prm->beam;
  Plan pl = make_plan(P0, chi, 1);
  const int f64 = fp64_rows_of<T>(prm, P0);
  const spg_mlp* ws = ng == 1 ? warm_of(ctx, P0, prm) : nullptr;
  const bool check = ng == 1 && std::is_same<T, float>::value && prm->check_fp64 != 0;
  const size_t lcn = (size_t)cap * P0->n;  // one log-conditional per (state, site)
  const bool drops = prm->merge && prm->droplet_energy >= 0.0;
  size_t zstride = 0, tab = 0;
  char* gbase = nullptr;
  int rc;
  if (ng == 1) {
    size_t need = boundary_bytes<T>(P0, pl, f64, ws) + search_bytes<T>(P0, cap, chi, drops) + out_stage_bytes(P0, cap);
    if (check)
      need += boundary_bytes<double>(P0, pl) + search_bytes<double>(P0, cap, chi) + 2 * sizeof(double) * lcn + 4096;
    if ((rc = ensure_arena(ctx, need))) return rc;
  } else {
    zstride = group_stride<T>(P0, prm);
    tab = (P0->dev_bytes + 1023) & ~size_t(1023);
    if ((rc = ensure_arena(ctx, zstride * ng + 1024))) return rc;
    gbase = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(ctx->arena) + 1023) & ~uintptr_t(1023));
  }
  // the problem the enqueue functions see (instance 0 of a group: its tables
  // in the group's block)
  spg_problem Vg;
  if (ng > 1) Vg = group_view(P0, gbase);
  const spg_problem* P = ng > 1 ? &Vg : P0;
  Arena ar = ng > 1 ? Arena{gbase + tab, 0, zstride - tab} : Arena{ctx->arena, 0, ctx->arena_bytes};
  BoundaryBufs<T> bb;
  SearchBufs<T> sb;
  if ((rc = carve_boundary<T>(ctx, P, pl, ar, bb, false, f64, ws))) return rc;
  if ((rc = carve_search<T>(ctx, P, cap, chi, ar, sb, false, drops))) return rc;
  sb.tc_rows = renv_tc_rows(P, pl);
  sb.mflops = marginal_flops(P, pl);
  if (drops) {
    sb.ds.dcut = (int64_t)std::floor(std::ldexp(prm->droplet_energy, P->shift));
    sb.ds.dham = prm->droplet_hamming;
  }
  for (int g = 0; g < ng; ++g) Rs[g]->fp64_rows = std::min(f64, std::max(0, P->rows - 1));
  OutStage o;
  const size_t out_used = carve_out(ar, P, cap, o);
  if (!out_used) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  if (sizeof(T) == sizeof(double)) bb.wd = *reinterpret_cast<DevWeights<double>*>(&bb.wt);
  // the plain FP64 boundary and search buffers of the check
  BoundaryBufs<double> bb64;
  SearchBufs<double> sb64;
  double *lc_mixed = nullptr, *lc_fp64 = nullptr;
  if (check) {
    if ((rc = carve_boundary<double>(ctx, P, pl, ar, bb64, false))) return rc;
    if ((rc = carve_search<double>(ctx, P, cap, chi, ar, sb64, false))) return rc;
    bb64.wd = bb64.wt;
    lc_mixed = ar.get<double>(lcn);
    lc_fp64 = ar.get<double>(lcn);
    if (!lc_fp64) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  }
  // host data uploaded outside any capture: the plan's dims, and in a group
  // every instance's tables (problems may have been updated in place)
  for (int g = 0; g < ng; ++g) {
    const size_t zo = (size_t)g * zstride;
    CK(cudaMemcpyAsync(reinterpret_cast<char*>(bb.dimA_dev) + zo, pl.dimA.data(), sizeof(int) * pl.dimA.size(),
                       cudaMemcpyHostToDevice, st));
    if (ng > 1) CK(cudaMemcpyAsync(gbase + zo, probs[g]->dev, P0->dev_bytes, cudaMemcpyDeviceToDevice, st));
  }
  if (check)
    CK(cudaMemcpyAsync(bb64.dimA_dev, pl.dimA.data(), sizeof(int) * pl.dimA.size(), cudaMemcpyHostToDevice, st));

  spg_ctx::Graph* gr_entry = nullptr;
  // a warm-started solve uploads each row's network inputs from the host on
  // the way, so it is never captured
  const bool capturable = !prm->warm_start;
  if (capturable)
    for (auto& e : ctx->graphs)
      if (e.problem == P0 && e.group_n == ng && e.tsize == (int)sizeof(T) && e.arena == ctx->arena &&
          e.arena_bytes == ctx->arena_bytes && std::memcmp(&e.prm, prm, sizeof(spg_params)) == 0)
        gr_entry = &e;
  const bool profiling = kernel_profile().on;
  const long long l0 = thread_launches();
  GroupScope gscope(ng, zstride, gbase);
  // the whole solve: stamp, boundary phase, stamp, search phase, stamp
  auto enqueue_all = [&]() -> int {
    CK(launch_stamp(o.stamp + 0, st));
    int r2 = enqueue_boundary<T>(ctx, P, prm, pl, bb);
    if (r2) return r2;
    CK(launch_stamp(o.stamp + 1, st));
    if ((r2 = enqueue_search<T>(ctx, P, prm, bb, sb, o))) return r2;
    CK(launch_stamp(o.stamp + 2, st));
    if (check) {
      // the returned states' own conditionals: mixed (the boundary MPSs of
      // this solve) against plain FP64 boundary MPSs
      if ((r2 = enqueue_forced<T>(ctx, P, bb, sb, o, lc_mixed))) return r2;
      if ((r2 = enqueue_boundary<double>(ctx, P, prm, pl, bb64))) return r2;
      if ((r2 = enqueue_forced<double>(ctx, P, bb64, sb64, o, lc_fp64))) return r2;
      CK(launch_logmarg_err(lc_mixed, lc_fp64, o.n, P->n, o.err, st));
    } else {
      // 0 in the FP64 mode; NaN (all bits set) when the mixed mode is unchecked
      CK(zfill(o.err, sizeof(T) == sizeof(double) ? 0 : 0xff, sizeof(double), st));
    }
    if (profiling) profile_mark(st);  // closes the last kernel's interval
    if (group().bad) return fail(ctx, SPG_EINVAL, "a launch of the group referenced memory outside its block");
    return SPG_OK;
  };
  // capture into an executable graph (nullptr on failure, rc set)
  auto capture = [&](cudaGraphExec_t* ex) -> int {
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int r2 = enqueue_all();
    const cudaError_t e1 = cudaStreamEndCapture(st, &gr);
    if (r2 || e1 != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return r2 ? r2 : fail(ctx, SPG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
    }
    const cudaError_t e2 = cudaGraphInstantiate(ex, gr, 0);
    cudaGraphDestroy(gr);
    if (e2 != cudaSuccess) return fail(ctx, SPG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
    return SPG_OK;
  };
  long long launches = 0;
  if (profiling && capturable) {
    // captured with the profiler's per-kernel event records as graph nodes,
    // so that the times between them are device times without host gaps
    cudaGraphExec_t ex = nullptr;
    if ((rc = capture(&ex))) return rc;
    CK(cudaGraphLaunch(ex, st));
    launches = thread_launches() - l0;
    CK(cudaStreamSynchronize(st));
    cudaGraphExecDestroy(ex);
  } else if (gr_entry && gr_entry->exec) {
    CK(cudaGraphLaunch(gr_entry->exec, st));
    launches = gr_entry->launches;
  } else if (gr_entry) {
    if ((rc = capture(&gr_entry->exec))) return rc;
    gr_entry->launches = thread_launches() - l0;
    CK(cudaGraphLaunch(gr_entry->exec, st));
    launches = gr_entry->launches;
  } else if (!capturable) {
    if ((rc = enqueue_all())) return rc;
    launches = thread_launches() - l0;
  } else {
    if ((rc = enqueue_all())) return rc;
    launches = thread_launches() - l0;
    if (ctx->graphs.size() >= 8) {  // keep the most recent entries
      auto& old = ctx->graphs.front();
      if (old.exec) cudaGraphExecDestroy(old.exec);
      ctx->graphs.erase(ctx->graphs.begin());
    }
    spg_ctx::Graph ne;
    ne.problem = P0;
    ne.group_n = ng;
    ne.prm = *prm;
    ne.tsize = (int)sizeof(T);
    ne.arena = ctx->arena;
    ne.arena_bytes = ctx->arena_bytes;
    ctx->graphs.push_back(ne);
  }
  // staged outputs into each result's own block (one layout, one copy)
  for (int g = 0; g < ng; ++g) {
    spg_result* R = Rs[g];
    R->launches = launches;
    R->group_size = ng;
    CK(cudaMemcpyAsync(R->blk, reinterpret_cast<const char*>(o.states) + (size_t)g * zstride, out_used,
                       cudaMemcpyDeviceToDevice, st));
    CK(cudaEventRecord(R->ev[2], st));
  }
  return SPG_OK;
}

void drop_graphs(spg_ctx* ctx, const void* problem) {
  for (spg_ctx* c : std::vector<spg_ctx*>{ctx}) {
    for (size_t k = 0; k < c->graphs.size();) {
      auto& e = c->graphs[k];
      if (problem == nullptr || e.problem == problem) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        c->graphs.erase(c->graphs.begin() + k);
      } else {
        ++k;
      }
    }
  }
}

template <typename T>
int debug_marginals_impl(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, int site, int n_prefix,
                         const uint16_t* prefixes, double* out) {
  cudaStream_t st = ctx->stream;
  const int chi = prm->chi;
  const int cap = std::max(1, n_prefix);
  Plan pl = make_plan(P, chi, 1);
  const int f64 = fp64_rows_of<T>(prm, P);
  const spg_mlp* ws = warm_of(ctx, P, prm);
  const size_t need = boundary_bytes<T>(P, pl, f64, ws) + search_bytes<T>(P, cap, chi);
  int rc = ensure_arena(ctx, need);
  if (rc) return rc;
  Arena ar{ctx->arena, 0, ctx->arena_bytes};
  BoundaryBufs<T> bb;
  SearchBufs<T> sb;
  if ((rc = carve_boundary<T>(ctx, P, pl, ar, bb, true, f64, ws))) return rc;
  if ((rc = carve_search<T>(ctx, P, cap, chi, ar, sb))) return rc;
  if (sizeof(T) == sizeof(double)) bb.wd = *reinterpret_cast<DevWeights<double>*>(&bb.wt);
  // rows down to the site's own row: building row i brings B_{i+1} (the MPS
  // the site's conditionals read) to the left-canonical gauge in place, as
  // in a solve, so the conditionals are those the solve computes
  const int row = site / P->cols;
  if ((rc = run_boundary<T>(ctx, P, prm, pl, bb, std::max(1, row)))) return rc;
  DevSearch& ds = sb.ds;
  std::vector<uint16_t> st_h((size_t)cap * P->n, 0);
  for (int k = 0; k < n_prefix; ++k)
    for (int t = 0; t < site; ++t) st_h[(size_t)k * P->n + t] = prefixes[(size_t)k * site + t];
  CK(cudaMemcpyAsync(ds.states[0], st_h.data(), sizeof(uint16_t) * st_h.size(), cudaMemcpyHostToDevice, st));
  int nb[2] = {n_prefix, 0};
  CK(cudaMemcpyAsync(ds.n_beam, nb, sizeof(nb), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(ds.E[0], 0, sizeof(int64_t) * cap, st));
  sb.tc_rows = renv_tc_rows(P, pl);
  CK(right_envs<T>(P, bb, sb, row, 0, st));
  CK(launch_lenv_from_prefix<T>(P->tb, bb.mps, site, ds, sb.bt, 0, st));
  CK(launch_marginals<T>(P->tb, bb.wt, bb.wd, bb.mps, site, ds, sb.bt, 0, st));
  const int d = P->d[site];
  std::vector<double> lc((size_t)cap * P->dmax);
  CK(cudaMemcpyAsync(lc.data(), ds.logc, sizeof(double) * lc.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int k = 0; k < n_prefix; ++k)
    for (int x = 0; x < d; ++x) out[(size_t)k * d + x] = lc[(size_t)k * P->dmax + x];
  return SPG_OK;
}

template <typename T>
int logz_impl(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, double* log_z) {
  cudaStream_t st = ctx->stream;
  Plan pl = make_plan(P, prm->chi, 0);
  const int f64 = fp64_rows_of<T>(prm, P);
  const spg_mlp* ws = warm_of(ctx, P, prm);
  int rc = ensure_arena(ctx, boundary_bytes<T>(P, pl, f64, ws));
  if (rc) return rc;
  Arena ar{ctx->arena, 0, ctx->arena_bytes};
  BoundaryBufs<T> bb;
  if ((rc = carve_boundary<T>(ctx, P, pl, ar, bb, true, f64, ws))) return rc;
  if (sizeof(T) == sizeof(double)) bb.wd = *reinterpret_cast<DevWeights<double>*>(&bb.wt);
  if ((rc = run_boundary<T>(ctx, P, prm, pl, bb, 0))) return rc;
  double* dv = reinterpret_cast<double*>(bb.s1) + 2;
  CK(launch_mps_value<T>(bb.mps, 0, P->cols, dv, st));
  double h[2];
  CK(cudaMemcpyAsync(h, bb.mps.lognorm, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h + 1, dv, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double beta_u = prm->beta * std::ldexp(1.0, -P->shift);
  *log_z = h[0] + std::log(h[1]) - beta_u * P->min_sum;
  return SPG_OK;
}

template <typename T>
int export_impl(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, int row, int fix, void* out,
                int32_t* dims_host) {
  cudaStream_t st = ctx->stream;
  if (row == 0) {  // every row 1 .. rows-1 as it is finished
    Plan pl = make_plan(P, prm->chi, 1);
    const int f64 = fp64_rows_of<T>(prm, P);
    const spg_mlp* ws = warm_of(ctx, P, prm);
    int rc = ensure_arena(ctx, boundary_bytes<T>(P, pl, f64, ws));
    if (rc) return rc;
    Arena ar{ctx->arena, 0, ctx->arena_bytes};
    BoundaryBufs<T> bb;
    if ((rc = carve_boundary<T>(ctx, P, pl, ar, bb, true, f64, ws))) return rc;
    if (sizeof(T) == sizeof(double)) bb.wd = *reinterpret_cast<DevWeights<double>*>(&bb.wt);
    bb.exp_out = static_cast<T*>(out);
    bb.exp_fix = fix;
    if ((rc = run_boundary<T>(ctx, P, prm, pl, bb, 1))) return rc;
    CK(cudaStreamSynchronize(st));
    if (dims_host)
      for (int r = 1; r < P->rows; ++r)
        for (int j = 0; j < P->cols; ++j)
          for (int q = 0; q < 3; ++q)
            dims_host[((size_t)(r - 1) * P->cols + j) * 3 + q] = pl.dimA[((size_t)r * P->cols + j) * 3 + q];
    return SPG_OK;
  }
  Plan pl = make_plan(P, prm->chi, row);
  const int f64 = fp64_rows_of<T>(prm, P);
  const spg_mlp* ws = warm_of(ctx, P, prm);
  int rc = ensure_arena(ctx, boundary_bytes<T>(P, pl, f64, ws));
  if (rc) return rc;
  Arena ar{ctx->arena, 0, ctx->arena_bytes};
  BoundaryBufs<T> bb;
  if ((rc = carve_boundary<T>(ctx, P, pl, ar, bb, true, f64, ws))) return rc;
  if (sizeof(T) == sizeof(double)) bb.wd = *reinterpret_cast<DevWeights<double>*>(&bb.wt);
  if ((rc = run_boundary<T>(ctx, P, prm, pl, bb, row))) return rc;
  CK(launch_export_row<T>(bb.mps, row, P->cols, prm->chi, static_cast<T*>(out),
                          bb.dimA_dev + (size_t)row * P->cols * 3, fix, st));
  CK(cudaStreamSynchronize(st));
  if (dims_host)
    for (int j = 0; j < P->cols; ++j)
      for (int q = 0; q < 3; ++q) dims_host[j * 3 + q] = pl.dimA[((size_t)row * P->cols + j) * 3 + q];
  return SPG_OK;
}

template <typename T>
int trace_impl(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, int row, int init, int n_sweeps,
               double* out) {
  cudaStream_t st = ctx->stream;
  spg_params base = *prm;  // the rows below are built as a plain solve builds them
  base.warm_start = 0;
  spg_params net = *prm;
  net.warm_start = 1;
  const spg_mlp* ws = init >= 1 ? warm_of(ctx, P, &net) : nullptr;
  if (init >= 1 && !ws) return fail(ctx, SPG_EINVAL, "no warm-start network for this problem and chi");
  Plan pl = make_plan(P, prm->chi, row);
  const int f64 = fp64_rows_of<T>(prm, P);
  int rc = ensure_arena(ctx, boundary_bytes<T>(P, pl, f64, ws));
  if (rc) return rc;
  Arena ar{ctx->arena, 0, ctx->arena_bytes};
  BoundaryBufs<T> bb;
  if ((rc = carve_boundary<T>(ctx, P, pl, ar, bb, true, f64, nullptr))) return rc;
  if (sizeof(T) == sizeof(double)) bb.wd = *reinterpret_cast<DevWeights<double>*>(&bb.wt);
  if ((rc = run_boundary<T>(ctx, P, &base, pl, bb, row + 1))) return rc;
  if (ws) {
    // the network's buffers, carved after the boundary's
    bb.ws = ws;
    bb.wsX = ar.get<float>((size_t)P->cols * SPG_WS_FEATURES);
    bb.wsY = ar.get<float>((size_t)P->cols * MAXP * prm->chi * prm->chi);
    bb.wswork = ar.get<float>(mlp_infer_elems(ws, P->cols));
    if (!bb.wswork) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  }
  // init 2: the zipper's trace, then the network's on the same B_{row+1}
  // (its left-canonical QR again is a change of gauge only)
  const int first = init == 2 ? 0 : init, last = init == 2 ? 1 : init;
  for (int mode = first; mode <= last; ++mode) {
    if ((rc = build_row<T>(ctx, P, prm, pl, bb, row, mode == 1))) return rc;
    double* o = out + (size_t)(mode - first) * n_sweeps;
    for (int k = 0; k < n_sweeps; ++k) {
      CK(variational_sweeps<T>(P->tb, bb.wt, bb.mps, row, P->cols, pl.dimA.data(), P->dims.data(), P->d.data(),
                               P->gD.data(), 1, bb.swork, bb.sdbl, st));
      double ln[2];
      CK(cudaMemcpyAsync(ln, bb.mps.lognorm + row, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      o[k] = ln[0] - ln[1];
    }
  }
  return SPG_OK;
}

// out[b][s] = in[b][map[s]] for b < *n (the states of a transformed lattice
// read back on the original sites)
__global__ void k_permute_sites(const uint16_t* __restrict__ in, uint16_t* __restrict__ out, const int* n_dev,
                                int N, const int* __restrict__ map) {
  const size_t tot = (size_t)(*n_dev) * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / N;
    const int s = (int)(e % N);
    out[e] = in[b * N + map[s]];
  }
}

}  // namespace

// ================================================================== C ABI
extern "C" {

int spg_version(void) { return 100; }

int spg_lattice_site_map(int32_t rows, int32_t cols, int32_t k, int32_t* site_map, int32_t* new_rows,
                         int32_t* new_cols) {
  if (rows < 1 || cols < 1 || k < 0 || k > 7 || !site_map) return SPG_EINVAL;
  const int R = (k & 4) ? cols : rows, C = (k & 4) ? rows : cols;
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) {
      int a = i, b = j;
      if (k & 4) {
        a = j;
        b = i;
      }
      if (k & 1) a = R - 1 - a;
      if (k & 2) b = C - 1 - b;
      site_map[i * cols + j] = a * C + b;
    }
  if (new_rows) *new_rows = R;
  if (new_cols) *new_cols = C;
  return SPG_OK;
}

int spg_params_default(spg_params* p) {
  if (!p) return SPG_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->beta = 1.0;
  p->chi = 16;
  p->num_sweeps = 0;
  p->beam = 256;
  p->precision = SPG_FP64;
  p->cut_off_prob = 0.0;
  p->svd_iters = -1;
  p->merge = 1;
  p->fp64_rows = -1;
  p->check_fp64 = 0;
  p->droplet_hamming = 0;
  p->droplet_energy = -1.0;
  return SPG_OK;
}

int spg_create(spg_ctx** out, int device, void* cuda_stream) {
  if (!out) return SPG_EINVAL;
  *out = nullptr;
  spg_ctx* ctx = new (std::nothrow) spg_ctx();
  if (!ctx) return SPG_ENOMEM;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    delete ctx;
    return SPG_ECUDA;
  }
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return SPG_ECUDA;
  }
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return SPG_ECUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return SPG_OK;
}

}  // extern "C"

static void ctx_free(spg_ctx* ctx) {
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  drop_graphs(ctx, nullptr);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

void spg::ctx_retain(spg_ctx* ctx) {
  std::lock_guard<std::mutex> lock(ctx->life_mu);
  ++ctx->children;
}

void spg::ctx_release(spg_ctx* ctx) {
  bool last;
  {
    std::lock_guard<std::mutex> lock(ctx->life_mu);
    --ctx->children;
    last = ctx->closing && ctx->children == 0;
  }
  if (last) ctx_free(ctx);
}

extern "C" {

void spg_destroy(spg_ctx* ctx) {
  if (!ctx) return;
  for (spg_ctx* w : ctx->workers) spg_destroy(w);
  ctx->workers.clear();
  bool now;
  {
    std::lock_guard<std::mutex> lock(ctx->life_mu);
    ctx->closing = true;
    now = ctx->children == 0;
  }
  if (now) ctx_free(ctx);
}

const char* spg_last_error(const spg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

}  // extern "C"

namespace {
// The Ising form's tables (S1); upload = false builds the host tables only.
int build_ising(spg_ctx* ctx, int32_t n_spins, int32_t n_edges, const int32_t* ei, const int32_t* ej,
                const double* J, const double* h, const int32_t* cluster_of_spin, int32_t grid_rows,
                int32_t grid_cols, const int32_t* cluster_row, const int32_t* cluster_col, int32_t energy_shift,
                int32_t node_type, spg_problem** out, bool upload) {
  if (!ctx || !out) return SPG_EINVAL;
  *out = nullptr;
  if (n_spins <= 0 || n_edges < 0 || grid_rows <= 0 || grid_cols <= 0 || !cluster_of_spin || !cluster_row ||
      !cluster_col || (n_edges > 0 && (!ei || !ej || !J)))
    return fail(ctx, SPG_EINVAL, "bad sizes or NULL arrays");
  if (energy_shift < 0 || energy_shift > 52) return fail(ctx, SPG_EINVAL, "energy_shift outside 0..52");
  if (node_type != SPG_SQUARE && node_type != SPG_KING) return fail(ctx, SPG_EINVAL, "bad node_type");
  if (grid_cols > SPG_MAX_COLS) return fail(ctx, SPG_EUNSUPPORTED, "grid wider than the built limit");
  const int n = grid_rows * grid_cols;
  std::vector<int> site_of_cluster(n, -1), used(n, 0);
  for (int c = 0; c < n; ++c) {
    const int r = cluster_row[c], cc = cluster_col[c];
    if (r < 0 || r >= grid_rows || cc < 0 || cc >= grid_cols) return fail(ctx, SPG_EINVAL, "cluster outside grid");
    const int s = r * grid_cols + cc;
    if (used[s]) return fail(ctx, SPG_EINVAL, "two clusters on one grid cell");
    used[s] = 1;
    site_of_cluster[c] = s;
  }
  std::vector<int> site_of_spin(n_spins);
  std::vector<std::vector<int>> spins(n);
  for (int i = 0; i < n_spins; ++i) {
    const int c = cluster_of_spin[i];
    if (c < 0 || c >= n) return fail(ctx, SPG_EINVAL, "cluster id out of range");
    site_of_spin[i] = site_of_cluster[c];
    spins[site_of_cluster[c]].push_back(i);  // ascending spin index
  }
  const double scale = std::ldexp(1.0, energy_shift);
  auto to_int = [&](double v, int64_t* o) {
    const double x = v * scale;
    if (!std::isfinite(x) || std::rint(x) != x || std::fabs(x) >= 4503599627370496.0) return false;
    *o = (int64_t)x;
    return true;
  };
  spg_problem* P = new (std::nothrow) spg_problem();
  if (!P) return SPG_ENOMEM;
  P->ctx = ctx;
  P->rows = grid_rows;
  P->cols = grid_cols;
  P->n = n;
  P->node_type = node_type;
  P->shift = energy_shift;
  P->d.resize(n);
  int dmax = 1;
  std::vector<int> pos(n_spins);
  for (int s = 0; s < n; ++s) {
    const int k = (int)spins[s].size();
    if (k > 8) {
      delete P;
      return fail(ctx, SPG_EUNSUPPORTED, "cluster with more than 8 spins");
    }
    P->d[s] = 1 << k;
    dmax = std::max(dmax, P->d[s]);
    for (int q = 0; q < k; ++q) pos[spins[s][q]] = q;
  }
  P->dmax = dmax;
  P->E.assign((size_t)n * dmax, 0);
  auto spin = [](int x, int q) { return ((x >> q) & 1) ? 1 : -1; };
  for (int i = 0; i < n_spins; ++i) {
    int64_t hv = 0;
    if (h && !to_int(h[i], &hv)) {
      delete P;
      return fail(ctx, SPG_EINEXACT, "h not on the 2^-energy_shift grid");
    }
    if (hv == 0) continue;
    const int s = site_of_spin[i];
    for (int x = 0; x < P->d[s]; ++x) P->E[(size_t)s * dmax + x] += hv * spin(x, pos[i]);
  }
  struct Coupler {
    int pa, pb;
    int64_t J;
  };
  std::map<std::pair<int, int>, std::vector<Coupler>> inter;
  for (int e = 0; e < n_edges; ++e) {
    const int a = ei[e], b = ej[e];
    if (a < 0 || a >= n_spins || b < 0 || b >= n_spins || a == b) {
      delete P;
      return fail(ctx, SPG_EINVAL, "bad coupling endpoints");
    }
    int64_t Jv;
    if (!to_int(J[e], &Jv)) {
      delete P;
      return fail(ctx, SPG_EINEXACT, "J not on the 2^-energy_shift grid");
    }
    int sa = site_of_spin[a], sb = site_of_spin[b];
    if (sa == sb) {
      for (int x = 0; x < P->d[sa]; ++x) P->E[(size_t)sa * dmax + x] += Jv * spin(x, pos[a]) * spin(x, pos[b]);
      continue;
    }
    int pa = pos[a], pb = pos[b];
    if (sa > sb) {
      std::swap(sa, sb);
      std::swap(pa, pb);
    }
    const int dr = std::abs(sa / grid_cols - sb / grid_cols), dc = std::abs(sa % grid_cols - sb % grid_cols);
    const bool adj = node_type == SPG_SQUARE ? (dr + dc == 1) : (std::max(dr, dc) == 1);
    if (!adj) {
      delete P;
      return fail(ctx, SPG_EINVAL, "coupling between clusters that are not grid neighbours");
    }
    inter[{sa, sb}].push_back({pa, pb, Jv});
  }
  // warm-start coupling blocks per site: couplings between the cluster's
  // spin positions, fields, summed couplings to the cluster below and to the
  // cluster on the right, by spin position (king's diagonals not included)
  P->wsblk.assign((size_t)n * SPG_WS_PER_CLUSTER, 0.0);
  if (h)
    for (int i = 0; i < n_spins; ++i) P->wsblk[(size_t)site_of_spin[i] * SPG_WS_PER_CLUSTER + 28 + pos[i]] += h[i];
  for (int e = 0; e < n_edges; ++e) {
    const int a = ei[e], b = ej[e];
    const int sa = site_of_spin[a], sb = site_of_spin[b];
    const int ra = sa / grid_cols, ca = sa % grid_cols, rb = sb / grid_cols, cb = sb % grid_cols;
    if (sa == sb) {
      const int q1 = std::min(pos[a], pos[b]), q2 = std::max(pos[a], pos[b]);
      P->wsblk[(size_t)sa * SPG_WS_PER_CLUSTER + ws_pair_slot(q1, q2)] += J[e];
    } else if (ca == cb && std::abs(ra - rb) == 1) {
      const int up = ra < rb ? a : b;
      P->wsblk[(size_t)site_of_spin[up] * SPG_WS_PER_CLUSTER + 36 + pos[up]] += J[e];
    } else if (ra == rb && std::abs(ca - cb) == 1) {
      const int left = ca < cb ? a : b;
      P->wsblk[(size_t)site_of_spin[left] * SPG_WS_PER_CLUSTER + 44 + pos[left]] += J[e];
    }
  }
  // pairwise tables over the spins that carry couplers, then projectors
  std::map<std::pair<int, int>, EdgeTab> edges;
  for (auto& kv : inter) {
    const int m = kv.first.first, nn = kv.first.second;
    std::vector<int> Sm, Sn;
    for (auto& c : kv.second) {
      Sm.push_back(c.pa);
      Sn.push_back(c.pb);
    }
    std::sort(Sm.begin(), Sm.end());
    Sm.erase(std::unique(Sm.begin(), Sm.end()), Sm.end());
    std::sort(Sn.begin(), Sn.end());
    Sn.erase(std::unique(Sn.begin(), Sn.end()), Sn.end());
    const int am = 1 << Sm.size(), an = 1 << Sn.size();
    // sub-configuration of a state: bits of the involved spins, ascending
    auto sub = [](int x, const std::vector<int>& S) {
      int a = 0;
      for (size_t q = 0; q < S.size(); ++q) a |= ((x >> S[q]) & 1) << q;
      return a;
    };
    std::vector<int64_t> Tsub((size_t)am * an, 0);
    for (auto& c : kv.second) {
      const int qa = (int)(std::lower_bound(Sm.begin(), Sm.end(), c.pa) - Sm.begin());
      const int qb = (int)(std::lower_bound(Sn.begin(), Sn.end(), c.pb) - Sn.begin());
      for (int a = 0; a < am; ++a)
        for (int b = 0; b < an; ++b) Tsub[(size_t)a * an + b] += c.J * spin(a, qa) * spin(b, qb);
    }
    EdgeTab sube;
    if (!reduce_full(Tsub, am, an, sube)) {
      delete P;
      return fail(ctx, SPG_EUNSUPPORTED, "pairwise table with more than 16 distinct rows or columns");
    }
    // first occurrence over x ascending equals first occurrence over the
    // sub-configuration ascending (the embedding keeps bit order)
    EdgeTab e;
    e.Dm = sube.Dm;
    e.Dn = sube.Dn;
    e.R = sube.R;
    e.Pm.resize(P->d[m]);
    e.Pn.resize(P->d[nn]);
    for (int x = 0; x < P->d[m]; ++x) e.Pm[x] = sube.Pm[sub(x, Sm)];
    for (int y = 0; y < P->d[nn]; ++y) e.Pn[y] = sube.Pn[sub(y, Sn)];
    edges[{m, nn}] = e;
  }
  int rc = finish_problem(ctx, P, edges, upload);
  if (rc) {
    spg_problem_destroy(P);
    return rc;
  }
  P->raw.n_spins = n_spins;
  P->raw.ei.assign(ei, ei + n_edges);
  P->raw.ej.assign(ej, ej + n_edges);
  P->raw.J.assign(J, J + n_edges);
  if (h) P->raw.h.assign(h, h + n_spins);
  P->raw.cos.assign(cluster_of_spin, cluster_of_spin + n_spins);
  P->raw.crow.assign(cluster_row, cluster_row + n);
  P->raw.ccol.assign(cluster_col, cluster_col + n);
  ctx_retain(ctx);
  P->counted = true;
  *out = P;
  return SPG_OK;
}
}  // namespace

extern "C" {

int spg_problem_ising(spg_ctx* ctx, int32_t n_spins, int32_t n_edges, const int32_t* ei, const int32_t* ej,
                      const double* J, const double* h, const int32_t* cluster_of_spin, int32_t grid_rows,
                      int32_t grid_cols, const int32_t* cluster_row, const int32_t* cluster_col,
                      int32_t energy_shift, int32_t node_type, spg_problem** out) {
  return build_ising(ctx, n_spins, n_edges, ei, ej, J, h, cluster_of_spin, grid_rows, grid_cols, cluster_row,
                     cluster_col, energy_shift, node_type, out, true);
}

int spg_problem_update_ising(spg_problem* P, const double* J, const double* h) {
  if (!P || !P->ctx) return SPG_EINVAL;
  spg_ctx* ctx = P->ctx;
  const auto& rw = P->raw;
  if (rw.potts) return fail(ctx, SPG_EINVAL, "spg_problem_update_ising: not an Ising problem");
  if (!J && !rw.ei.empty()) return fail(ctx, SPG_EINVAL, "spg_problem_update_ising: J is NULL");
  spg_problem* Q = nullptr;
  int rc = build_ising(ctx, rw.n_spins, (int32_t)rw.ei.size(), rw.ei.data(), rw.ej.data(), J, h, rw.cos.data(),
                       P->rows, P->cols, rw.crow.data(), rw.ccol.data(), P->shift, P->node_type, &Q, false);
  if (rc) return rc;
  const bool same = Q->d == P->d && Q->dmax == P->dmax && Q->PL == P->PL && Q->PR == P->PR && Q->PU == P->PU &&
                    Q->PD == P->PD && Q->PG == P->PG && Q->dims == P->dims && Q->gD == P->gD && Q->xsL == P->xsL &&
                    Q->xoffL == P->xoffL && Q->keys == P->keys && Q->kbits == P->kbits && Q->bmax == P->bmax &&
                    Q->lstride == P->lstride && Q->RL.size() == P->RL.size();
  if (!same) {
    spg_problem_destroy(Q);
    return fail(ctx, SPG_EUNSUPPORTED,
                "spg_problem_update_ising: the new couplings change the tables' structure; build a new problem");
  }
  // the solves that read the old tables finish first
  if (cudaSetDevice(ctx->device) != cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    spg_problem_destroy(Q);
    return fail(ctx, SPG_ECUDA, "spg_problem_update_ising: synchronisation failed");
  }
  for (spg_ctx* w : ctx->workers) cudaStreamSynchronize(w->stream);
  P->E.swap(Q->E);
  P->RL.swap(Q->RL);
  P->RU.swap(Q->RU);
  P->RA.swap(Q->RA);
  P->min_sum = Q->min_sum;
  P->wsblk.swap(Q->wsblk);
  P->raw.J.swap(Q->raw.J);
  P->raw.h.swap(Q->raw.h);
  spg_problem_destroy(Q);
  char* base = (char*)P->dev;
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(base + P->o_E, P->E.data(), sizeof(int64_t) * P->E.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + P->o_RL, P->RL.data(), sizeof(int64_t) * P->RL.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + P->o_RU, P->RU.data(), sizeof(int64_t) * P->RU.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(base + P->o_RA, P->RA.data(), sizeof(int64_t) * P->RA.size(), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return SPG_OK;
}

int spg_problem_potts(spg_ctx* ctx, int32_t grid_rows, int32_t grid_cols, const int32_t* d, const int64_t* local_E,
                      int32_t n_edges, const int32_t* em, const int32_t* en, const int64_t* pair_E,
                      int32_t energy_shift, int32_t node_type, spg_problem** out) {
  if (!ctx || !out) return SPG_EINVAL;
  *out = nullptr;
  if (grid_rows <= 0 || grid_cols <= 0 || !d || !local_E || n_edges < 0 || (n_edges > 0 && (!em || !en || !pair_E)))
    return fail(ctx, SPG_EINVAL, "bad sizes or NULL arrays");
  if (node_type != SPG_SQUARE && node_type != SPG_KING) return fail(ctx, SPG_EINVAL, "bad node_type");
  if (grid_cols > SPG_MAX_COLS) return fail(ctx, SPG_EUNSUPPORTED, "grid wider than the built limit");
  const int n = grid_rows * grid_cols;
  spg_problem* P = new (std::nothrow) spg_problem();
  if (!P) return SPG_ENOMEM;
  P->ctx = ctx;
  P->rows = grid_rows;
  P->cols = grid_cols;
  P->n = n;
  P->node_type = node_type;
  P->shift = energy_shift;
  P->d.assign(d, d + n);
  int dmax = 1;
  for (int s = 0; s < n; ++s) {
    if (d[s] < 1 || d[s] > SPG_MAX_STATES) {
      delete P;
      return fail(ctx, d[s] < 1 ? SPG_EINVAL : SPG_EUNSUPPORTED, "states per site outside 1..256");
    }
    dmax = std::max(dmax, d[s]);
  }
  P->dmax = dmax;
  P->E.assign((size_t)n * dmax, 0);
  size_t off = 0;
  for (int s = 0; s < n; ++s)
    for (int x = 0; x < d[s]; ++x) P->E[(size_t)s * dmax + x] = local_E[off++];
  std::map<std::pair<int, int>, std::vector<int64_t>> full;
  off = 0;
  for (int k = 0; k < n_edges; ++k) {
    int m = em[k], nn = en[k];
    if (m < 0 || m >= n || nn < 0 || nn >= n || m == nn) {
      delete P;
      return fail(ctx, SPG_EINVAL, "bad edge endpoints");
    }
    const int dm = d[m], dn = d[nn];
    const int64_t* T = pair_E + off;
    off += (size_t)dm * dn;
    const int dr = std::abs(m / grid_cols - nn / grid_cols), dc = std::abs(m % grid_cols - nn % grid_cols);
    const bool adj = node_type == SPG_SQUARE ? (dr + dc == 1) : (std::max(dr, dc) == 1);
    if (!adj) {
      delete P;
      return fail(ctx, SPG_EINVAL, "pairwise table between sites that are not grid neighbours");
    }
    const bool swap = m > nn;
    const int a = swap ? nn : m, b = swap ? m : nn;
    auto& acc = full[{a, b}];
    if (acc.empty()) acc.assign((size_t)d[a] * d[b], 0);
    for (int x = 0; x < dm; ++x)
      for (int y = 0; y < dn; ++y) {
        const int64_t v = T[(size_t)x * dn + y];
        if (swap)
          acc[(size_t)y * dm + x] += v;
        else
          acc[(size_t)x * dn + y] += v;
      }
  }
  std::map<std::pair<int, int>, EdgeTab> edges;
  for (auto& kv : full) {
    EdgeTab e;
    if (!reduce_full(kv.second, d[kv.first.first], d[kv.first.second], e)) {
      delete P;
      return fail(ctx, SPG_EUNSUPPORTED, "pairwise table with more than 16 distinct rows or columns");
    }
    edges[kv.first] = e;
  }
  int rc = finish_problem(ctx, P, edges);
  if (rc) {
    spg_problem_destroy(P);
    return rc;
  }
  P->raw.potts = true;
  P->raw.d.assign(d, d + n);
  size_t nloc = 0, npair = 0;
  for (int s2 = 0; s2 < n; ++s2) nloc += (size_t)d[s2];
  for (int k = 0; k < n_edges; ++k) npair += (size_t)d[em[k]] * d[en[k]];
  P->raw.local.assign(local_E, local_E + nloc);
  P->raw.em.assign(em, em + n_edges);
  P->raw.en.assign(en, en + n_edges);
  P->raw.pair.assign(pair_E, pair_E + npair);
  ctx_retain(ctx);
  P->counted = true;
  *out = P;
  return SPG_OK;
}

void spg_problem_destroy(spg_problem* P) {
  if (!P) return;
  if (P->ctx) {
    cudaSetDevice(P->ctx->device);
    drop_graphs(P->ctx, P);
    for (spg_ctx* w : P->ctx->workers) drop_graphs(w, P);
  }
  if (P->dev) {
    cudaSetDevice(P->ctx->device);
    cudaStreamSynchronize(P->ctx->stream);
    cudaFree(P->dev);
  }
  spg_ctx* ctx = P->counted ? P->ctx : nullptr;
  delete P;
  if (ctx) ctx_release(ctx);
}

int spg_problem_shape(const spg_problem* P, int32_t* rows, int32_t* cols, int32_t* d_per_site) {
  if (!P) return SPG_EINVAL;
  if (rows) *rows = P->rows;
  if (cols) *cols = P->cols;
  if (d_per_site)
    for (int s = 0; s < P->n; ++s) d_per_site[s] = P->d[s];
  return SPG_OK;
}

}  // extern "C"

namespace {

// A result handle with its device block (the staged outputs' layout).
int make_result(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, spg_result** out) {
  *out = nullptr;
  spg_result* R = new (std::nothrow) spg_result();
  if (!R) return SPG_ENOMEM;
  R->ctx = ctx;
  ctx_retain(ctx);
  R->N = P->n;
  R->cap = prm->beam;
  cudaStream_t st = ctx->stream;
  // completion event (the phase times come from GPU timer stamps)
  if (cudaEventCreateWithFlags(&R->ev[2], cudaEventDisableTiming) != cudaSuccess) {
    spg_result_destroy(R);
    return fail(ctx, SPG_ECUDA, "event create");
  }
  const size_t bytes = out_stage_bytes(P, R->cap);
  if (cudaMallocAsync(&R->blk, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    R->blk = nullptr;
    spg_result_destroy(R);
    return fail(ctx, SPG_ENOMEM, "result allocation failed");
  }
  Arena ar{static_cast<char*>(R->blk), 0, bytes};
  OutStage o;
  R->blk_used = carve_out(ar, P, R->cap, o);
  R->d_states = o.states;
  R->d_E = o.E;
  R->d_logp = o.logp;
  R->d_n = o.n;
  R->d_diag = o.diag;
  R->d_cand = o.cand;
  R->d_stamp = o.stamp;
  R->d_err = o.err;
  R->d_dn = o.dn;
  R->d_dE = o.dE;
  R->d_dst = o.dst;
  *out = R;
  return SPG_OK;
}

bool runs_fp64(const spg_problem* P, const spg_params* prm) {
  return prm->precision == SPG_FP64 || fp32_range_exceeded(P, prm);
}

// Whether problems a and b with parameters pa, pb can share a lockstep group.
bool groupable(const spg_problem* a, const spg_params* pa, const spg_problem* b, const spg_params* pb) {
  return std::memcmp(pa, pb, sizeof(spg_params)) == 0 && !pa->warm_start && !pa->check_fp64 &&
         runs_fp64(a, pa) == runs_fp64(b, pb) && same_structure(a, b);
}

// Lockstep group of n problems (n >= 1) on ctx: results in out[0 .. n).
int solve_group(spg_ctx* ctx, int n, const spg_problem* const* probs, const spg_params* prm, spg_result** out) {
  for (int g = 0; g < n; ++g) out[g] = nullptr;
  for (int g = 0; g < n; ++g) {
    const int rc = make_result(ctx, probs[g], prm, &out[g]);
    if (rc) {
      for (int h = 0; h < n; ++h) {
        spg_result_destroy(out[h]);
        out[h] = nullptr;
      }
      return rc;
    }
  }
  const bool use64 = runs_fp64(probs[0], prm);
  for (int g = 0; g < n; ++g) out[g]->precision_used = use64 ? SPG_FP64 : SPG_MIXED;
  const int rc = use64 ? solve_impl<double>(ctx, probs, n, prm, out) : solve_impl<float>(ctx, probs, n, prm, out);
  if (rc) {
    for (int g = 0; g < n; ++g) {
      spg_result_destroy(out[g]);
      out[g] = nullptr;
    }
  }
  return rc;
}

// Most instances of one lockstep group: one per SM fills the GPU with the
// group's one-CTA kernels in a single wave; at most half the free device
// memory; the grid limit of the state-batched sweep products (states x
// instances < 65536).
// Largest state batch (grid.z of one instance) of the sweeps' products.
int max_state_batch(const spg_problem* P) {
  int m = 1;
  for (int s = 0; s < P->n; ++s) {
    const int* dm = &P->dims[(size_t)s * DIMW];
    m = std::max(m, std::max(P->d[s], MAXP * std::max(dm[D_DR], dm[D_NL])));
  }
  return m;
}

int group_cap(const spg_ctx* ctx, const spg_problem* P, const spg_params* prm) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const size_t per = runs_fp64(P, prm) ? group_stride<double>(P, prm) : group_stride<float>(P, prm);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = 0;
  }
  const size_t by_mem = per ? (fr / 2 + (size_t)ctx->arena_bytes) / per : 1;
  int cap = std::max(1, sms);
  cap = (int)std::min<size_t>((size_t)cap, std::max<size_t>(1, by_mem));
  cap = std::min(cap, std::max(1, 65535 / max_state_batch(P)));
  return std::min(cap, SPG_MAX_GROUP);
}

}  // namespace

extern "C" {

int spg_solve(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, spg_result** out) {
  if (!ctx || !P || !out) return SPG_EINVAL;
  *out = nullptr;
  int rc = check_params(ctx, P, prm);
  if (rc) return rc;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SPG_ECUDA, "cudaSetDevice failed");
  return solve_group(ctx, 1, &P, prm, out);
}

int spg_solve_group(spg_ctx* ctx, int32_t n, const spg_problem* const* probs, const spg_params* prm,
                    spg_result** out) {
  if (!ctx || !probs || !prm || !out || n < 1) return SPG_EINVAL;
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  if (n > SPG_MAX_GROUP) return fail(ctx, SPG_EUNSUPPORTED, "group larger than SPG_MAX_GROUP");
  for (int i = 0; i < n; ++i) {
    if (!probs[i]) return fail(ctx, SPG_EINVAL, "NULL problem in group");
    const int rc = check_params(ctx, probs[i], prm);
    if (rc) return rc;
  }
  if (prm->warm_start || prm->check_fp64)
    return fail(ctx, SPG_EUNSUPPORTED, "warm_start and check_fp64 solves are not grouped");
  for (int i = 1; i < n; ++i)
    if (!groupable(probs[0], prm, probs[i], prm))
      return fail(ctx, SPG_EINVAL, "group item " + std::to_string(i) + " differs in structure from item 0");
  if ((long long)n * max_state_batch(probs[0]) > 65535)
    return fail(ctx, SPG_EUNSUPPORTED, "group too large for this lattice's state batches (n x states < 65536)");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SPG_ECUDA, "cudaSetDevice failed");
  return solve_group(ctx, n, probs, prm, out);
}

int spg_solve_batch(spg_ctx* ctx, int32_t n, const spg_problem* const* probs, const spg_params* prms,
                    spg_result** out) {
  if (!ctx || !probs || !prms || !out || n < 1) return SPG_EINVAL;
  for (int i = 0; i < n; ++i) {
    out[i] = nullptr;
    if (!probs[i]) return fail(ctx, SPG_EINVAL, "NULL problem in batch");
    const int rc = check_params(ctx, probs[i], &prms[i]);
    if (rc) return rc;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SPG_ECUDA, "cudaSetDevice failed");
  // lockstep groups: items of one structure and equal parameters, in order of
  // first occurrence, at most group_cap (or prm.group_max) per group, the
  // items of a class spread evenly over its groups
  std::vector<std::vector<int>> classes;
  for (int i = 0; i < n; ++i) {
    bool placed = false;
    if (prms[i].group_max != 1)
      for (auto& c : classes)
        if (prms[c[0]].group_max != 1 && groupable(probs[c[0]], &prms[c[0]], probs[i], &prms[i])) {
          c.push_back(i);
          placed = true;
          break;
        }
    if (!placed) classes.push_back({i});
  }
  std::vector<std::vector<int>> groups;
  for (auto& c : classes) {
    const int gmax = prms[c[0]].group_max > 0
                         ? std::min(std::min(prms[c[0]].group_max, SPG_MAX_GROUP),
                                    std::max(1, 65535 / max_state_batch(probs[c[0]])))
                         : group_cap(ctx, probs[c[0]], &prms[c[0]]);
    const int ng = ((int)c.size() + gmax - 1) / gmax;
    for (int k = 0; k < ng; ++k) {
      std::vector<int> g;
      for (size_t q = (size_t)k * c.size() / ng; q < (size_t)(k + 1) * c.size() / ng; ++q) g.push_back(c[q]);
      groups.push_back(std::move(g));
    }
  }
  const int G = (int)groups.size();
  const int K = std::min(G, 32);
  while ((int)ctx->workers.size() < K) {
    spg_ctx* w = nullptr;
    const int rc = spg_create(&w, ctx->device, nullptr);
    if (rc) return fail(ctx, rc, "worker context creation failed");
    ctx->workers.push_back(w);
  }
  for (spg_ctx* w : ctx->workers) w->warm = ctx->warm;
  // the batch starts after the work already on the context's stream
  cudaEvent_t start;
  CK(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  CK(cudaEventRecord(start, ctx->stream));
  for (int k = 0; k < K; ++k) CK(cudaStreamWaitEvent(ctx->workers[k]->stream, start, 0));
  std::vector<int> rcs(G, SPG_OK);
  std::vector<std::thread> threads;
  for (int k = 0; k < K; ++k)
    threads.emplace_back([&, k] {
      cudaSetDevice(ctx->device);
      for (int q = k; q < G; q += K) {
        const std::vector<int>& g = groups[q];
        std::vector<const spg_problem*> gp(g.size());
        std::vector<spg_result*> gr(g.size(), nullptr);
        for (size_t i = 0; i < g.size(); ++i) gp[i] = probs[g[i]];
        rcs[q] = solve_group(ctx->workers[k], (int)g.size(), gp.data(), &prms[g[0]], gr.data());
        for (size_t i = 0; i < g.size(); ++i) out[g[i]] = gr[i];
      }
    });
  for (auto& t : threads) t.join();
  // later work on the context's stream runs after the batch
  for (int k = 0; k < K; ++k) {
    cudaEvent_t done;
    CK(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    CK(cudaEventRecord(done, ctx->workers[k]->stream));
    CK(cudaStreamWaitEvent(ctx->stream, done, 0));
    cudaEventDestroy(done);
  }
  cudaEventDestroy(start);
  for (int q = 0; q < G; ++q)
    if (rcs[q] != SPG_OK) {
      const std::string msg = ctx->workers[q % K]->err;
      for (int j = 0; j < n; ++j) {
        spg_result_destroy(out[j]);
        out[j] = nullptr;
      }
      return fail(ctx, rcs[q], "batch item " + std::to_string(groups[q][0]) + ": " + msg);
    }
  return SPG_OK;
}

static int fetch(spg_result* R) {
  spg_ctx* ctx = R->ctx;
  if (R->fetched) return SPG_OK;
  CK(cudaSetDevice(ctx->device));
  CK(cudaEventSynchronize(R->ev[2]));
  CK(cudaMemcpy(&R->n, R->d_n, sizeof(int), cudaMemcpyDeviceToHost));
  unsigned long long ts[3];
  CK(cudaMemcpy(ts, R->d_stamp, sizeof(ts), cudaMemcpyDeviceToHost));
  R->ms_boundary = (float)((double)(ts[1] - ts[0]) * 1e-6);
  R->ms_search = (float)((double)(ts[2] - ts[1]) * 1e-6);
  R->fetched = true;
  return SPG_OK;
}

int spg_result_get(spg_result* R, int32_t* n_states, int32_t* n_sites, uint16_t* states, int64_t* energies_fixed,
                   double* energies, double* log_probs, double* max_logmarg_err) {
  if (!R) return SPG_EINVAL;
  spg_ctx* ctx = R->ctx;
  int rc = fetch(R);
  if (rc) return rc;
  int diag[4];
  CK(cudaMemcpy(diag, R->d_diag, sizeof(int) * 4, cudaMemcpyDeviceToHost));
  if (n_states) *n_states = R->n;
  if (n_sites) *n_sites = R->N;
  if (states)
    CK(cudaMemcpy(states, R->d_states, sizeof(uint16_t) * (size_t)R->n * R->N, cudaMemcpyDeviceToHost));
  std::vector<int64_t> E(R->n);
  if (energies_fixed || energies) CK(cudaMemcpy(E.data(), R->d_E, sizeof(int64_t) * R->n, cudaMemcpyDeviceToHost));
  if (energies_fixed) std::memcpy(energies_fixed, E.data(), sizeof(int64_t) * R->n);
  if (energies)
    for (int k = 0; k < R->n; ++k) energies[k] = (double)E[k];
  if (log_probs) CK(cudaMemcpy(log_probs, R->d_logp, sizeof(double) * R->n, cudaMemcpyDeviceToHost));
  if (max_logmarg_err) CK(cudaMemcpy(max_logmarg_err, R->d_err, sizeof(double), cudaMemcpyDeviceToHost));
  if (diag[1] & ERR_TIMEOUT) return fail(ctx, SPG_ETIMEOUT, "a bounded wait in a kernel gave up");
  if (diag[1] & ERR_ENERGY) return fail(ctx, SPG_ENUMERIC, "final energies disagree with the running energies");
  if (diag[1] & ERR_KEY) return fail(ctx, SPG_EUNSUPPORTED, "merge key overflow");
  return SPG_OK;
}

int spg_result_info(spg_result* R, spg_info* info) {
  if (!R || !info) return SPG_EINVAL;
  spg_ctx* ctx = R->ctx;
  int rc = fetch(R);
  if (rc) return rc;
  int diag[4];
  double cand[2];
  CK(cudaMemcpy(diag, R->d_diag, sizeof(int) * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(cand, R->d_cand, sizeof(double) * 2, cudaMemcpyDeviceToHost));
  std::memset(info, 0, sizeof(*info));
  info->n_states = R->n;
  info->near_ties = diag[0];
  info->error_flags = diag[1];
  info->degenerate_cuts = diag[2];
  info->ms_boundary = R->ms_boundary;
  info->ms_search = R->ms_search;
  info->candidates = cand[0];
  info->boundary_lognorm = cand[1];
  info->kernel_launches = R->launches;
  info->jacobi_sweeps_max = diag[3];
  info->fp64_rows = R->fp64_rows;
  info->precision_used = R->precision_used;
  info->group_size = R->group_size;
  int dnf[2] = {0, 0};
  CK(cudaMemcpy(dnf, R->d_dn, sizeof(int) * 2, cudaMemcpyDeviceToHost));
  info->droplet_overflow = dnf[1];
  CK(cudaMemcpy(&info->max_logmarg_err, R->d_err, sizeof(double), cudaMemcpyDeviceToHost));
  return SPG_OK;
}

void spg_result_destroy(spg_result* R) {
  if (!R) return;
  cudaSetDevice(R->ctx->device);
  // stream-ordered frees: after the solve that wrote the buffers, without
  // holding the host (a worker stream may already run the next batch)
  cudaStream_t st = R->ctx->stream;
  if (R->blk) cudaFreeAsync(R->blk, st);
  for (int k = 0; k < 3; ++k)
    if (R->ev[k]) cudaEventDestroy(R->ev[k]);
  cudaGetLastError();
  spg_ctx* ctx = R->ctx;
  delete R;
  ctx_release(ctx);
}

int spg_debug_marginals(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, int32_t site, int32_t n_prefix,
                        const uint16_t* prefixes, double* log_marg) {
  if (!ctx || !P || !log_marg) return SPG_EINVAL;
  int rc = check_params(ctx, P, prm);
  if (rc) return rc;
  if (site < 0 || site >= P->n || n_prefix < 1 || n_prefix > SPG_MAX_BEAM || (site > 0 && !prefixes))
    return fail(ctx, SPG_EINVAL, "bad site or prefixes");
  for (int k = 0; k < n_prefix; ++k)
    for (int t = 0; t < site; ++t)
      if (prefixes[(size_t)k * site + t] >= P->d[t]) return fail(ctx, SPG_EINVAL, "prefix state out of range");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SPG_ECUDA, "cudaSetDevice failed");
  return (prm->precision == SPG_FP64 || fp32_range_exceeded(P, prm))
             ? debug_marginals_impl<double>(ctx, P, prm, site, n_prefix, prefixes, log_marg)
             : debug_marginals_impl<float>(ctx, P, prm, site, n_prefix, prefixes, log_marg);
}

int spg_log_partition(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, double* log_z) {
  if (!ctx || !P || !log_z) return SPG_EINVAL;
  int rc = check_params(ctx, P, prm);
  if (rc) return rc;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SPG_ECUDA, "cudaSetDevice failed");
  return (prm->precision == SPG_FP64 || fp32_range_exceeded(P, prm)) ? logz_impl<double>(ctx, P, prm, log_z)
                                                                       : logz_impl<float>(ctx, P, prm, log_z);
}

int spg_truncate(spg_ctx* ctx, const double* M, int32_t m, int32_t n, int32_t keep, int32_t iters, double* V,
                 double* US, double* sigma) {
  if (!ctx || !M || !V || !US || !sigma) return SPG_EINVAL;
  if (m < 1 || n < 1 || m > 16384 || n > 16384 || keep < 1 || keep > std::min(64, std::min(m, n)) || iters < 0 ||
      iters > 64)
    return fail(ctx, SPG_EINVAL, "spg_truncate: sizes outside the limits");
  CK(cudaSetDevice(ctx->device));
  const size_t work = truncated_svd_work(m, n, keep);
  const size_t bytes = sizeof(double) * work + 1024;
  int rc = ensure_arena(ctx, bytes);
  if (rc) return rc;
  Arena ar{ctx->arena, 0, ctx->arena_bytes};
  double* w = ar.get<double>(work);
  double* s1 = ar.get<double>(2);
  int* flag = ar.get<int>(2);
  if (!flag) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(flag, 0, sizeof(int) * 2, st));
  CK(truncated_svd<double>(M, m, n, keep, iters, 0x5eedull, V, US, w, work, s1, flag, st));
  CK(cudaMemcpyAsync(sigma, w + truncated_svd_sigma_offset(m, n, keep), sizeof(double) * keep,
                     cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return SPG_OK;
}

int spg_tc_product(spg_ctx* ctx, const float* M, int32_t m, int32_t n, const float* Bt, int32_t s, int32_t trans,
                   float* out) {
  if (!ctx || !M || !Bt || !out) return SPG_EINVAL;
  if (m < 1 || n < 1 || s < 1) return fail(ctx, SPG_EINVAL, "spg_tc_product: sizes must be positive");
  if (!tc_gemm_eligible(m, n, s)) return fail(ctx, SPG_EUNSUPPORTED, "spg_tc_product: sizes outside the limits");
  CK(cudaSetDevice(ctx->device));
  const size_t work = tc_gemm_elems(m, n, s);
  int rc = ensure_arena(ctx, sizeof(float) * work + 1024);
  if (rc) return rc;
  Arena ar{ctx->arena, 0, ctx->arena_bytes};
  float* w = ar.get<float>(work);
  int* flag = ar.get<int>(1);
  if (!flag) return fail(ctx, SPG_ENOMEM, "workspace carve overflow");
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
  TcGemm tc(w, work, M, m, n, flag, st);
  CK(tc.run(trans != 0, Bt, s, out));
  int h = 0;
  CK(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h) return fail(ctx, SPG_ETIMEOUT, "spg_tc_product: a bounded wait in the kernel gave up");
  return SPG_OK;
}

int spg_profile(spg_ctx* ctx, int enable) {
  if (!ctx) return SPG_EINVAL;
  KernelProfile& p = kernel_profile();
  p.on = enable != 0;
  return SPG_OK;
}

int spg_profile_report(spg_ctx* ctx, char* json_out, size_t cap) {
  if (!ctx || !json_out || cap == 0) return SPG_EINVAL;
  KernelProfile& p = kernel_profile();
  CK(cudaSetDevice(ctx->device));
  struct Agg {
    long long n = 0;
    double ms = 0.0, flops = 0.0;
  };
  std::map<std::string, Agg> agg;
  if (p.used > 0) {
    cudaEvent_t end;
    CK(cudaEventCreate(&end));
    CK(cudaEventRecord(end, p.streams[p.used - 1]));
    CK(cudaEventSynchronize(end));
    for (size_t i = 0; i < p.used; ++i) {
      float ms = 0.f;
      if (!p.names[i]) continue;  // a closing mark
      cudaEvent_t nxt = i + 1 < p.used && p.streams[i + 1] == p.streams[i] ? p.pool[i + 1] : end;
      if (cudaEventElapsedTime(&ms, p.pool[i], nxt) != cudaSuccess) {
        cudaGetLastError();
        ms = 0.f;
      }
      auto& a = agg[p.names[i]];
      a.n += 1;
      a.ms += ms;
      a.flops += p.flops[i];
    }
    cudaEventDestroy(end);
  }
  std::string out = "{";
  bool first = true;
  for (auto& kv : agg) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s\"%s\": [%lld, %.6f, %.6e]", first ? "" : ", ", kv.first.c_str(), kv.second.n,
                  kv.second.ms, kv.second.flops);
    out += buf;
    first = false;
  }
  out += "}";
  std::strncpy(json_out, out.c_str(), cap - 1);
  json_out[cap - 1] = 0;
  p.names.clear();
  p.streams.clear();
  p.flops.clear();
  p.used = 0;
  return SPG_OK;
}


int spg_warm_features(const spg_problem* P, int32_t row, float* out) {
  if (!P || !out || row < 0 || row >= P->rows) return SPG_EINVAL;
  if (P->wsblk.empty()) return SPG_EUNSUPPORTED;
  ws_features(P, row, out);
  return SPG_OK;
}

int spg_boundary_export(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, int32_t row, int32_t fix_signs,
                        void* out, int32_t* dims) {
  if (!ctx || !P || !out) return SPG_EINVAL;
  int rc = check_params(ctx, P, prm);
  if (rc) return rc;
  if (row < 0 || row >= P->rows || (row == 0 && P->rows < 2))
    return fail(ctx, SPG_EINVAL, "spg_boundary_export: row outside 0 .. rows-1");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SPG_ECUDA, "cudaSetDevice failed");
  return prm->precision == SPG_FP64 ? export_impl<double>(ctx, P, prm, row, fix_signs != 0, out, dims)
                                    : export_impl<float>(ctx, P, prm, row, fix_signs != 0, out, dims);
}

int spg_mlp_create(spg_ctx* ctx, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, spg_mlp** out) {
  if (!ctx || !out) return SPG_EINVAL;
  *out = nullptr;
  if (n_in < 1 || n_in > 4096 || n_hidden < 1 || n_hidden > 1024 || n_out < 1 || n_out > 65536)
    return fail(ctx, SPG_EUNSUPPORTED, "spg_mlp_create: sizes outside the limits");
  CK(cudaSetDevice(ctx->device));
  spg_mlp* m = new (std::nothrow) spg_mlp();
  if (!m) return SPG_ENOMEM;
  m->device = ctx->device;
  m->stream = ctx->stream;
  m->ctx = ctx;
  ctx_retain(ctx);
  m->n_in = n_in;
  m->n_hidden = n_hidden;
  m->n_out = n_out;
  int rc = mlp_setup(m);
  if (!rc) rc = mlp_init_params(m, seed);
  if (rc) {
    spg_mlp_destroy(m);
    return fail(ctx, rc, "spg_mlp_create: device allocation or initialisation failed");
  }
  *out = m;
  return SPG_OK;
}

int spg_set_warm_start(spg_ctx* ctx, spg_mlp* mlp) {
  if (!ctx) return SPG_EINVAL;
  if (mlp && mlp->device != ctx->device) return fail(ctx, SPG_EINVAL, "network on another device");
  ctx->warm = mlp;
  for (spg_ctx* w : ctx->workers) w->warm = mlp;
  return SPG_OK;
}

int spg_sweep_trace(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, int32_t row, int32_t init,
                    int32_t n_sweeps, double* log_overlap) {
  if (!ctx || !P || !log_overlap) return SPG_EINVAL;
  int rc = check_params(ctx, P, prm);
  if (rc) return rc;
  if (row < 1 || row >= P->rows || init < 0 || init > 2 || n_sweeps < 1 || n_sweeps > 256)
    return fail(ctx, SPG_EINVAL, "spg_sweep_trace: bad row, init or n_sweeps");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SPG_ECUDA, "cudaSetDevice failed");
  return prm->precision == SPG_FP64 ? trace_impl<double>(ctx, P, prm, row, init, n_sweeps, log_overlap)
                                    : trace_impl<float>(ctx, P, prm, row, init, n_sweeps, log_overlap);
}

int spg_check_bounded_wait(spg_ctx* ctx, int64_t polls) {
  if (!ctx || polls < 0 || polls > (int64_t)1 << 40) return SPG_EINVAL;
  CK(cudaSetDevice(ctx->device));
  int rc = ensure_arena(ctx, 4096);
  if (rc) return rc;
  int* flag = reinterpret_cast<int*>(ctx->arena);
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
  CK(launch_wait_check((long)polls, flag, st));
  int h = 0;
  CK(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h & ERR_TIMEOUT) return fail(ctx, SPG_ETIMEOUT, "bounded wait gave up (as it must: nothing completes it)");
  return fail(ctx, SPG_ECUDA, "bounded wait check: the wait did not report its timeout");
}

int spg_inject_alloc_failure(int32_t after) {
  alloc_failure_countdown().store(after < 0 ? -1 : after);
  return SPG_OK;
}

int spg_solve_lattice8(spg_ctx* ctx, const spg_problem* P, const spg_params* prm, spg_result** out,
                       int32_t* best_k, int64_t* best_per_lattice) {
  if (!ctx || !P || !prm || !out) return SPG_EINVAL;
  *out = nullptr;
  int rc = check_params(ctx, P, prm);
  if (rc) return rc;
  const int rows = P->rows, cols = P->cols, n = P->n;
  std::vector<spg_problem*> probs(8, nullptr);
  std::vector<std::vector<int32_t>> maps(8, std::vector<int32_t>(n));
  auto release = [&]() {
    for (int k = 1; k < 8; ++k) spg_problem_destroy(probs[k]);
  };
  for (int k = 0; k < 8; ++k) {
    int32_t R = 0, C = 0;
    spg_lattice_site_map(rows, cols, k, maps[k].data(), &R, &C);
    if (k == 0) {
      probs[0] = const_cast<spg_problem*>(P);
      continue;
    }
    if (C > SPG_MAX_COLS) {
      release();
      return fail(ctx, SPG_EUNSUPPORTED, "a transposed lattice is wider than the built limit");
    }
    const auto& rw = P->raw;
    if (!rw.potts) {
      std::vector<int32_t> crow(n), ccol(n);
      for (int c = 0; c < n; ++c) {
        const int t = maps[k][rw.crow[c] * cols + rw.ccol[c]];
        crow[c] = t / C;
        ccol[c] = t % C;
      }
      rc = spg_problem_ising(ctx, rw.n_spins, (int32_t)rw.ei.size(), rw.ei.data(), rw.ej.data(), rw.J.data(),
                             rw.h.empty() ? nullptr : rw.h.data(), rw.cos.data(), R, C, crow.data(), ccol.data(),
                             P->shift, P->node_type, &probs[k]);
    } else {
      // sites move with their local tables; edges keep their tables
      std::vector<int32_t> d2(n), em2(rw.em.size()), en2(rw.en.size());
      std::vector<size_t> off(n + 1, 0);
      for (int s2 = 0; s2 < n; ++s2) off[s2 + 1] = off[s2] + (size_t)rw.d[s2];
      std::vector<int32_t> old_of(n);
      for (int s2 = 0; s2 < n; ++s2) old_of[maps[k][s2]] = s2;
      std::vector<int64_t> local;
      local.reserve(rw.local.size());
      for (int t = 0; t < n; ++t) {
        const int o = old_of[t];
        d2[t] = rw.d[o];
        local.insert(local.end(), rw.local.begin() + off[o], rw.local.begin() + off[o + 1]);
      }
      for (size_t e = 0; e < rw.em.size(); ++e) {
        em2[e] = maps[k][rw.em[e]];
        en2[e] = maps[k][rw.en[e]];
      }
      rc = spg_problem_potts(ctx, R, C, d2.data(), local.data(), (int32_t)em2.size(), em2.data(), en2.data(),
                             rw.pair.data(), P->shift, P->node_type, &probs[k]);
    }
    if (rc) {
      release();
      return rc;
    }
  }
  std::vector<spg_params> prms(8, *prm);
  std::vector<spg_result*> res(8, nullptr);
  rc = spg_solve_batch(ctx, 8, probs.data(), prms.data(), res.data());
  if (rc) {
    release();
    return rc;
  }
  // the first lowest best energy
  int kb = -1;
  int64_t bestE = 0;
  for (int k = 0; k < 8 && !rc; ++k) {
    int32_t ns = 0;
    rc = spg_result_get(res[k], &ns, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    int64_t e0 = INT64_MAX;
    if (!rc && ns > 0) rc = spg_result_get(res[k], nullptr, nullptr, nullptr, &e0, nullptr, nullptr, nullptr);
    if (best_per_lattice) best_per_lattice[k] = e0;
    if (!rc && (kb < 0 || e0 < bestE)) {
      kb = k;
      bestE = e0;
    }
  }
  for (int k = 0; k < 8; ++k)
    if (k != kb || rc) spg_result_destroy(res[k]);
  if (rc) {
    release();
    return rc;
  }
  // the chosen lattice's states on the original sites
  spg_result* R = res[kb];
  spg_ctx* rctx = R->ctx;
  cudaStream_t st = rctx->stream;
  uint16_t* remapped = nullptr;
  int* map_dev = nullptr;
  if (cudaMallocAsync((void**)&remapped, sizeof(uint16_t) * (size_t)R->cap * R->N, st) != cudaSuccess ||
      cudaMallocAsync((void**)&map_dev, sizeof(int) * n, st) != cudaSuccess) {
    cudaGetLastError();
    spg_result_destroy(R);
    release();
    return fail(ctx, SPG_ENOMEM, "lattice remap: allocation failed");
  }
  CK(cudaMemcpyAsync(map_dev, maps[kb].data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  k_permute_sites<<<std::max(1, std::min(1024, (R->cap * R->N + 255) / 256)), 256, 0, st>>>(R->d_states, remapped,
                                                                                             R->d_n, R->N, map_dev);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(R->d_states, remapped, sizeof(uint16_t) * (size_t)R->cap * R->N, cudaMemcpyDeviceToDevice, st));
  cudaFreeAsync(remapped, st);
  cudaFreeAsync(map_dev, st);
  CK(cudaStreamSynchronize(st));
  release();
  if (best_k) *best_k = kb;
  *out = R;
  return SPG_OK;
}

int spg_result_droplets(spg_result* R, int32_t* n, int64_t* energies, uint16_t* states) {
  if (!R) return SPG_EINVAL;
  spg_ctx* ctx = R->ctx;
  int rc = fetch(R);
  if (rc) return rc;
  int dnf[2] = {0, 0};
  CK(cudaMemcpy(dnf, R->d_dn, sizeof(int) * 2, cudaMemcpyDeviceToHost));
  if (n) *n = dnf[0];
  if (energies && dnf[0] > 0) CK(cudaMemcpy(energies, R->d_dE, sizeof(int64_t) * dnf[0], cudaMemcpyDeviceToHost));
  if (states && dnf[0] > 0)
    CK(cudaMemcpy(states, R->d_dst, sizeof(uint16_t) * (size_t)dnf[0] * R->N, cudaMemcpyDeviceToHost));
  return SPG_OK;
}

}  // extern "C"
