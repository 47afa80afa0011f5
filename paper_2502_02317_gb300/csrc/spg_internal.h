// Internal declarations shared by the host orchestration and the kernels of
// libspg.  Not part of the C ABI.
#pragma once

#include <atomic>
#include <cstdint>
#include <functional>
#include <mutex>
#include <type_traits>
#include <vector>
#include <cuda_runtime.h>

struct spg_ctx;

// The warm-start network (include/spg.h spg_mlp_*): sizes, the flat FP32
// parameters, their gradient and Adam moments (one allocation, 4 x
// n_params), a BF16 copy of the parameters for inference, and scratch.
struct spg_mlp {
  spg_ctx* ctx = nullptr;  // counted as a handle of its context
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_in = 0, n_hidden = 0, n_out = 0;
  int64_t n_params = 0;
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;  // offsets in the flat layout
  float* p = nullptr;
  float* g = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  void* pbf = nullptr;  // __nv_bfloat16[n_params]
  int t = 0;            // Adam steps taken
  float* scratch = nullptr;
  size_t scratch_elems = 0;
};

namespace spg {

// Handle counting of a context (problems, results, networks): a context
// destroyed while handles made through it are alive is released when the
// last of them is destroyed, whatever the order of the destroy calls.
void ctx_retain(spg_ctx* ctx);
void ctx_release(spg_ctx* ctx);

// The lockstep group of the calling host thread (see the group section
// below): instances every launch covers, and their byte stride.
struct Group {
  int n = 1;
  size_t zs = 0;
  const char* lo = nullptr;
  bool bad = false;  // a launch was refused
};
inline Group& group() {
  thread_local Group g;
  return g;
}
inline unsigned zn() { return (unsigned)group().n; }
inline size_t zs() { return group().zs; }

// Kernels enqueued by this library since load (every launcher adds its own).
inline std::atomic<long long>& launch_counter() {
  static std::atomic<long long> c{0};
  return c;
}

// Opt-in per-kernel timing: while enabled, an event is recorded on the
// launching stream just before every kernel, so that after a synchronize the
// time between consecutive events is the device time of each kernel (kernels
// on one stream run one after another).
struct KernelProfile {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<const char*> names;
  std::vector<cudaStream_t> streams;
  std::vector<double> flops;  // algorithmic flops of each launch (0: not counted)
  size_t used = 0;
};
inline KernelProfile& kernel_profile() {
  static KernelProfile p;
  return p;
}

// Kernels enqueued by the calling host thread (a solve counts its own).
inline long long& thread_launches() {
  thread_local long long c = 0;
  return c;
}

// Inside a stream capture an external record becomes an event-record node of
// the graph (timed when the graph runs); outside, a plain record.
inline void record_mark(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else
    cudaEventRecord(e, st);
}

inline void count_launches(const char* name, cudaStream_t st, double flops = 0.0) {
  launch_counter().fetch_add(1, std::memory_order_relaxed);
  ++thread_launches();
  KernelProfile& p = kernel_profile();
  if (!p.on) return;
  std::lock_guard<std::mutex> lock(p.mu);
  if (p.used == p.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    p.pool.push_back(e);
  }
  record_mark(p.pool[p.used], st);
  p.names.push_back(name);
  p.streams.push_back(st);
  p.flops.push_back(flops * zn());  // a launch covers every instance of the group
  ++p.used;
}

// Closing mark of a profiled stretch of work: an event record without a
// kernel, so that the last kernel's time ends where the work ends (report
// entries without a name are not listed).
inline void profile_mark(cudaStream_t st) {
  KernelProfile& p = kernel_profile();
  if (!p.on) return;
  std::lock_guard<std::mutex> lock(p.mu);
  if (p.used == p.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    p.pool.push_back(e);
  }
  record_mark(p.pool[p.used], st);
  p.names.push_back(nullptr);
  p.streams.push_back(st);
  p.flops.push_back(0.0);
  ++p.used;
}

// Autotuner (autotune.cpp): the variant of a kernel to launch for a shape.
// `launch(v)` enqueues variant v on `st` (not counted as a library launch);
// `valid` has bit v set for every variant that may run this shape; `dflt` is
// the built-in choice.  The variants of one kernel must give bit-identical
// results and must not read what they write (each may run several times).
constexpr int TUNE_MAX_VARIANTS = 4;
int tune_pick(const char* kernel, const long long* shape, int n_shape, cudaStream_t st, int n_var, unsigned valid,
              int dflt, const std::function<void(int)>& launch);

constexpr int MAXS = 256;   // states of one cluster
constexpr int MAXP = 16;    // projected (reduced-table) dimension
constexpr int MAXCHI = 64;  // boundary-MPS bond
constexpr int KEYW = 8;     // 64-bit words of a packed merge key
constexpr int SMAX = 128;   // columns of the truncation's working block
#define SPG_MAXFINAL 4096   // final states ordered by the last kernel

// Device error flags (OR-ed into DevSearch::err).
enum : int {
  ERR_ENERGY = 1,     // incremental energy != energy recomputed from the tables
  ERR_NAN = 2,        // NaN / Inf in a normalisation
  ERR_KEY = 4,        // a packed key overflowed its words
  ERR_TIMEOUT = 8,    // a bounded wait inside a kernel gave up
};

// Integer tables of the cluster factor graph (S1) in device memory, for the
// square lattice and the king's graph (diagonal couplings).  Per site s
// (row-major, (i, j)), padded to dmax states:
//   E[s][x]        local energy (int64, units of 2^-shift)
//   PL/PU/PR/PD/PG joint projections of state x (classes of equal table rows
//                  in order of first occurrence, all <= MAXP):
//                    PL: edges to (i, j-1), (i-1, j-1)   PU: edge to (i-1, j)
//                    PR: edges to (i, j+1), (i-1, j+1)   PG: edge to (i+1, j+1)
//                    PD: edges to (i+1, j-1), (i+1, j), (i+1, j+1)
//   dims[s][DIMW]  D_* entries below
//   RL[s][l][h]    energy of the left and up-left edges, l = a * Gin + g the
//                  left bond (a: PR class of (i, j-1), g: PG class of
//                  (i-1, j-1)), h = PL class (row stride MAXP, site stride
//                  lstride)
//   RU[s][u][h]    energy of the up edge, u = PD class of (i-1, j), h = PU
//   RA[s][a][u]    energy of the anti-diagonal edge (i-1, j)-(i, j-1),
//                  a = PR class of (i, j-1), u = PD class of (i-1, j)
//   gD[s][u]       PG class of the states in PD class u of site s
//   xsL[s][..]     states of s grouped by PL (CSR with xoffL[s][0..MAXP])
// On the square lattice every G is 1 and RA is 0.
enum : int {
  D_DL = 0,    // left bond = NRl * Gin
  D_DR = 1,    // right bond = NR * Gout
  D_DU = 2,    // up index = ND of (i-1, j)
  D_DD = 3,    // ND: boundary-MPS physical dimension below this site
  D_NL = 4,
  D_NU = 5,
  D_XIN = 6,   // 1 if the site has an edge to a later site (merge key)
  D_NR = 7,
  D_GIN = 8,   // NG of (i-1, j-1)
  D_GOUT = 9,  // NG of (i-1, j)
  D_NRL = 10,  // NR of (i, j-1)
  D_UCPL = 11, // 1 if W depends on u beyond b_up (Gout > 1 or an anti-diagonal edge)
  DIMW = 16
};
struct DevTables {
  int rows, cols, n, dmax;
  int lstride;  // elements per site of RL / bL (bmax * MAXP)
  int bmax;     // largest bond dimension of any site
  const int* d;
  const int64_t* E;
  const uint8_t *PL, *PR, *PU, *PD, *PG;
  const int* dims;
  const int64_t* RL;
  const int64_t* RU;
  const int64_t* RA;
  const uint8_t* gD;
  const int16_t* xsL;
  const int* xoffL;
  const int* keys;   // [n][MAXKEY+1]: count, then sites of the reduced parent key
  const int* kshift; // bits per packed state
};
constexpr int MAXKEY = 136;  // key sites: a row plus the sites around the current one
constexpr int MAXBOND = MAXP * MAXP;

// Boltzmann pieces (S2), each table shifted by its minimum so that every
// weight is <= 1: w[s][x], bL[s][l][h] (stride lstride), bU[s][u][h] and
// bA[s][a][u] (16 x 16) from RL, RU, RA.
template <typename T>
struct DevWeights {
  T* w;
  T* bL;
  T* bU;
  T* bA;
};

// Boundary MPSs: site (r, j) of B_r at A + (r*cols + j)*site_stride, laid out
// [p][chiL][chiR] with the dims of dimA[(r*cols + j)*3 + {0,1,2}].
template <typename T>
struct DevMPS {
  T* A;
  size_t site_stride;
  const int* dimA;  // device copy
  double* lognorm;  // [rows+1]
};

// ------------------------------------------------------------------ kernels
// All launchers enqueue on `st` and return cudaGetLastError().

template <typename T>
cudaError_t launch_weights(const DevTables& tb, DevWeights<T> wt, double beta_u, cudaStream_t st);

// QR sweep of B (row r) to left-canonical form, in place; lognorm[r] += log
// of the last site's norm.  Scratch: MAXP*chi*chi T (used when the staged
// site does not fit in shared memory).
template <typename T>
cudaError_t launch_left_canonical(DevMPS<T> mps, int r, int cols, const int* dimA_host,
                                  T* scratch, cudaStream_t st);

// M[(l,a),(u,k)] = bA[a(l),u] sum_{x} bL[l,PL x] bU[u,PU x] w(x)
//                  sum_a' B[PD x][a][a'] C[PR x * Gout + gD_up(u)][a'][k]
// for site (r, j) of the MPO applied to B_{r+1} (site j); carry C [DR][chiR][K].
template <typename T>
cudaError_t launch_zip_matrix(const DevTables& tb, DevWeights<T> wt, const T* B, int chiL, int p,
                              int chiR, const T* C, int DR, int K, int site, int DL, int DU,
                              T* T1, T* M, cudaStream_t st);

// Truncated SVD of M (m x n row-major): V (n x keep, column k = k-th right
// singular vector) and US (m x keep); s1 = sigma_1 written to *s1_dev,
// degenerate-cut flag OR-ed into *flag_dev.
// tcw / tcw_elems: optional FP32 workspace of the tensor-core products
// (used by the FP32 instance when tc_gemm_eligible and large enough); flag_dev
// holds 4 ints: degenerate cuts, Jacobi sweeps, error flags, unused.
template <typename T>
cudaError_t truncated_svd(const T* M, int m, int n, int keep, int iters, uint64_t seed, T* V, T* US,
                          T* work, size_t work_elems, double* s1_dev, int* flag_dev, cudaStream_t st,
                          float* tcw = nullptr, size_t tcw_elems = 0);

// Tensor-core (tcgen05, split TF32) products of an FP32 truncation with one
// zipper matrix M (m x n, row-major), whose high/low TF32 parts and those of
// M^T are prepared once by the constructor (in `work`, tc_gemm_elems
// elements).  run(false, Zt, s, Yt): Yt = (M Z)^T; run(true, Yt, s, Zt):
// Zt = (M^T Y)^T, with Zt [s x n] and Yt [s x m] row-major.
size_t tc_gemm_elems(int m, int n, int s);
bool tc_gemm_eligible(int m, int n, int s);
class TcGemm {
 public:
  TcGemm(float* work, size_t elems, const float* M, int m, int n, int* err, cudaStream_t st);
  cudaError_t run(bool trans, const float* Bt, int s, float* out);

 private:
  int m_, n_, mp_, np_;
  int* err_;
  cudaStream_t st_;
  float *Mh_, *Ml_, *MTh_, *MTl_, *Bh_, *Bl_, *part_;
};
cudaError_t launch_or_flag(int* dst, const int* src, cudaStream_t st);
// One bounded mbarrier wait that nothing completes: ERR_TIMEOUT into *err
// after `limit` polls (the failure path of the kernels' bounded waits).
cudaError_t launch_wait_check(long limit, int* err, cudaStream_t st);
// Test hook: the (n+1)-th device workspace allocation from now fails as if
// the device were out of memory (n < 0: off).
std::atomic<int>& alloc_failure_countdown();
// Writes the GPU's global nanosecond timer into *slot when the stream reaches it.
cudaError_t launch_stamp(unsigned long long* slot, cudaStream_t st);
size_t truncated_svd_work(int m, int n, int keep);
// Offset (elements) of the sigma array inside the truncation's work buffer.
size_t truncated_svd_sigma_offset(int m, int n, int keep);

// New site j of B_r ([DU][keep][K]) from V, next carry ([DL][chiL][keep]) from US / s1;
// lognorm[r] += log s1.
template <typename T>
cudaError_t launch_zip_write(const T* V, const T* US, int DL, int chiL, int DU, int K, int keep,
                             T* site_out, T* carry_out, const double* s1_dev, double* lognorm_r,
                             cudaStream_t st);
// Site 0: [DU][1][K] = M / ||M||; lognorm[r] += log ||M||.
template <typename T>
cudaError_t launch_zip_site0(const T* M, int DU, int K, T* site_out, double* lognorm_r, cudaStream_t st);

// CGS2 orthonormalisation of nvec contiguous vectors of length len (in place);
// R (nvec x nvec) to Rout when non-null.
template <typename T>
void launch_cgs2_rows(T* X, int nvec, int len, T* Rout, cudaStream_t st);

// num_sweeps variational sweeps of row `row`'s boundary MPS (S4) against
// W_row B_{row+1}; dimA / hdims are the host copies of the MPS dims and the
// table dims, hgD the host copy of gD; work holds sweep_work_elems<T>(cols,
// chi, bmax) T, dscratch 2 doubles.
template <typename T>
size_t sweep_work_elems(int cols, int chi, int bmax);
template <typename T>
cudaError_t variational_sweeps(const DevTables& tb, DevWeights<T> wt, DevMPS<T> mps, int row, int cols,
                               const int* dimA, const int* hdims, const int* hstates, const uint8_t* hgD,
                               int sweeps, T* work, double* dscratch, cudaStream_t st);

// Value of an MPS whose physical dims are all 1 (row 0 closed from above).
template <typename T>
cudaError_t launch_mps_value(DevMPS<T> mps, int r, int cols, double* out, cudaStream_t st);

// Generic small GEMM: C[m x n] = op(A) * B, row-major, op(A) = A or A^T.
template <typename T>
cudaError_t gemm(bool transA, int m, int n, int k, const T* A, int lda, const T* B, int ldb, T* C,
                 int ldc, cudaStream_t st);
// C[m x n] = op(A) op(B), row-major; op(B) = B^T reads B stored n x k.
template <typename T>
cudaError_t gemm2(bool transA, bool transB, int m, int n, int k, const T* A, int lda, const T* B, int ldb,
                  T* C, int ldc, cudaStream_t st);
// dst[e] = (To) src[e] for e < count (a contiguous block changes precision).
template <typename From, typename To>
cudaError_t launch_convert(const From* src, To* dst, size_t count, cudaStream_t st);
// base[e * stride] = v for e < count.
template <typename T>
cudaError_t launch_set_strided(T* base, size_t stride, int count, T v, cudaStream_t st);

// ------------------------------------------------------------------ search
struct DevSearch {
  int cap;        // beam capacity
  int N;          // sites
  int dmax;
  uint16_t* states[2];  // [cap][N]
  int64_t* E[2];        // [cap]
  double* logp[2];      // [cap]
  int* rid[2];          // [cap] row-start index of the right environments
  int* n_beam;          // [2] live count of each buffer
  double* logc;         // [cap][dmax] log-conditionals
  int64_t* candE;       // [cap][dmax]
  int* win;             // [cap][dmax] winner parent of (class rep b, x), -1 otherwise
  unsigned long long* wmin;  // [cap][dmax] class minimum of the candidate energy (ordered bits)
  int* wkey;            // [cap] winner (member * dmax + x) of a class when the site is not in the key
  unsigned long long* key;  // [cap][KEYW]
  int* rep;             // [cap] class representative
  int* nxt;             // [cap] hash slot of the element's class
  int* htab;            // [hsize] class table: owner index + 1 (0 empty)
  int* hmin;            // [hsize] lowest member index of each slot
  int hsize;            // power of two >= 2 cap
  unsigned* hist;       // [65536]
  unsigned long long* sel_state;  // select-state words
  int* sel_list;        // [cap] selected candidate ids (b*dmax + x)
  int* sel_count;
  int* pend;            // [cap][dmax] candidate ids of the chosen top digit, refined by later passes
  int* pend_n;
  unsigned* done_ctr;
  int* near_ties;
  int* err;
  double* candidates;   // running sum of live beam x d
  int* deg_cuts;
  // droplets (low-energy excitations collected in the merges), per beam
  // element of each buffer: count, energy above the element, full states
  int64_t dcut = -1;    // energy cutoff (units of 2^-shift); < 0: off
  int dham = 0;         // Hamming cutoff
  int* dn[2] = {nullptr, nullptr};       // [cap]
  int64_t* dE[2] = {nullptr, nullptr};   // [cap][MAXDROP]
  uint16_t* dst[2] = {nullptr, nullptr}; // [cap][MAXDROP][N]
  int* dflow = nullptr;                  // droplets not kept (list full)
};
constexpr int MAXDROP = 16;     // droplets kept per partial configuration
constexpr int MAXDCAND = 256;   // droplet candidates of one merge class considered

template <typename T>
struct DevBeamT {
  T* lenv[2];  // [cap][chi]
  T* R;        // [cap][cols+1][chi][rs]
  int rs;      // bond stride of R (the largest bond dimension)
  int chi;
};

// ------------------------------------------------------------------ lockstep groups
// A group is n instances whose device data (tables, workspace, staged
// outputs) have the same layout, instance g at a byte offset g * zs from
// instance 0's.  While a group is set on the calling host thread, every
// launcher runs its grid once per instance (blockIdx.z = instance) and
// passes zs; each kernel shifts its pointers by blockIdx.z * zs on entry.
// Before a launch the host checks that every pointer argument lies inside
// instance 0's block [lo, lo + zs) (a pointer outside it would be shifted
// into another allocation), and refuses the launch otherwise.  Without a
// group n = 1 and zs = 0: the same kernels, no shift.

// zadd: every pointer moved by `off` bytes (null stays null); zp: by the
// block's instance, blockIdx.z * zs.
template <typename T>
__host__ __device__ __forceinline__ T* zadd(T* p, size_t off) {
  return p ? reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<typename std::remove_const<T>::type*>(p)) + off)
           : p;
}
__host__ __device__ __forceinline__ DevTables zadd(DevTables t, size_t off) {
  t.d = zadd(t.d, off);
  t.E = zadd(t.E, off);
  t.PL = zadd(t.PL, off);
  t.PR = zadd(t.PR, off);
  t.PU = zadd(t.PU, off);
  t.PD = zadd(t.PD, off);
  t.PG = zadd(t.PG, off);
  t.dims = zadd(t.dims, off);
  t.RL = zadd(t.RL, off);
  t.RU = zadd(t.RU, off);
  t.RA = zadd(t.RA, off);
  t.gD = zadd(t.gD, off);
  t.xsL = zadd(t.xsL, off);
  t.xoffL = zadd(t.xoffL, off);
  t.keys = zadd(t.keys, off);
  t.kshift = zadd(t.kshift, off);
  return t;
}
template <typename T>
__host__ __device__ __forceinline__ DevWeights<T> zadd(DevWeights<T> w, size_t off) {
  w.w = zadd(w.w, off);
  w.bL = zadd(w.bL, off);
  w.bU = zadd(w.bU, off);
  w.bA = zadd(w.bA, off);
  return w;
}
template <typename T>
__host__ __device__ __forceinline__ DevMPS<T> zadd(DevMPS<T> m, size_t off) {
  m.A = zadd(m.A, off);
  m.dimA = zadd(m.dimA, off);
  m.lognorm = zadd(m.lognorm, off);
  return m;
}
__host__ __device__ __forceinline__ DevSearch zadd(DevSearch d, size_t off) {
  for (int k = 0; k < 2; ++k) {
    d.states[k] = zadd(d.states[k], off);
    d.E[k] = zadd(d.E[k], off);
    d.logp[k] = zadd(d.logp[k], off);
    d.rid[k] = zadd(d.rid[k], off);
    d.dn[k] = zadd(d.dn[k], off);
    d.dE[k] = zadd(d.dE[k], off);
    d.dst[k] = zadd(d.dst[k], off);
  }
  d.n_beam = zadd(d.n_beam, off);
  d.logc = zadd(d.logc, off);
  d.candE = zadd(d.candE, off);
  d.win = zadd(d.win, off);
  d.wmin = zadd(d.wmin, off);
  d.wkey = zadd(d.wkey, off);
  d.key = zadd(d.key, off);
  d.rep = zadd(d.rep, off);
  d.nxt = zadd(d.nxt, off);
  d.htab = zadd(d.htab, off);
  d.hmin = zadd(d.hmin, off);
  d.hist = zadd(d.hist, off);
  d.sel_state = zadd(d.sel_state, off);
  d.sel_list = zadd(d.sel_list, off);
  d.sel_count = zadd(d.sel_count, off);
  d.pend = zadd(d.pend, off);
  d.pend_n = zadd(d.pend_n, off);
  d.done_ctr = zadd(d.done_ctr, off);
  d.near_ties = zadd(d.near_ties, off);
  d.err = zadd(d.err, off);
  d.candidates = zadd(d.candidates, off);
  d.deg_cuts = zadd(d.deg_cuts, off);
  d.dflow = zadd(d.dflow, off);
  return d;
}
template <typename T>
__host__ __device__ __forceinline__ DevBeamT<T> zadd(DevBeamT<T> b, size_t off) {
  b.lenv[0] = zadd(b.lenv[0], off);
  b.lenv[1] = zadd(b.lenv[1], off);
  b.R = zadd(b.R, off);
  return b;
}

// Element k (0 or 1) of a pointer pair by selection, not indexing: a
// kernel's shifted copy of DevSearch / DevBeamT then stays in registers
// (indexing the copy's arrays by a runtime k would place it in local memory).
template <typename P>
__device__ __forceinline__ P pick(P const (&a)[2], int k) {
  return k ? a[1] : a[0];
}

template <typename X>
__device__ __forceinline__ X zp(X x, size_t zs) {
  return zadd(x, (size_t)blockIdx.z * zs);
}

// Host check of a launch's pointer arguments against instance 0's block
// (always true without a group); a failure marks the group bad.
inline bool zin(const void* p) {
  const Group& g = group();
  if (g.n <= 1 || !p) return true;
  const char* c = static_cast<const char*>(p);
  return c >= g.lo && c < g.lo + g.zs;
}
inline bool zin1(const DevTables& t) {
  return zin(t.d) && zin(t.E) && zin(t.PL) && zin(t.PR) && zin(t.PU) && zin(t.PD) && zin(t.PG) && zin(t.dims) &&
         zin(t.RL) && zin(t.RU) && zin(t.RA) && zin(t.gD) && zin(t.xsL) && zin(t.xoffL) && zin(t.keys) &&
         zin(t.kshift);
}
template <typename T>
inline bool zin1(const DevWeights<T>& w) {
  return zin(w.w) && zin(w.bL) && zin(w.bU) && zin(w.bA);
}
template <typename T>
inline bool zin1(const DevMPS<T>& m) {
  return zin(m.A) && zin(m.dimA) && zin(m.lognorm);
}
inline bool zin1(const DevSearch& d) {
  for (int k = 0; k < 2; ++k)
    if (!(zin(d.states[k]) && zin(d.E[k]) && zin(d.logp[k]) && zin(d.rid[k]) && zin(d.dn[k]) && zin(d.dE[k]) &&
          zin(d.dst[k])))
      return false;
  return zin(d.n_beam) && zin(d.logc) && zin(d.candE) && zin(d.win) && zin(d.wmin) && zin(d.wkey) &&
         zin(d.key) && zin(d.rep) && zin(d.nxt) && zin(d.htab) && zin(d.hmin) && zin(d.hist) &&
         zin(d.sel_state) && zin(d.sel_list) && zin(d.sel_count) && zin(d.pend) && zin(d.pend_n) &&
         zin(d.done_ctr) && zin(d.near_ties) && zin(d.err) && zin(d.candidates) && zin(d.deg_cuts) &&
         zin(d.dflow);
}
template <typename T>
inline bool zin1(const DevBeamT<T>& b) {
  return zin(b.lenv[0]) && zin(b.lenv[1]) && zin(b.R);
}
template <typename T>
inline bool zin1(T* p) {
  return zin(p);
}
inline bool zin1(int) { return true; }
// true when every argument lies in instance 0's block; otherwise the group
// is marked bad and the caller returns without launching
template <typename... A>
inline bool zok(const A&... a) {
  const bool ok = !group().bad && (zin1(a) && ...);
  if (!ok) group().bad = true;
  return ok;
}
#define ZOK(...)                                        \
  do {                                                  \
    if (!::spg::zok(__VA_ARGS__)) return cudaErrorInvalidValue; \
  } while (0)
// Device copies and fills inside a solve, once per instance of the group.
cudaError_t zcopy(void* dst, const void* src, size_t bytes, cudaStream_t st);
cudaError_t zfill(void* dst, int byte, size_t bytes, cudaStream_t st);

template <typename T>
cudaError_t launch_right_envs(const DevTables& tb, DevWeights<T> wt, DevMPS<T> mps, int row,
                              const DevSearch& ds, DevBeamT<T> bt, int cur, cudaStream_t st);
// The right environments of a row on the tensor cores (renv_tc.cu; FP32,
// rows that pass renv_tc_row_ok), with `work` holding renv_tc_elems(cols,
// cap) floats (256-byte aligned).
size_t renv_tc_elems(int cols, int cap);
cudaError_t launch_right_envs_tc(const DevTables& tb, DevWeights<float> wt, DevMPS<float> mps, int row,
                                 const DevSearch& ds, DevBeamT<float> bt, int cur, float* work, cudaStream_t st);
template <typename T>
// flops: the launch's algorithmic flops for the profiler (0: not counted).
cudaError_t launch_marginals(const DevTables& tb, DevWeights<T> wt, DevWeights<double> wd, DevMPS<T> mps, int site,
                             const DevSearch& ds, DevBeamT<T> bt, int cur, cudaStream_t st, double flops = 0.0);
cudaError_t launch_merge(const DevTables& tb, int site, const DevSearch& ds, int cur, int merge,
                         cudaStream_t st);
cudaError_t launch_select(const DevTables& tb, int site, const DevSearch& ds, int cur,
                          double log_cut, cudaStream_t st);
template <typename T>
cudaError_t launch_update(const DevTables& tb, DevMPS<T> mps, int site, const DevSearch& ds,
                          DevBeamT<T> bt, int cur, cudaStream_t st);
cudaError_t launch_final(const DevTables& tb, const DevSearch& ds, int cur, uint16_t* out_states,
                         int64_t* out_E, double* out_logp, int* out_n, cudaStream_t st);
// Teacher forcing: fill beam buffer `cur` from host-given prefixes (already
// copied to states[cur]); lenv from B_{i+1} sites 0..j-1.
template <typename T>
cudaError_t launch_lenv_from_prefix(const DevTables& tb, DevMPS<T> mps, int site,
                                    const DevSearch& ds, DevBeamT<T> bt, int cur, cudaStream_t st);
cudaError_t launch_reset_beam(const DevSearch& ds, int cur, cudaStream_t st);
// Droplets of the new beam elements (buffer cur ^ 1) after the prune of
// `site`: each keeps its winner parent's droplets and accepts, in (dE, state)
// order, the losers of its merge class and the losers with one of their own
// droplets applied, within the energy cutoff and beyond the Hamming cutoff
// of the state and of every droplet kept so far.
cudaError_t launch_droplets(const DevTables& tb, int site, const DevSearch& ds, int cur, int merge, cudaStream_t st);
// The droplets of the best final state (lowest (energy, lex index)) sorted by
// (energy, state): out_n, out_E [MAXDROP] (absolute energies), out_states
// [MAXDROP][N].
cudaError_t launch_final_droplets(const DevSearch& ds, int cur, int* out_n, int64_t* out_E, uint16_t* out_states,
                                  cudaStream_t st);

// ------------------------------------------------------------------ warm start
// Offsets of the flat parameter layout and the device buffers (SPG_ENOMEM on
// failure); initial parameters from a seed (synchronous).
int mlp_setup(spg_mlp* m);
int mlp_init_params(spg_mlp* m, uint64_t seed);
// BF16 inference of n samples X [n][n_in] -> Y [n][n_out] (device), with
// `work` holding mlp_infer_elems(m, n) floats.
size_t mlp_infer_elems(const spg_mlp* m, int n);
cudaError_t mlp_infer_bf16(const spg_mlp* m, const float* X, int n, float* work, float* Y, cudaStream_t st);
// Row `row` of an MPS from padded network sites Y [cols][16][chi][chi]
// (entries beyond each site's dims ignored).
template <typename T>
cudaError_t launch_ws_scatter(const float* Y, int chi, int cols, DevMPS<T> mps, int row, cudaStream_t st);
// Row `row` of an MPS to padded sites out [cols][16][chi][chi] (zeros beyond
// the dims); fix_signs applies the sign gauge (dims_dev: the row's [cols][3]).
template <typename T>
cudaError_t launch_export_row(DevMPS<T> mps, int row, int cols, int chi, T* out, const int* dims_dev, int fix_signs,
                              cudaStream_t st);
// Teacher forcing along the n (= *n_dev) full states `targets` ([n][N]):
// launch_force_init fills beam buffer `cur` with n empty prefixes; per site,
// after the right environments (row start) and the marginals, launch_force
// makes each element's target state its only child and writes that state's
// log-conditional to out[b][site]; launch_update then extends the prefixes.
cudaError_t launch_force_init(const DevSearch& ds, const int* n_dev, int cur, cudaStream_t st);
cudaError_t launch_force(int site, const DevSearch& ds, int cur, const uint16_t* targets, double* out,
                         cudaStream_t st);
// *out = max over the n x N entries of |a - r| / max(1, |r|) (inf when one
// side is -inf and the other is not).
cudaError_t launch_logmarg_err(const double* a, const double* r, const int* n_dev, int N, double* out,
                               cudaStream_t st);

}  // namespace spg
