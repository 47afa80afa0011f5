// Variational sweeps of a boundary MPS (S4): one-site updates of phi that
// maximise |<phi| W psi>| with the other sites orthonormal, left to right
// (QR moves the centre right) then right to left (LQ moves it left).
//
// Paper: Sec. 3.1 (MpsParameters(bond_dim, num_sweeps)); Sec. 2 (boundary
// MPS contraction of the PEPS).
//
// Layouts (row r of the MPO, psi = B_{r+1} sites B[s][b][b'], phi sites
// P[u][a][a'], both [p][chi_l][chi_r]):
//   environments  E[l][a][b]  (MPO bond < 16, phi bond, psi bond)
// Sites whose tensor depends on the up index beyond b_up (king's graph: the
// anti-diagonal factor and the down-right offset of the right bond) are
// contracted one up index at a time with per-u coefficient tables.
//   W[l,r,u,s] = sum_x w(x) bL[l][PL x] bU[u][PU x] [r = PR x][s = PD x]
// Every contraction groups the cluster states x by their projections, so the
// dense MPO is never formed.
#include <cmath>

#include "spg_internal.h"

namespace spg {

namespace {

template <typename T>
__device__ __forceinline__ T warp_max_abs(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Batched strided GEMM over a "state" index q (one grid.z slice per q):
//   C_q[i][j] = sum_k A[offA(q) + i*sAi + k*sAk] * B[offB(q) + k*sBk + j*sBj]
// written to C + q*M*N (row-major M x N).  The operand offsets follow from
// q through the site's projections: off = c1 * v(id1, q) + c2 * v(id2, q)
// with id 0: none, 1: P_L, 2: P_R, 3: P_U, 4: P_D, 5: q / n2, 6: q % n2.
struct XOff {
  int id1, id2;
  long long c1, c2;
};

__device__ __forceinline__ long long xval(const DevTables& tb, int s, int id, int q, int n2) {
  const size_t so = (size_t)s * tb.dmax;
  switch (id) {
    case 1: return tb.PL[so + q];
    case 2: return tb.PR[so + q];
    case 3: return tb.PU[so + q];
    case 4: return tb.PD[so + q];
    case 5: return q / n2;
    case 6: return q % n2;
    default: return 0;
  }
}

// One 32 x 32 output tile of state q's product per group of 64 threads, QPB
// states per block (1, 2 or 4, the autotuner's choice); each thread holds a
// 4 x 4 register tile and reads a four-wide column of A and row of B from
// shared memory per k (two vector loads per 16 multiply-adds).  Every output
// sums over k in order, as a one-entry-per-thread kernel would, whatever QPB
// is.  grid: (N tiles,
// M tiles, state blocks x instances of a lockstep group).
template <typename T, int QPB>
__global__ void __launch_bounds__(64 * QPB) k_xgemm(DevTables tb, int s, int n2, int M, int N, int K,
                                                    const T* __restrict__ A, XOff oa, int sAi, int sAk,
                                                    const T* __restrict__ B, XOff ob, int sBk, int sBj,
                                                    T* __restrict__ C, int nq, size_t zs) {
  constexpr int BT = 32, LD = BT + 4;  // tile edge; padded row (a multiple of 4 for the vector loads)
  __shared__ __align__(16) T sA[QPB][BT][LD];  // [k][i]
  __shared__ __align__(16) T sB[QPB][BT][LD];  // [k][j]
  const int nqb = (nq + QPB - 1) / QPB;
  const int qb = blockIdx.z % nqb;
  const size_t zo = (size_t)(blockIdx.z / nqb) * zs;
  tb = zadd(tb, zo);
  A = zadd(A, zo);
  B = zadd(B, zo);
  C = zadd(C, zo);
  const int g = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int q = qb * QPB + g;
  const bool live = q < nq;
  const int qq = live ? q : 0;
  const long long offA = oa.c1 * xval(tb, s, oa.id1, qq, n2) + oa.c2 * xval(tb, s, oa.id2, qq, n2);
  const long long offB = ob.c1 * xval(tb, s, ob.id1, qq, n2) + ob.c2 * xval(tb, s, ob.id2, qq, n2);
  const T* Aq = A + offA;
  const T* Bq = B + offB;
  const int ty = t >> 3, tx = t & 7;  // rows ty*4.., columns tx*4..
  const int row0 = blockIdx.y * BT, col0 = blockIdx.x * BT;
  T acc[4][4] = {};
  for (int kk = 0; kk < K; kk += BT) {
    // consecutive threads along the operand's unit-stride index (coalesced)
    const bool a_k = sAk == 1, b_j = sBj == 1 || sBk != 1;
    for (int e = t; e < BT * BT; e += 64) {
      const int i = a_k ? e / BT : e % BT, kq = a_k ? e % BT : e / BT;
      const int gi = row0 + i, gk = kk + kq;
      sA[g][kq][i] = (live && gi < M && gk < K) ? Aq[(long long)gi * sAi + (long long)gk * sAk] : T(0);
      const int kb = b_j ? e / BT : e % BT, j = b_j ? e % BT : e / BT;
      const int gj = col0 + j, gkb = kk + kb;
      sB[g][kb][j] = (live && gj < N && gkb < K) ? Bq[(long long)gkb * sBk + (long long)gj * sBj] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kq = 0; kq < BT; ++kq) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a[r] = sA[g][kq][ty * 4 + r];
        b[r] = sB[g][kq][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
    }
    __syncthreads();
  }
  if (!live) return;
  T* Cq = C + (size_t)q * M * N;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = row0 + ty * 4 + r;
    if (gi >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = col0 + tx * 4 + c;
      if (gj < N) Cq[(size_t)gi * N + gj] = acc[r][c];
    }
  }
}

// Coefficients of the weighted sum over states (K x d, row-major):
//   mode 0: coef[u][x] = bU[u][PU x] w(x)      (local tensor)
//   mode 1: coef[l][x] = bL[l][PL x] w(x)      (right environment)
//   mode 2: coef[r][x] = [PR x == r] w(x)      (left environment)
// and, for one up index u of a site whose tensor depends on u beyond b_up
// (king's graph: the anti-diagonal factor bA and the right-bond offset g):
//   mode 3: coef[0][x] = bU[u][PU x] w(x)
//   mode 4: coef[l][x] = bA[l / Gin][u] bL[l][PL x] bU[u][PU x] w(x)
//   mode 5: coef[r][x] = [PR x * Gout + g == r] bU[u][PU x] w(x)
template <typename T>
__global__ void k_state_coef(DevTables tb, DevWeights<T> wt, int s, int mode, int K, int u, int g,
                             T* __restrict__ coef, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  coef = zp(coef, zs);
  const int d = tb.d[s];
  const size_t so = (size_t)s * tb.dmax;
  const int* dm = tb.dims + s * DIMW;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * d; e += gridDim.x * blockDim.x) {
    const int k = e / d, x = e % d;
    T v;
    if (mode == 0)
      v = wt.bU[(size_t)s * 256 + k * 16 + tb.PU[so + x]];
    else if (mode == 1)
      v = wt.bL[(size_t)s * tb.lstride + k * MAXP + tb.PL[so + x]];
    else if (mode == 2)
      v = tb.PR[so + x] == k ? T(1) : T(0);
    else if (mode == 3)
      v = wt.bU[(size_t)s * 256 + u * 16 + tb.PU[so + x]];
    else if (mode == 4)
      v = wt.bA[(size_t)s * 256 + (k / dm[D_GIN]) * 16 + u] * wt.bL[(size_t)s * tb.lstride + k * MAXP + tb.PL[so + x]] *
          wt.bU[(size_t)s * 256 + u * 16 + tb.PU[so + x]];
    else
      v = (tb.PR[so + x] * dm[D_GOUT] + g == k) ? wt.bU[(size_t)s * 256 + u * 16 + tb.PU[so + x]] : T(0);
    coef[e] = v * wt.w[so + x];
  }
}

// bLu[l][h] = bA[l / Gin][u] bL[l][h]: the left weights of one up index u.
template <typename T>
__global__ void k_left_weights_u(DevTables tb, DevWeights<T> wt, int s, int u, T* __restrict__ out, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  out = zp(out, zs);
  const int* dm = tb.dims + s * DIMW;
  const int DL = dm[D_DL];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < DL * MAXP; e += gridDim.x * blockDim.x) {
    const int l = e / MAXP;
    out[e] = wt.bA[(size_t)s * 256 + (l / dm[D_GIN]) * 16 + u] * wt.bL[(size_t)s * tb.lstride + e];
  }
}

template <typename T>
__global__ void k_axpy(T* __restrict__ y, const T* __restrict__ x, size_t n, size_t zs) {
  y = zp(y, zs);
  x = zp(x, zs);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] += x[e];
}

// In-place scaling of buf[0..n) to max |.| = 1, log of the scale added to *logacc.
template <typename T>
__global__ void __launch_bounds__(1024) k_scale_max(T* buf, int n, double* logacc, size_t zs) {
  buf = zp(buf, zs);
  logacc = zp(logacc, zs);
  __shared__ T red[32];
  T m = T(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = max(m, (T)fabs((double)buf[i]));
  m = warp_max_abs(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    T t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
    t = warp_max_abs(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  const T mx = red[0];
  const T inv = mx > T(0) ? T(1) / mx : T(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] *= inv;
  if (threadIdx.x == 0 && logacc && mx > T(0)) *logacc += log((double)mx);
}

// Site [p][chiL][chiR] <-> contiguous vectors.
//   mode 0: the chiR columns (vector a' = entries (u, a) of column a')
//   mode 1: the chiL rows    (vector a  = entries (u, a') of row a)
template <typename T>
__global__ void k_site_vectors(const T* __restrict__ S, int p, int chiL, int chiR, int mode, int to_vectors,
                               T* __restrict__ V, T* __restrict__ Sout, size_t zs) {
  S = zp(S, zs);
  V = zp(V, zs);
  Sout = zp(Sout, zs);
  const int n = p * chiL * chiR;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int ap = e % chiR, a = (e / chiR) % chiL, u = e / (chiR * chiL);
    size_t vi;
    if (mode == 0)
      vi = (size_t)ap * (p * chiL) + (size_t)u * chiL + a;
    else
      vi = (size_t)a * (p * chiR) + (size_t)u * chiR + ap;
    if (to_vectors)
      V[vi] = S[e];
    else
      Sout[e] = V[vi];
  }
}

template <typename T>
__global__ void k_set_unit_env(T* E, size_t zs) {
  E = zp(E, zs);
  if (threadIdx.x == 0 && blockIdx.x == 0) E[0] = T(1);
}

// lognorm[r] = lognorm[r+1] + log ||C|| + Rsum; site0 = C / ||C||
template <typename T>
__global__ void k_finish_centre(const T* __restrict__ C, int n, T* __restrict__ site0, const double* lognorm_in,
                                const double* rsum, double* lognorm_out, size_t zs) {
  C = zp(C, zs);
  site0 = zp(site0, zs);
  lognorm_in = zp(lognorm_in, zs);
  rsum = zp(rsum, zs);
  lognorm_out = zp(lognorm_out, zs);
  __shared__ double red[32];
  double part = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) part += (double)C[i] * (double)C[i];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  const double nrm = sqrt(tot);
  const T inv = nrm > 0 ? (T)(1.0 / nrm) : T(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) site0[i] = C[i] * inv;
  if (threadIdx.x == 0) *lognorm_out = *lognorm_in + log(nrm) + *rsum;
}

inline int nblk(size_t n, int t = 256) { return (int)std::min<size_t>((n + t - 1) / t, 4096); }

}  // namespace

// ---------------------------------------------------------------- host driver
template <typename T>
size_t sweep_work_elems(int cols, int chi, int bmax) {
  const size_t env = (size_t)chi * bmax * chi;
  // Lcache (cols+1 envs), R (cols+1 envs), Rcur, Rtmp, pairs
  // (16 * max(16, bmax) * chi * chi), F, Lp, C, vectors (16*chi*chi each),
  // per-state products (MAXS*chi*chi), coefficients (max(16, bmax) * MAXS), one
  // more env (per-u partial sums), per-u left weights (bmax * 16)
  return (size_t)(2 * (cols + 1) + 3) * env + (size_t)MAXP * std::max(MAXP, bmax) * chi * chi +
         4 * (size_t)MAXP * chi * chi + (size_t)MAXS * chi * chi + (size_t)std::max(MAXP, bmax) * MAXS +
         (size_t)bmax * MAXP + 64;
}

template <typename T>
cudaError_t variational_sweeps(const DevTables& tb, DevWeights<T> wt, DevMPS<T> mps, int row, int cols,
                               const int* dimA, const int* hdims, const int* hstates, const uint8_t* hgD,
                               int sweeps, T* work, double* dscratch, cudaStream_t st) {
  auto tb_dims_host = [&](int s, int k) { return hdims[(size_t)s * DIMW + k]; };
  auto hd_states = [&](int s) { return hstates[s]; };
  auto cgs_rows = [&](T* X, int nvec, int len, cudaStream_t stm) { launch_cgs2_rows<T>(X, nvec, len, nullptr, stm); };
  const int chi = (int)std::lround(std::sqrt((double)(mps.site_stride / MAXP)));
  const size_t env = (size_t)chi * tb.bmax * chi;
  T* Lc = work;                                 // [cols+1][env]
  T* Rs = Lc + (size_t)(cols + 1) * env;        // [cols+1][env]
  T* Rcur = Rs + (size_t)(cols + 1) * env;      // [env]
  T* Rtmp = Rcur + env;                         // [env]
  T* Ctmp = Rtmp + env;                         // [env] per-u partial sums
  T* Pp = Ctmp + env;                           // pairs [16*max(16,bmax)*chi*chi]
  T* F = Pp + (size_t)MAXP * std::max(MAXP, tb.bmax) * chi * chi;  // [16*chi*chi]
  T* Lp = F + (size_t)MAXP * chi * chi;         // [chi*16*chi]
  T* C = Lp + (size_t)MAXP * chi * chi;         // [16*chi*chi]
  T* Vv = C + (size_t)MAXP * chi * chi;         // vectors [16*chi*chi]
  T* G = Vv + (size_t)MAXP * chi * chi;         // per-state products [MAXS*chi*chi]
  T* Cf = G + (size_t)MAXS * chi * chi;         // state coefficients [max(16,bmax)*MAXS] (K <= DU, DL or DR)
  T* Bu = Cf + (size_t)std::max(MAXP, tb.bmax) * MAXS;  // left weights of one up index [bmax*16]
  double* rsum = dscratch;                      // [1]
  double* junk = dscratch + 1;
  auto site_ptr = [&](int r, int j) { return mps.A + (size_t)(r * cols + j) * mps.site_stride; };
  auto dims = [&](int r, int j) { return dimA + ((size_t)r * cols + j) * 3; };
  auto zero_env = [&](T* E) { return zfill(E, 0, sizeof(T) * env, st); };
  // every pointer below lies in work, dscratch, the MPS or the tables
  if (!zok(tb, wt, mps, work, work + sweep_work_elems<T>(cols, chi, tb.bmax) - 1, dscratch + 1))
    return cudaErrorInvalidValue;
  cudaError_t err;
#define SPG_TRY(x)                 \
  do {                             \
    if ((err = (x)) != cudaSuccess) return err; \
  } while (0)

  // Environments are E[m][a][b] (MPO bond m < 16 outermost, phi bond a, psi
  // bond b).  Per site: tables' dims from the host copy.
  auto xgemm = [&](int s, int nq, int n2, int M, int N, int K, const T* A, XOff oa, int sAi, int sAk, const T* B,
                   XOff ob, int sBk, int sBj, T* C) {
    // variant v: 2^v states per block (FP64 up to 2: the tiles of 4 states
    // exceed the static shared memory); a variant whose grid would have
    // more than 65535 blocks along z is not valid for the shape
    auto grid_of = [&](int v) {
      const int qpb = 1 << v;
      return dim3((N + 31) / 32, (M + 31) / 32, (unsigned)(((nq + qpb - 1) / qpb) * zn()));
    };
    auto run = [&](int v) {
      const dim3 grid = grid_of(v);
      if (v == 0)
        k_xgemm<T, 1><<<grid, 64, 0, st>>>(tb, s, n2, M, N, K, A, oa, sAi, sAk, B, ob, sBk, sBj, C, nq, zs());
      else if (v == 1)
        k_xgemm<T, 2><<<grid, 128, 0, st>>>(tb, s, n2, M, N, K, A, oa, sAi, sAk, B, ob, sBk, sBj, C, nq, zs());
      else if constexpr (sizeof(T) == 4)
        k_xgemm<T, 4><<<grid, 256, 0, st>>>(tb, s, n2, M, N, K, A, oa, sAi, sAk, B, ob, sBk, sBj, C, nq, zs());
    };
    const int nvar = sizeof(T) == 4 ? 3 : 2;
    unsigned valid = 0;
    for (int v = 0; v < nvar; ++v)
      if ((size_t)((nq + (1 << v) - 1) >> v) * zn() <= 65535) valid |= 1u << v;
    const long long shape[] = {(long long)sizeof(T), M, N, K, nq, sAi, sAk, sBk, sBj};
    const int v = tune_pick("k_xgemm", shape, 9, st, nvar, valid, nvar - 1, run);
    count_launches("k_xgemm", st, 2.0 * nq * M * N * K);
    run(v);
  };
  auto coef = [&](int s, int mode, int K, int u = 0, int g = 0) {
    const int d = hd_states(s);
    count_launches("k_state_coef", st);
    k_state_coef<T><<<dim3(nblk((size_t)K * d), 1, zn()), 256, 0, st>>>(tb, wt, s, mode, K, u, g, Cf, zs());
  };
  // king's graph: per up index u, the right-bond offset g = gD_up[u]
  auto g_of = [&](int s, int u) { return s >= cols ? (int)hgD[(size_t)(s - cols) * MAXP + u] : 0; };
  auto u_coupled = [&](int s) { return tb_dims_host(s, D_UCPL) != 0; };
  auto axpy = [&](T* y, const T* x, size_t n) {
    count_launches("k_axpy", st);
    k_axpy<T><<<dim3(nblk(n), 1, zn()), 256, 0, st>>>(y, x, n, zs());
  };
  // Lp[h][a][b] = sum_l bA[l / Gin][u] bL[l][h] E[l][a][b]
  auto left_prime_u = [&](int s, const T* Lenv, int chiA, int chiB, int u) {
    const int DL = tb_dims_host(s, 0), NL = tb_dims_host(s, 4);
    count_launches("k_left_weights_u", st);
    k_left_weights_u<T><<<dim3(nblk((size_t)DL * MAXP), 1, zn()), 256, 0, st>>>(tb, wt, s, u, Bu, zs());
    gemm2<T>(true, false, NL, chiA * chiB, DL, Bu, MAXP, Lenv, chiA * chiB, Lp, chiA * chiB, st);
  };
  // Lp[h][a][b] = sum_l bL[l][h] E[l][a][b]
  auto left_prime = [&](int s, const T* Lenv, int chiA, int chiB) {
    const int DL = tb_dims_host(s, 0), NL = tb_dims_host(s, 4);
    gemm2<T>(true, false, NL, chiA * chiB, DL, wt.bL + (size_t)s * tb.lstride, MAXP, Lenv, chiA * chiB, Lp,
             chiA * chiB, st);
  };
  // F[v][a][a'] = sum_u bU[u][v] P[u][a][a']
  auto phi_prime = [&](int s, const T* P, int DU, int chiA, int chiAr) {
    const int NU = tb_dims_host(s, 5);
    gemm2<T>(true, false, NU, chiA * chiAr, DU, wt.bU + (size_t)s * 256, 16, P, chiA * chiAr, F, chiA * chiAr, st);
  };
  // Pr[s'][r][b][a'] = sum_b' B[s'][b][b'] R[r][a'][b']
  auto pairs_right = [&](int s, const T* B, int p, int chiBl, int chiBr, const T* Renv, int chiAr) {
    const int DR = tb_dims_host(s, 1);
    xgemm(s, p * DR, DR, chiBl, chiAr, chiBr, B, XOff{5, 0, (long long)chiBl * chiBr, 0}, chiBr, 1, Renv,
          XOff{6, 0, (long long)chiAr * chiBr, 0}, 1, chiBr, Pp);
  };
  // local tensor C[u][a][a'] at site j from left env Lenv, right env Renv
  auto local = [&](int j, const T* Lenv, const T* Renv) -> cudaError_t {
    const int s = row * cols + j;
    const int* dB = dims(row + 1, j);
    const int* dP = dims(row, j);
    const int p = dB[0], chiBl = dB[1], chiBr = dB[2];
    const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
    const int DR = tb_dims_host(s, 1), d = hd_states(s);
    const T* B = site_ptr(row + 1, j);
    if (u_coupled(s)) {
      // one up index at a time: C[u] = sum_x bU[u][PU x] w(x) Lp_u[PL x] Pr[PD x][PR x * Gout + g_u]
      const int Gout = tb_dims_host(s, D_GOUT);
      pairs_right(s, B, p, chiBl, chiBr, Renv, chiAr);
      for (int u = 0; u < DU; ++u) {
        const int g = g_of(s, u);
        left_prime_u(s, Lenv, chiA, chiBl, u);
        xgemm(s, d, 1, chiA, chiAr, chiBl, Lp, XOff{1, 0, (long long)chiA * chiBl, 0}, chiBl, 1,
              Pp + (size_t)g * chiBl * chiAr,
              XOff{4, 2, (long long)DR * chiBl * chiAr, (long long)Gout * chiBl * chiAr}, chiAr, 1, G);
        coef(s, 3, 1, u, g);
        gemm2<T>(false, false, 1, chiA * chiAr, d, Cf, d, G, chiA * chiAr, C + (size_t)u * chiA * chiAr,
                 chiA * chiAr, st);
      }
      return cudaGetLastError();
    }
    left_prime(s, Lenv, chiA, chiBl);
    pairs_right(s, B, p, chiBl, chiBr, Renv, chiAr);
    // G_x[a][a'] = sum_b Lp[PL x][a][b] Pr[PD x][PR x][b][a']
    xgemm(s, d, 1, chiA, chiAr, chiBl, Lp, XOff{1, 0, (long long)chiA * chiBl, 0}, chiBl, 1, Pp,
          XOff{4, 2, (long long)DR * chiBl * chiAr, (long long)chiBl * chiAr}, chiAr, 1, G);
    coef(s, 0, DU);
    gemm2<T>(false, false, DU, chiA * chiAr, d, Cf, d, G, chiA * chiAr, C, chiA * chiAr, st);
    return cudaGetLastError();
  };
  auto env_right = [&](int j, const T* Renv, T* out, double* logacc) -> cudaError_t {
    const int s = row * cols + j;
    const int* dB = dims(row + 1, j);
    const int* dP = dims(row, j);
    const int p = dB[0], chiBl = dB[1], chiBr = dB[2];
    const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
    const int DL = tb_dims_host(s, 0), DR = tb_dims_host(s, 1), d = hd_states(s);
    const T* B = site_ptr(row + 1, j);
    const T* P = site_ptr(row, j);
    if (u_coupled(s)) {
      // out[l] = sum_u sum_x bA[l/Gin][u] bL[l][PL x] bU[u][PU x] w(x) P[u] Pr[PD x][PR x * Gout + g_u]
      const int Gout = tb_dims_host(s, D_GOUT);
      pairs_right(s, B, p, chiBl, chiBr, Renv, chiAr);
      SPG_TRY(zero_env(out));
      for (int u = 0; u < DU; ++u) {
        const int g = g_of(s, u);
        xgemm(s, d, 1, chiA, chiBl, chiAr, P + (size_t)u * chiA * chiAr, XOff{0, 0, 0, 0}, chiAr, 1,
              Pp + (size_t)g * chiBl * chiAr,
              XOff{4, 2, (long long)DR * chiBl * chiAr, (long long)Gout * chiBl * chiAr}, 1, chiAr, G);
        coef(s, 4, DL, u, g);
        gemm2<T>(false, false, DL, chiA * chiBl, d, Cf, d, G, chiA * chiBl, Ctmp, chiA * chiBl, st);
        axpy(out, Ctmp, (size_t)DL * chiA * chiBl);
      }
      count_launches("k_scale_max", st);
      k_scale_max<T><<<dim3(1, 1, zn()), 1024, 0, st>>>(out, (int)env, logacc, zs());
      return cudaGetLastError();
    }
    phi_prime(s, P, DU, chiA, chiAr);
    pairs_right(s, B, p, chiBl, chiBr, Renv, chiAr);
    // Y_x[a][b] = sum_a' F[PU x][a][a'] Pr[PD x][PR x][b][a']
    xgemm(s, d, 1, chiA, chiBl, chiAr, F, XOff{3, 0, (long long)chiA * chiAr, 0}, chiAr, 1, Pp,
          XOff{4, 2, (long long)DR * chiBl * chiAr, (long long)chiBl * chiAr}, 1, chiAr, G);
    coef(s, 1, DL);
    SPG_TRY(zero_env(out));
    gemm2<T>(false, false, DL, chiA * chiBl, d, Cf, d, G, chiA * chiBl, out, chiA * chiBl, st);
    count_launches("k_scale_max", st);
    k_scale_max<T><<<dim3(1, 1, zn()), 1024, 0, st>>>(out, (int)env, logacc, zs());
    return cudaGetLastError();
  };
  auto env_left = [&](int j, const T* Lenv, T* out) -> cudaError_t {
    const int s = row * cols + j;
    const int* dB = dims(row + 1, j);
    const int* dP = dims(row, j);
    const int p = dB[0], chiBl = dB[1], chiBr = dB[2];
    const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
    const int DR = tb_dims_host(s, 1), NL = tb_dims_host(s, 4), d = hd_states(s);
    const T* B = site_ptr(row + 1, j);
    const T* P = site_ptr(row, j);
    if (u_coupled(s)) {
      // out[r] = sum_u sum_x [PR x * Gout + g_u == r] bU[u][PU x] w(x) P[u]^T Ql_u[PL x][PD x]
      SPG_TRY(zero_env(out));
      for (int u = 0; u < DU; ++u) {
        const int g = g_of(s, u);
        left_prime_u(s, Lenv, chiA, chiBl, u);
        xgemm(s, NL * p, p, chiA, chiBr, chiBl, Lp, XOff{5, 0, (long long)chiA * chiBl, 0}, chiBl, 1, B,
              XOff{6, 0, (long long)chiBl * chiBr, 0}, chiBr, 1, Pp);
        xgemm(s, d, 1, chiAr, chiBr, chiA, P + (size_t)u * chiA * chiAr, XOff{0, 0, 0, 0}, 1, chiAr, Pp,
              XOff{1, 4, (long long)p * chiA * chiBr, (long long)chiA * chiBr}, chiBr, 1, G);
        coef(s, 5, DR, u, g);
        gemm2<T>(false, false, DR, chiAr * chiBr, d, Cf, d, G, chiAr * chiBr, Ctmp, chiAr * chiBr, st);
        axpy(out, Ctmp, (size_t)DR * chiAr * chiBr);
      }
      count_launches("k_scale_max", st);
      k_scale_max<T><<<dim3(1, 1, zn()), 1024, 0, st>>>(out, (int)env, junk, zs());
      return cudaGetLastError();
    }
    left_prime(s, Lenv, chiA, chiBl);
    // Ql[h][s'][a][b'] = sum_b Lp[h][a][b] B[s'][b][b']
    xgemm(s, NL * p, p, chiA, chiBr, chiBl, Lp, XOff{5, 0, (long long)chiA * chiBl, 0}, chiBl, 1, B,
          XOff{6, 0, (long long)chiBl * chiBr, 0}, chiBr, 1, Pp);
    phi_prime(s, P, DU, chiA, chiAr);
    // Z_x[a'][b'] = sum_a F[PU x][a][a'] Ql[PL x][PD x][a][b']
    xgemm(s, d, 1, chiAr, chiBr, chiA, F, XOff{3, 0, (long long)chiA * chiAr, 0}, 1, chiAr, Pp,
          XOff{1, 4, (long long)p * chiA * chiBr, (long long)chiA * chiBr}, chiBr, 1, G);
    coef(s, 2, DR);
    SPG_TRY(zero_env(out));
    gemm2<T>(false, false, DR, chiAr * chiBr, d, Cf, d, G, chiAr * chiBr, out, chiAr * chiBr, st);
    count_launches("k_scale_max", st);
    k_scale_max<T><<<dim3(1, 1, zn()), 1024, 0, st>>>(out, (int)env, junk, zs());
    return cudaGetLastError();
  };

  for (int sw = 0; sw < sweeps; ++sw) {
    // right environments of the current (right-orthonormal) phi
    SPG_TRY(zero_env(Rs + (size_t)(cols - 1) * env));
    count_launches("k_set_unit_env", st);
    k_set_unit_env<T><<<dim3(1, 1, zn()), 32, 0, st>>>(Rs + (size_t)(cols - 1) * env, zs());
    for (int j = cols - 1; j >= 1; --j) SPG_TRY(env_right(j, Rs + (size_t)j * env, Rs + (size_t)(j - 1) * env, junk));
    // left to right
    SPG_TRY(zero_env(Lc));
    count_launches("k_set_unit_env", st);
    k_set_unit_env<T><<<dim3(1, 1, zn()), 32, 0, st>>>(Lc, zs());
    for (int j = 0; j < cols - 1; ++j) {
      SPG_TRY(local(j, Lc + (size_t)j * env, Rs + (size_t)j * env));
      const int* dP = dims(row, j);
      const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
      const int n = DU * chiA * chiAr;
      count_launches("k_site_vectors", st);
      k_site_vectors<T><<<dim3(nblk(n), 1, zn()), 256, 0, st>>>(C, DU, chiA, chiAr, 0, 1, Vv, nullptr, zs());
      cgs_rows(Vv, chiAr, DU * chiA, st);
      count_launches("k_site_vectors", st);
      k_site_vectors<T><<<dim3(nblk(n), 1, zn()), 256, 0, st>>>(nullptr, DU, chiA, chiAr, 0, 0, Vv, site_ptr(row, j), zs());
      SPG_TRY(env_left(j, Lc + (size_t)j * env, Lc + (size_t)(j + 1) * env));
    }
    // right to left
    SPG_TRY(zfill(rsum, 0, sizeof(double), st));
    SPG_TRY(zero_env(Rcur));
    count_launches("k_set_unit_env", st);
    k_set_unit_env<T><<<dim3(1, 1, zn()), 32, 0, st>>>(Rcur, zs());
    for (int j = cols - 1; j >= 1; --j) {
      SPG_TRY(local(j, Lc + (size_t)j * env, Rcur));
      const int* dP = dims(row, j);
      const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
      const int n = DU * chiA * chiAr;
      count_launches("k_site_vectors", st);
      k_site_vectors<T><<<dim3(nblk(n), 1, zn()), 256, 0, st>>>(C, DU, chiA, chiAr, 1, 1, Vv, nullptr, zs());
      cgs_rows(Vv, chiA, DU * chiAr, st);
      count_launches("k_site_vectors", st);
      k_site_vectors<T><<<dim3(nblk(n), 1, zn()), 256, 0, st>>>(nullptr, DU, chiA, chiAr, 1, 0, Vv, site_ptr(row, j), zs());
      SPG_TRY(env_right(j, Rcur, Rtmp, rsum));
      SPG_TRY(zcopy(Rcur, Rtmp, sizeof(T) * env, st));
    }
    SPG_TRY(local(0, Lc, Rcur));
    const int* dP = dims(row, 0);
    count_launches("k_finish_centre", st);
    k_finish_centre<T><<<dim3(1, 1, zn()), 256, 0, st>>>(C, dP[0] * dP[1] * dP[2], site_ptr(row, 0),
                                                         mps.lognorm + row + 1, rsum, mps.lognorm + row, zs());
  }
#undef SPG_TRY
  return cudaGetLastError();
}

template size_t sweep_work_elems<double>(int, int, int);
template size_t sweep_work_elems<float>(int, int, int);
template cudaError_t variational_sweeps<double>(const DevTables&, DevWeights<double>, DevMPS<double>, int, int,
                                                const int*, const int*, const int*, const uint8_t*, int, double*,
                                                double*, cudaStream_t);
template cudaError_t variational_sweeps<float>(const DevTables&, DevWeights<float>, DevMPS<float>, int, int,
                                               const int*, const int*, const int*, const uint8_t*, int, float*,
                                               double*, cudaStream_t);

}  // namespace spg
