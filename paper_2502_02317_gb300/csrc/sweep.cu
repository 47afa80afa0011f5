// Variational sweeps of a boundary MPS (S4): one-site updates of phi that
// maximise |<phi| W psi>| with the other sites orthonormal, left to right
// (QR moves the centre right) then right to left (LQ moves it left).
//
// Paper: Sec. 3.1 (MpsParameters(bond_dim, num_sweeps)); Sec. 2 (boundary
// MPS contraction of the PEPS).
//
// Layouts (row r of the MPO, psi = B_{r+1} sites B[s][b][b'], phi sites
// P[u][a][a'], both [p][chi_l][chi_r]):
//   environments  E[a][l][b]  (phi bond, MPO bond < 16, psi bond)
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

// Per-site tables staged in shared memory.
template <typename T>
struct SiteSmem {
  T w[MAXS];
  T bL[256];
  T bU[256];
  uint8_t PL[MAXS], PR[MAXS], PU[MAXS], PD[MAXS];
};

template <typename T>
__device__ void stage_site(SiteSmem<T>& sm, const DevTables& tb, const DevWeights<T>& wt, int s) {
  const size_t so = (size_t)s * tb.dmax;
  const int d = tb.d[s];
  for (int x = threadIdx.x; x < d; x += blockDim.x) {
    sm.w[x] = wt.w[so + x];
    sm.PL[x] = tb.PL[so + x];
    sm.PR[x] = tb.PR[so + x];
    sm.PU[x] = tb.PU[so + x];
    sm.PD[x] = tb.PD[so + x];
  }
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    sm.bL[e] = wt.bL[(size_t)s * 256 + e];
    sm.bU[e] = wt.bU[(size_t)s * 256 + e];
  }
}

// F[v][a][a'] = sum_u bU[u][v] P[u][a][a']   (v < NU)
template <typename T>
__global__ void k_phi_prime(DevTables tb, DevWeights<T> wt, int s, const T* __restrict__ P, int DU, int chiL,
                            int chiR, T* __restrict__ F) {
  const int NU = tb.dims[s * 8 + 5];
  const int n = NU * chiL * chiR;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int v = e / (chiL * chiR), rest = e % (chiL * chiR);
    T acc = T(0);
    for (int u = 0; u < DU; ++u) acc += wt.bU[(size_t)s * 256 + u * 16 + v] * P[(size_t)u * chiL * chiR + rest];
    F[e] = acc;
  }
}

// Lp[a][h][b] = sum_l L[a][l][b] bL[l][h]   (h < NL)
template <typename T>
__global__ void k_left_prime(DevTables tb, DevWeights<T> wt, int s, const T* __restrict__ L, int chiA, int DL,
                             int chiB, T* __restrict__ Lp) {
  const int NL = tb.dims[s * 8 + 4];
  const int n = chiA * NL * chiB;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int b = e % chiB, h = (e / chiB) % NL, a = e / (chiB * NL);
    T acc = T(0);
    for (int l = 0; l < DL; ++l) acc += L[((size_t)a * MAXP + l) * chiB + b] * wt.bL[(size_t)s * 256 + l * 16 + h];
    Lp[((size_t)a * MAXP + h) * chiB + b] = acc;
  }
}

// Pr[s][r][b][a'] = sum_b' B[s][b][b'] R[a'][r][b']       (right pairs)
template <typename T>
__global__ void k_pairs_right(const T* __restrict__ B, int p, int chiBl, int chiBr, const T* __restrict__ R,
                              int chiA, int DR, T* __restrict__ Pr) {
  const size_t n = (size_t)p * DR * chiBl * chiA;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int ap = e % chiA;
    size_t t = e / chiA;
    const int b = t % chiBl;
    t /= chiBl;
    const int r = t % DR, sg = (int)(t / DR);
    const T* brow = B + ((size_t)sg * chiBl + b) * chiBr;
    const T* rrow = R + ((size_t)ap * MAXP + r) * chiBr;
    T acc = T(0);
    for (int bp = 0; bp < chiBr; ++bp) acc += brow[bp] * rrow[bp];
    Pr[e] = acc;
  }
}

// Ql[h][s][a][b'] = sum_b Lp[a][h][b] B[s][b][b']           (left pairs)
template <typename T>
__global__ void k_pairs_left(const T* __restrict__ Lp, int NL, int chiA, int chiBl, const T* __restrict__ B, int p,
                             int chiBr, T* __restrict__ Ql) {
  const size_t n = (size_t)NL * p * chiA * chiBr;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int bp = e % chiBr;
    size_t t = e / chiBr;
    const int a = t % chiA;
    t /= chiA;
    const int sg = t % p, h = (int)(t / p);
    const T* lrow = Lp + ((size_t)a * MAXP + h) * chiBl;
    const T* bcol = B + (size_t)sg * chiBl * chiBr + bp;
    T acc = T(0);
    for (int b = 0; b < chiBl; ++b) acc += lrow[b] * bcol[(size_t)b * chiBr];
    Ql[e] = acc;
  }
}

// local: C[u][a][a'] = sum_x w(x) bU[u][PU x] sum_b Lp[a][PL x][b] Pr[PD x][PR x][b][a']
// one thread per (a, a'), states grouped into the NU accumulators of PU x.
template <typename T>
__global__ void k_local_x(DevTables tb, DevWeights<T> wt, int s, const T* __restrict__ Lp, const T* __restrict__ Pr,
                          int chiA, int chiAr, int chiBl, int DR, int DU, T* __restrict__ C) {
  __shared__ SiteSmem<T> sm;
  stage_site(sm, tb, wt, s);
  __syncthreads();
  const int d = tb.d[s], NU = tb.dims[s * 8 + 5];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= chiA * chiAr) return;
  const int a = e / chiAr, ap = e % chiAr;
  T H[MAXP];
#pragma unroll
  for (int v = 0; v < MAXP; ++v) H[v] = T(0);
  for (int x = 0; x < d; ++x) {
    const T* lrow = Lp + ((size_t)a * MAXP + sm.PL[x]) * chiBl;
    const T* pcol = Pr + (((size_t)sm.PD[x] * DR + sm.PR[x]) * chiBl) * chiAr + ap;
    T g0 = T(0), g1 = T(0);
    int b = 0;
    for (; b + 1 < chiBl; b += 2) {
      g0 += lrow[b] * pcol[(size_t)b * chiAr];
      g1 += lrow[b + 1] * pcol[(size_t)(b + 1) * chiAr];
    }
    if (b < chiBl) g0 += lrow[b] * pcol[(size_t)b * chiAr];
    const T g = sm.w[x] * (g0 + g1);
    const int v = sm.PU[x];
#pragma unroll
    for (int q = 0; q < MAXP; ++q)
      if (q == v) H[q] += g;
  }
  for (int u = 0; u < DU; ++u) {
    T acc = T(0);
#pragma unroll
    for (int v = 0; v < MAXP; ++v)
      if (v < NU) acc += sm.bU[u * 16 + v] * H[v];
    C[((size_t)u * chiA + a) * chiAr + ap] = acc;
  }
}

// right environment: Rn[a][l][b] = sum_h bL[l][h] sum_{x: PL x = h} w(x)
//                    sum_a' F[PU x][a][a'] Pr[PD x][PR x][b][a']
// one thread per (a, b).
template <typename T>
__global__ void k_env_right_x(DevTables tb, DevWeights<T> wt, int s, const T* __restrict__ F, const T* __restrict__ Pr,
                              int chiA, int chiAr, int chiBl, int DR, int DL, T* __restrict__ Rn) {
  __shared__ SiteSmem<T> sm;
  stage_site(sm, tb, wt, s);
  __syncthreads();
  const int d = tb.d[s], NL = tb.dims[s * 8 + 4];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= chiA * chiBl) return;
  const int a = e / chiBl, b = e % chiBl;
  T Y[MAXP];
#pragma unroll
  for (int h = 0; h < MAXP; ++h) Y[h] = T(0);
  for (int x = 0; x < d; ++x) {
    const T* frow = F + ((size_t)sm.PU[x] * chiA + a) * chiAr;
    const T* prow = Pr + (((size_t)sm.PD[x] * DR + sm.PR[x]) * chiBl + b) * chiAr;
    T g0 = T(0), g1 = T(0);
    int ap = 0;
    for (; ap + 1 < chiAr; ap += 2) {
      g0 += frow[ap] * prow[ap];
      g1 += frow[ap + 1] * prow[ap + 1];
    }
    if (ap < chiAr) g0 += frow[ap] * prow[ap];
    const T g = sm.w[x] * (g0 + g1);
    const int h = sm.PL[x];
#pragma unroll
    for (int q = 0; q < MAXP; ++q)
      if (q == h) Y[q] += g;
  }
  for (int l = 0; l < MAXP; ++l) {
    T acc = T(0);
    if (l < DL) {
#pragma unroll
      for (int h = 0; h < MAXP; ++h)
        if (h < NL) acc += sm.bL[l * 16 + h] * Y[h];
    }
    Rn[((size_t)a * MAXP + l) * chiBl + b] = acc;
  }
}

// left environment: Ln[a'][r][b'] = sum_{x: PR x = r} w(x)
//                   sum_a F[PU x][a][a'] Ql[PL x][PD x][a][b']
// one thread per (a', b').
template <typename T>
__global__ void k_env_left_x(DevTables tb, DevWeights<T> wt, int s, const T* __restrict__ F, const T* __restrict__ Ql,
                             int chiA, int chiAr, int chiBr, int p, int DR, T* __restrict__ Ln) {
  __shared__ SiteSmem<T> sm;
  stage_site(sm, tb, wt, s);
  __syncthreads();
  const int d = tb.d[s];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= chiAr * chiBr) return;
  const int ap = e / chiBr, bp = e % chiBr;
  T O[MAXP];
#pragma unroll
  for (int r = 0; r < MAXP; ++r) O[r] = T(0);
  for (int x = 0; x < d; ++x) {
    const T* fcol = F + (size_t)sm.PU[x] * chiA * chiAr + ap;
    const T* qcol = Ql + (((size_t)sm.PL[x] * p + sm.PD[x]) * chiA) * chiBr + bp;
    T g0 = T(0), g1 = T(0);
    int a = 0;
    for (; a + 1 < chiA; a += 2) {
      g0 += fcol[(size_t)a * chiAr] * qcol[(size_t)a * chiBr];
      g1 += fcol[(size_t)(a + 1) * chiAr] * qcol[(size_t)(a + 1) * chiBr];
    }
    if (a < chiA) g0 += fcol[(size_t)a * chiAr] * qcol[(size_t)a * chiBr];
    const T g = sm.w[x] * (g0 + g1);
    const int r = sm.PR[x];
#pragma unroll
    for (int q = 0; q < MAXP; ++q)
      if (q == r) O[q] += g;
  }
  for (int r = 0; r < MAXP; ++r) Ln[((size_t)ap * MAXP + r) * chiBr + bp] = r < DR ? O[r] : T(0);
}

// In-place scaling of buf[0..n) to max |.| = 1, log of the scale added to *logacc.
template <typename T>
__global__ void k_scale_max(T* buf, int n, double* logacc) {
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
                               T* __restrict__ V, T* __restrict__ Sout) {
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
__global__ void k_set_unit_env(T* E) {
  if (threadIdx.x == 0 && blockIdx.x == 0) E[0] = T(1);
}

// lognorm[r] = lognorm[r+1] + log ||C|| + Rsum; site0 = C / ||C||
template <typename T>
__global__ void k_finish_centre(const T* __restrict__ C, int n, T* __restrict__ site0, const double* lognorm_in,
                                const double* rsum, double* lognorm_out) {
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
size_t sweep_work_elems(int cols, int chi) {
  const size_t env = (size_t)chi * MAXP * chi;
  // Lcache (cols+1 envs), R (cols+1 envs), Rcur, pairs (16*16*chi*chi), F and
  // Lp (16*chi*chi each), C (16*chi*chi), vectors (16*chi*chi), doubles
  return (size_t)(2 * (cols + 1) + 2) * env + (size_t)MAXP * MAXP * chi * chi + 4 * (size_t)MAXP * chi * chi + 64;
}

template <typename T>
cudaError_t variational_sweeps(const DevTables& tb, DevWeights<T> wt, DevMPS<T> mps, int row, int cols,
                               const int* dimA, const int* hdims, int sweeps, T* work, double* dscratch,
                               cudaStream_t st) {
  auto tb_dims_host = [&](int s, int k) { return hdims[s * 8 + k]; };
  auto cgs_rows = [&](T* X, int nvec, int len, cudaStream_t stm) { launch_cgs2_rows<T>(X, nvec, len, nullptr, stm); };
  const int chi = (int)std::lround(std::sqrt((double)(mps.site_stride / MAXP)));
  const size_t env = (size_t)chi * MAXP * chi;
  T* Lc = work;                                 // [cols+1][env]
  T* Rs = Lc + (size_t)(cols + 1) * env;        // [cols+1][env]
  T* Rcur = Rs + (size_t)(cols + 1) * env;      // [env]
  T* Rtmp = Rcur + env;                         // [env]
  T* Pp = Rtmp + env;                           // pairs [16*16*chi*chi]
  T* F = Pp + (size_t)MAXP * MAXP * chi * chi;  // [16*chi*chi]
  T* Lp = F + (size_t)MAXP * chi * chi;         // [chi*16*chi]
  T* C = Lp + (size_t)MAXP * chi * chi;         // [16*chi*chi]
  T* Vv = C + (size_t)MAXP * chi * chi;         // vectors [16*chi*chi]
  double* rsum = dscratch;                      // [1]
  double* junk = dscratch + 1;
  auto site_ptr = [&](int r, int j) { return mps.A + (size_t)(r * cols + j) * mps.site_stride; };
  auto dims = [&](int r, int j) { return dimA + ((size_t)r * cols + j) * 3; };
  auto zero_env = [&](T* E) { return cudaMemsetAsync(E, 0, sizeof(T) * env, st); };
  cudaError_t err;
#define SPG_TRY(x)                 \
  do {                             \
    if ((err = (x)) != cudaSuccess) return err; \
  } while (0)

  // local tensor C at site j from left env Lenv, right env Renv
  auto local = [&](int j, const T* Lenv, const T* Renv) -> cudaError_t {
    const int s = row * cols + j;
    const int* dB = dims(row + 1, j);
    const int* dP = dims(row, j);
    const int p = dB[0], chiBl = dB[1], chiBr = dB[2];
    const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
    const int DL = tb_dims_host(s, 0), DR = tb_dims_host(s, 1), NL = tb_dims_host(s, 4);
    (void)NL;
    const T* B = site_ptr(row + 1, j);
    count_launches("k_left_prime", st);
    k_left_prime<T><<<nblk((size_t)chiA * MAXP * chiBl), 256, 0, st>>>(tb, wt, s, Lenv, chiA, DL, chiBl, Lp);
    count_launches("k_pairs_right", st, 2.0 * p * DR * chiBl * chiAr * chiBr);
    k_pairs_right<T><<<nblk((size_t)p * DR * chiBl * chiAr), 256, 0, st>>>(B, p, chiBl, chiBr, Renv, chiAr, DR, Pp);
    count_launches("k_local_x", st);
    k_local_x<T><<<nblk((size_t)chiA * chiAr, 128), 128, 0, st>>>(tb, wt, s, Lp, Pp, chiA, chiAr, chiBl, DR, DU, C);
    return cudaGetLastError();
  };
  auto env_right = [&](int j, const T* Renv, T* out, double* logacc) -> cudaError_t {
    const int s = row * cols + j;
    const int* dB = dims(row + 1, j);
    const int* dP = dims(row, j);
    const int p = dB[0], chiBl = dB[1], chiBr = dB[2];
    const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
    const int DL = tb_dims_host(s, 0), DR = tb_dims_host(s, 1);
    const T* B = site_ptr(row + 1, j);
    const T* P = site_ptr(row, j);
    count_launches("k_phi_prime", st);
    k_phi_prime<T><<<nblk((size_t)MAXP * chiA * chiAr), 256, 0, st>>>(tb, wt, s, P, DU, chiA, chiAr, F);
    count_launches("k_pairs_right", st, 2.0 * p * DR * chiBl * chiAr * chiBr);
    k_pairs_right<T><<<nblk((size_t)p * DR * chiBl * chiAr), 256, 0, st>>>(B, p, chiBl, chiBr, Renv, chiAr, DR, Pp);
    SPG_TRY(zero_env(out));
    count_launches("k_env_right_x", st);
    k_env_right_x<T><<<nblk((size_t)chiA * chiBl, 128), 128, 0, st>>>(tb, wt, s, F, Pp, chiA, chiAr, chiBl, DR, DL,
                                                                      out);
    count_launches("k_scale_max", st);
    k_scale_max<T><<<1, 1024, 0, st>>>(out, (int)env, logacc);
    return cudaGetLastError();
  };
  auto env_left = [&](int j, const T* Lenv, T* out) -> cudaError_t {
    const int s = row * cols + j;
    const int* dB = dims(row + 1, j);
    const int* dP = dims(row, j);
    const int p = dB[0], chiBl = dB[1], chiBr = dB[2];
    const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
    const int DL = tb_dims_host(s, 0), DR = tb_dims_host(s, 1), NL = tb_dims_host(s, 4);
    const T* B = site_ptr(row + 1, j);
    const T* P = site_ptr(row, j);
    count_launches("k_left_prime", st);
    k_left_prime<T><<<nblk((size_t)chiA * MAXP * chiBl), 256, 0, st>>>(tb, wt, s, Lenv, chiA, DL, chiBl, Lp);
    count_launches("k_pairs_left", st, 2.0 * NL * p * chiA * chiBr * chiBl);
    k_pairs_left<T><<<nblk((size_t)NL * p * chiA * chiBr), 256, 0, st>>>(Lp, NL, chiA, chiBl, B, p, chiBr, Pp);
    count_launches("k_phi_prime", st);
    k_phi_prime<T><<<nblk((size_t)MAXP * chiA * chiAr), 256, 0, st>>>(tb, wt, s, P, DU, chiA, chiAr, F);
    SPG_TRY(zero_env(out));
    count_launches("k_env_left_x", st);
    k_env_left_x<T><<<nblk((size_t)chiAr * chiBr, 128), 128, 0, st>>>(tb, wt, s, F, Pp, chiA, chiAr, chiBr, p, DR,
                                                                     out);
    count_launches("k_scale_max", st);
    k_scale_max<T><<<1, 1024, 0, st>>>(out, (int)env, junk);
    return cudaGetLastError();
  };

  for (int sw = 0; sw < sweeps; ++sw) {
    // right environments of the current (right-orthonormal) phi
    SPG_TRY(zero_env(Rs + (size_t)(cols - 1) * env));
    count_launches("k_set_unit_env", st);
    k_set_unit_env<T><<<1, 32, 0, st>>>(Rs + (size_t)(cols - 1) * env);
    for (int j = cols - 1; j >= 1; --j) SPG_TRY(env_right(j, Rs + (size_t)j * env, Rs + (size_t)(j - 1) * env, junk));
    // left to right
    SPG_TRY(zero_env(Lc));
    count_launches("k_set_unit_env", st);
    k_set_unit_env<T><<<1, 32, 0, st>>>(Lc);
    for (int j = 0; j < cols - 1; ++j) {
      SPG_TRY(local(j, Lc + (size_t)j * env, Rs + (size_t)j * env));
      const int* dP = dims(row, j);
      const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
      const int n = DU * chiA * chiAr;
      count_launches("k_site_vectors", st);
      k_site_vectors<T><<<nblk(n), 256, 0, st>>>(C, DU, chiA, chiAr, 0, 1, Vv, nullptr);
      cgs_rows(Vv, chiAr, DU * chiA, st);
      count_launches("k_site_vectors", st);
      k_site_vectors<T><<<nblk(n), 256, 0, st>>>(nullptr, DU, chiA, chiAr, 0, 0, Vv, site_ptr(row, j));
      SPG_TRY(env_left(j, Lc + (size_t)j * env, Lc + (size_t)(j + 1) * env));
    }
    // right to left
    SPG_TRY(cudaMemsetAsync(rsum, 0, sizeof(double), st));
    SPG_TRY(zero_env(Rcur));
    count_launches("k_set_unit_env", st);
    k_set_unit_env<T><<<1, 32, 0, st>>>(Rcur);
    for (int j = cols - 1; j >= 1; --j) {
      SPG_TRY(local(j, Lc + (size_t)j * env, Rcur));
      const int* dP = dims(row, j);
      const int DU = dP[0], chiA = dP[1], chiAr = dP[2];
      const int n = DU * chiA * chiAr;
      count_launches("k_site_vectors", st);
      k_site_vectors<T><<<nblk(n), 256, 0, st>>>(C, DU, chiA, chiAr, 1, 1, Vv, nullptr);
      cgs_rows(Vv, chiA, DU * chiAr, st);
      count_launches("k_site_vectors", st);
      k_site_vectors<T><<<nblk(n), 256, 0, st>>>(nullptr, DU, chiA, chiAr, 1, 0, Vv, site_ptr(row, j));
      SPG_TRY(env_right(j, Rcur, Rtmp, rsum));
      SPG_TRY(cudaMemcpyAsync(Rcur, Rtmp, sizeof(T) * env, cudaMemcpyDeviceToDevice, st));
    }
    SPG_TRY(local(0, Lc, Rcur));
    const int* dP = dims(row, 0);
    count_launches("k_finish_centre", st);
    k_finish_centre<T><<<1, 256, 0, st>>>(C, dP[0] * dP[1] * dP[2], site_ptr(row, 0), mps.lognorm + row + 1, rsum,
                                          mps.lognorm + row);
  }
#undef SPG_TRY
  return cudaGetLastError();
}

template size_t sweep_work_elems<double>(int, int);
template size_t sweep_work_elems<float>(int, int);
template cudaError_t variational_sweeps<double>(const DevTables&, DevWeights<double>, DevMPS<double>, int, int,
                                                const int*, const int*, int, double*, double*, cudaStream_t);
template cudaError_t variational_sweeps<float>(const DevTables&, DevWeights<float>, DevMPS<float>, int, int,
                                               const int*, const int*, int, float*, double*, cudaStream_t);

}  // namespace spg
