// Boundary-MPS kernels: Boltzmann pieces of the PEPS (S2), the left-canonical
// QR sweep, the MPO-MPS zipper matrix and its truncated SVD (S3).
//
// Paper: Sec. 2 and Fig. 1(c)-(d) (PEPS of the Boltzmann distribution,
// approximate contraction with boundary MPSs), Sec. 3.1 (MpsParameters
// bond_dim; MpsContractor(SVDTruncate, ...)).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <optional>
#include <type_traits>

#include "spg_internal.h"

namespace spg {

namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one value; `red` holds >= 32 T.  All threads get the sum.
template <typename T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = lane < nw ? red[lane] : T(0);
  t = warp_sum(t);
  return t;
}

template <typename T>
__device__ __forceinline__ T dexp(double x) {
  return (T)exp(x);
}

// ---------------------------------------------------------------- weights (S2)
// One block per site: w = exp(-beta u (E - min E)); bL, bU, bA from RL, RU,
// RA alike, each over its valid entries (zero elsewhere).
template <typename T>
__global__ void k_weights(DevTables tb, DevWeights<T> wt, double beta_u, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  const int s = blockIdx.x;
  const int d = tb.d[s];
  const int* dm = tb.dims + s * DIMW;
  const int DL = dm[D_DL], NL = dm[D_NL], DU = dm[D_DU], NU = dm[D_NU], NRl = dm[D_NRL];
  const int64_t* RL = tb.RL + (size_t)s * tb.lstride;
  __shared__ long long mn[4];
  __shared__ long long red[32];
  // minima: one pass per table, warp 0 folds the block's partial minima
  for (int t = 0; t < 4; ++t) {
    long long m = LLONG_MAX;
    if (t == 0)
      for (int x = threadIdx.x; x < d; x += blockDim.x) m = min(m, (long long)tb.E[(size_t)s * tb.dmax + x]);
    else if (t == 1)
      for (int e = threadIdx.x; e < DL * NL; e += blockDim.x) m = min(m, (long long)RL[(e / NL) * MAXP + e % NL]);
    else if (t == 2)
      for (int e = threadIdx.x; e < DU * NU; e += blockDim.x)
        m = min(m, (long long)tb.RU[(size_t)s * 256 + (e / NU) * 16 + e % NU]);
    else
      for (int e = threadIdx.x; e < NRl * DU; e += blockDim.x)
        m = min(m, (long long)tb.RA[(size_t)s * 256 + (e / DU) * 16 + e % DU]);
    for (int o = 16; o > 0; o >>= 1) m = min(m, (long long)__shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long r = LLONG_MAX;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = min(r, red[w]);
      mn[t] = r;
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < tb.dmax; x += blockDim.x) {
    T v = T(0);
    if (x < d) v = dexp<T>(-beta_u * (double)(tb.E[(size_t)s * tb.dmax + x] - mn[0]));
    wt.w[(size_t)s * tb.dmax + x] = v;
  }
  for (int e = threadIdx.x; e < tb.lstride; e += blockDim.x) {
    const int l = e / MAXP, h = e % MAXP;
    T v = T(0);
    if (l < DL && h < NL) v = dexp<T>(-beta_u * (double)(RL[e] - mn[1]));
    wt.bL[(size_t)s * tb.lstride + e] = v;
  }
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int i = e >> 4, j = e & 15;
    T vu = T(0), va = T(0);
    if (i < DU && j < NU) vu = dexp<T>(-beta_u * (double)(tb.RU[(size_t)s * 256 + e] - mn[2]));
    if (i < NRl && j < DU) va = dexp<T>(-beta_u * (double)(tb.RA[(size_t)s * 256 + e] - mn[3]));
    wt.bU[(size_t)s * 256 + e] = vu;
    wt.bA[(size_t)s * 256 + e] = va;
  }
}

// ---------------------------------------------------------------- CGS2 QR
__device__ __forceinline__ int wid_of() { return (int)(threadIdx.x >> 5); }

constexpr int QR_PB = 16;  // vectors per panel of the block variant

template <typename T>
__host__ __device__ constexpr T qr_tol() {
  return sizeof(T) == 8 ? T(1e-13) : T(1e-5);
}

// One CGS2 step on vector k of nvec contiguous vectors of length len (stride
// ld), in place: two projection passes against the (orthonormal) vectors
// clo .. k-1, then normalisation.  The squared norm is accumulated in the
// second update and the norm before any projection follows from Pythagoras
// (||x||^2 = sum r^2 + ||x'||^2, the sum also over the coefficients inter[c *
// istride] of vectors c < clo that a block step removed earlier), so a vector
// costs five barriers.  A vector whose remainder falls below rel_tol of its
// norm is numerically dependent: zeroed, R_kk = 0.  Column k of R (nvec x
// nvec, row-major; x_k = sum_{c <= k} R[c][k] q_c) is written when Rout is set.
// Scratch: red >= 64 + 2 * SMAX T.
//
// Options of the block variant: inter == nullptr means no earlier
// coefficients; Rp (stride QR_PB) receives the panel's own column k - clo
// (rows clo .. k); dep_abs > 0 replaces the relative rule by nk <= dep_abs
// (unit input vectors); red[42] keeps the smallest nk / n0 of the vectors
// kept (the cancellation of the panel, reset by the caller).
template <typename T>
__device__ void cgs2_vec(T* V, int k, int clo, int nvec, int len, int ld, T* Rout, T* red, const T* inter,
                         int istride, T* Rp = nullptr, T dep_abs = T(0)) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  T* rc = red + 64;          // coefficients of the current pass [SMAX]
  T* racc = rc + SMAX;       // accumulated coefficients [SMAX]
  const T rel_tol = qr_tol<T>();
  T* xk = V + (size_t)k * ld;
  T part = T(0);
  for (int pass = 0; pass < 2; ++pass) {
    // dots <q_c, x_k>: warp w takes c = clo + w, clo + w + nw, ... up to four
    // at a time (independent accumulators, x_k loaded once per element)
    for (int c0 = clo + wid; c0 < k; c0 += 4 * nw) {
      const int c1 = c0 + nw, c2 = c0 + 2 * nw, c3 = c0 + 3 * nw;
      const T* x0 = V + (size_t)c0 * ld;
      const T* x1 = V + (size_t)(c1 < k ? c1 : c0) * ld;
      const T* x2 = V + (size_t)(c2 < k ? c2 : c0) * ld;
      const T* x3 = V + (size_t)(c3 < k ? c3 : c0) * ld;
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      for (int i = lane; i < len; i += 32) {
        const T v = xk[i];
        a0 += x0[i] * v;
        a1 += x1[i] * v;
        a2 += x2[i] * v;
        a3 += x3[i] * v;
      }
      a0 = warp_sum(a0);
      a1 = warp_sum(a1);
      a2 = warp_sum(a2);
      a3 = warp_sum(a3);
      if (lane == 0) {
        rc[c0] = a0;
        racc[c0] = pass == 0 ? a0 : racc[c0] + a0;
        if (c1 < k) {
          rc[c1] = a1;
          racc[c1] = pass == 0 ? a1 : racc[c1] + a1;
        }
        if (c2 < k) {
          rc[c2] = a2;
          racc[c2] = pass == 0 ? a2 : racc[c2] + a2;
        }
        if (c3 < k) {
          rc[c3] = a3;
          racc[c3] = pass == 0 ? a3 : racc[c3] + a3;
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < len; i += nt) {
      T v0 = xk[i], v1 = T(0), v2 = T(0), v3 = T(0);
      const T* vp = V + (size_t)clo * ld + i;
      int c = clo;
      for (; c + 3 < k; c += 4) {
        v0 -= rc[c] * vp[0];
        v1 -= rc[c + 1] * vp[ld];
        v2 -= rc[c + 2] * vp[2 * ld];
        v3 -= rc[c + 3] * vp[3 * ld];
        vp += 4 * ld;
      }
      for (; c < k; ++c, vp += ld) v0 -= rc[c] * vp[0];
      const T v = (v0 + v1) + (v2 + v3);
      xk[i] = v;
      if (pass == 1) part += v * v;
    }
    if (k == clo && pass == 0) {  // nothing to project against
      for (int i = tid; i < len; i += nt) part += xk[i] * xk[i];
      break;
    }
    if (pass == 0) __syncthreads();
  }
  part = warp_sum(part);
  if (lane == 0) red[wid] = part;
  __syncthreads();
  // one warp combines the partial norms with the projection coefficients
  // (Pythagoras) and publishes the scale and the diagonal entry
  if (wid == 0) {
    T nk2 = lane < nw ? red[lane] : T(0);
    nk2 = warp_sum(nk2);
    T r2 = T(0);
    for (int c = clo + lane; c < k; c += 32) r2 += racc[c] * racc[c];
    if (inter)
      for (int c = lane; c < clo; c += 32) r2 += inter[(size_t)c * istride] * inter[(size_t)c * istride];
    r2 = warp_sum(r2);
    if (lane == 0) {
      const T nk = sqrt(nk2);
      const T n0 = sqrt(nk2 + r2);
      const bool dep = dep_abs > T(0) ? !(nk > dep_abs) : (!(nk > rel_tol * n0) || n0 == T(0));
      red[40] = dep ? T(0) : T(1) / nk;
      red[41] = dep ? T(0) : nk;
      if (!dep) red[42] = min(red[42], nk / n0);
    }
  }
  __syncthreads();
  const T inv = red[40];
  for (int i = tid; i < len; i += nt) xk[i] *= inv;
  if (Rout)
    for (int c = tid; c < nvec; c += nt)
      Rout[(size_t)c * nvec + k] =
          c < clo ? (inter ? inter[(size_t)c * istride] : T(0)) : (c < k ? racc[c] : (c == k ? red[41] : T(0)));
  if (Rp)
    for (int c = clo + tid; c <= k; c += nt) Rp[(c - clo) * QR_PB + (k - clo)] = c < k ? racc[c] : red[41];
  __syncthreads();
}

// CGS2 on nvec contiguous vectors of length len (stride ld) in place, one
// vector at a time (cgs2_vec against all earlier vectors).
template <typename T>
__device__ void cgs2_core(T* V, int nvec, int len, int ld, T* Rout, T* red) {
  for (int k = 0; k < nvec; ++k) cgs2_vec(V, k, 0, nvec, len, ld, Rout, red, (const T*)nullptr, 0);
}

// Block Gram-Schmidt: panels of QR_PB vectors.  A panel is first projected
// twice against all earlier panels at once (bgs_project), then
// orthonormalised vector by vector inside the panel (cgs2_vec), which only
// projects against the panel's earlier vectors.  The same two-pass
// projections as cgs2_core, grouped so that most of the multiply-adds run as
// register-tiled panel products instead of one dot per (vector, earlier
// vector) pair.  A panel whose vectors lost most of their length to the
// projections (numerically near the span of the earlier vectors) is, where
// the caller needs an orthonormal result, projected once more after its
// normalisation and re-orthonormalised (panel_second_pass): normalising a
// remainder at the rounding level of the projections would otherwise carry
// that rounding, amplified, into its direction.

// Tile of the panel Gram step: TC earlier vectors x 4 panel vectors (FP64
// keeps 2 x 4 to stay inside the register budget of a 1024-thread CTA).
template <typename T>
struct BgsTile {
  static constexpr int TC = sizeof(T) == 8 ? 2 : 4;
  static constexpr int NV = TC * 4;
};

// One projection pass of panel k0 .. k0+b-1 against vectors 0 .. k0-1:
// C[c][j] = <q_c, x_{k0+j}> (one warp per tile of (c, j), entries strided
// over the lanes, the tile's partial sums reduced by a transposed butterfly:
// every shuffle halves the values a lane holds), Racc[c][j] (+)= C[c][j],
// then x_{k0+j} -= sum_c C[c][j] q_c (one thread per entry, the panel's
// vectors in registers).  Cs, Racc: [SMAX][QR_PB].
template <typename T>
__device__ void bgs_project(T* V, int k0, int b, int len, int ld, T* Cs, T* Racc, bool first) {
  constexpr int TC = BgsTile<T>::TC, NV = BgsTile<T>::NV;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int tc = (k0 + TC - 1) / TC, tj = (b + 3) >> 2;
  for (int t = wid; t < tc * tj; t += nw) {
    const int c0 = (t / tj) * TC, j0 = (t % tj) * 4;
    int qo[TC], xo[4];
#pragma unroll
    for (int u = 0; u < TC; ++u) qo[u] = min(c0 + u, k0 - 1) * ld;
#pragma unroll
    for (int w = 0; w < 4; ++w) xo[w] = (k0 + min(j0 + w, b - 1)) * ld;
    T a[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) a[v] = T(0);
    for (int i = lane; i < len; i += 32) {
      T qv[TC], xv[4];
#pragma unroll
      for (int u = 0; u < TC; ++u) qv[u] = V[qo[u] + i];
#pragma unroll
      for (int w = 0; w < 4; ++w) xv[w] = V[xo[w] + i];
#pragma unroll
      for (int u = 0; u < TC; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) a[u * 4 + w] += qv[u] * xv[w];
    }
    // transposed butterfly: at lane bit B the lane with the bit clear keeps
    // the lower half of its values and receives the partner's lower half; the
    // one with the bit set keeps and receives the upper half
    constexpr int stages = NV == 16 ? 4 : 3;
    int o = 0;
#pragma unroll
    for (int stg = 0; stg < stages; ++stg) {
      const int h = NV >> (stg + 1), bit = 16 >> stg;
      const bool up = (lane & bit) != 0;
#pragma unroll
      for (int v = 0; v < h; ++v) {
        const T send = up ? a[v] : a[v + h];
        const T keep = up ? a[v + h] : a[v];
        a[v] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
      }
      if (up) o += h;
    }
    // lanes that differ only in the bits below the last stage hold the same
    // output: sum them
    constexpr int rest = 32 / NV;  // 2 (NV 16) or 4 (NV 8)
#pragma unroll
    for (int m = rest / 2; m >= 1; m >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], m);
    const int c = c0 + o / 4, j = j0 + (o & 3);
    if ((lane & (rest - 1)) == 0 && c < k0 && j < b) {
      Cs[c * QR_PB + j] = a[0];
      Racc[c * QR_PB + j] = first ? a[0] : Racc[c * QR_PB + j] + a[0];
    }
  }
  __syncthreads();
  for (int i = tid; i < len; i += nt) {
    T acc[QR_PB];
#pragma unroll
    for (int j = 0; j < QR_PB; ++j) acc[j] = j < b ? V[(k0 + j) * ld + i] : T(0);
    for (int c = 0; c < k0; ++c) {
      const T qv = V[c * ld + i];
      const T* cr = Cs + c * QR_PB;
#pragma unroll
      for (int j = 0; j < QR_PB; ++j) acc[j] -= cr[j] * qv;
    }
#pragma unroll
    for (int j = 0; j < QR_PB; ++j)
      if (j < b) V[(k0 + j) * ld + i] = acc[j];
  }
  __syncthreads();
}

// Gram of the panel k0 .. k0+b-1: G[i][j] = <x_{k0+i}, x_{k0+j}> (i, j < b),
// one warp per 4 x 4 tile, entries strided over the lanes, the tile's 16
// partial sums reduced by the transposed butterfly of bgs_project.
template <typename T>
__device__ void panel_gram(const T* V, int k0, int b, int len, int ld, T* G) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int tb = (b + 3) >> 2;
  for (int t = wid; t < tb * tb; t += nw) {
    const int i0 = (t / tb) * 4, j0 = (t % tb) * 4;
    int io[4], jo[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      io[u] = (k0 + min(i0 + u, b - 1)) * ld;
      jo[u] = (k0 + min(j0 + u, b - 1)) * ld;
    }
    T a[16];
#pragma unroll
    for (int v = 0; v < 16; ++v) a[v] = T(0);
    for (int i = lane; i < len; i += 32) {
      T xi[4], xj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xi[u] = V[io[u] + i];
        xj[u] = V[jo[u] + i];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) a[u * 4 + w] += xi[u] * xj[w];
    }
    int o = 0;
#pragma unroll
    for (int stg = 0; stg < 4; ++stg) {
      const int h = 16 >> (stg + 1), bit = 16 >> stg;
      const bool up = (lane & bit) != 0;
#pragma unroll
      for (int v = 0; v < h; ++v) {
        const T send = up ? a[v] : a[v + h];
        const T keep = up ? a[v + h] : a[v];
        a[v] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
      }
      if (up) o += h;
    }
    a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
    const int i = i0 + o / 4, j = j0 + (o & 3);
    if ((lane & 1) == 0 && i < b && j < b) G[i * QR_PB + j] = a[0];
  }
  __syncthreads();
}

// Cholesky of the panel's Gram, G = L L^T, by warp 0 (lane r owns row r).  A
// pivot is dependent (zero column of L, zero vector in Q) when it falls below
// tol_c^2 of its diagonal entry (the Gram's rounding floor) or below
// tol_d^2 * ref2[k] (the dependency rule of cgs2_vec against the column's
// norm before any projection; ref2 == nullptr: not used).  inv[k] = 1 / L_kk
// or 0.
template <typename T>
__device__ void panel_cholesky(const T* G, int b, const T* ref2, T tol_c, T tol_d, T* L, T* inv) {
  if ((threadIdx.x >> 5) == 0) {
    const int r = threadIdx.x & 31;
    for (int e = r; e < QR_PB * QR_PB; e += 32) L[e] = T(0);
    __syncwarp();
    for (int k = 0; k < b; ++k) {
      if (r == k) {
        T d = G[k * QR_PB + k];
        for (int c = 0; c < k; ++c) d -= L[k * QR_PB + c] * L[k * QR_PB + c];
        T thr = tol_c * tol_c * G[k * QR_PB + k];
        if (ref2) thr = max(thr, tol_d * tol_d * ref2[k]);
        const bool dep = !(d > thr) || !(G[k * QR_PB + k] > T(0));
        const T lkk = dep ? T(0) : sqrt(d);
        L[k * QR_PB + k] = lkk;
        inv[k] = dep ? T(0) : T(1) / lkk;
      }
      __syncwarp();
      const T ik = inv[k];
      if (r > k && r < b) {
        T v = G[r * QR_PB + k];
        for (int c = 0; c < k; ++c) v -= L[r * QR_PB + c] * L[k * QR_PB + c];
        L[r * QR_PB + k] = v * ik;
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// x_k <- (x_k - sum_{c < k} L[k][c] q_c) * inv[k] for the panel's vectors,
// one thread per entry with the panel in registers.
template <typename T>
__device__ void panel_solve(T* V, int k0, int b, int len, int ld, const T* L, const T* inv) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    T q[QR_PB];
#pragma unroll
    for (int k = 0; k < QR_PB; ++k) {
      if (k < b) {
        T v = V[(k0 + k) * ld + i];
#pragma unroll
        for (int c = 0; c < k; ++c) v -= L[k * QR_PB + c] * q[c];
        q[k] = v * inv[k];
        V[(k0 + k) * ld + i] = q[k];
      } else {
        q[k] = T(0);
      }
    }
  }
  __syncthreads();
}

// Panel scratch of the Cholesky-QR path: G, L1, L2 (QR_PB^2 each), inv,
// ref2 (QR_PB each), one flag word.
template <typename T>
__host__ __device__ constexpr int chol_scratch_elems() { return 3 * QR_PB * QR_PB + 2 * QR_PB + 4; }

// Orthonormalises panel k0 .. k0+b-1 (already projected against the earlier
// panels; Racc holds those coefficients) by Cholesky-QR twice: P = Q1 L1^T,
// Q1 = Q2 L2^T, so R_panel = L2^T L1^T.  The result is accepted when the Gram
// of Q1 is within 0.1 of the identity, that of Q2 within 1e-5 (over the
// columns that are not dependent) and the second pass finds no column
// dependent that the first kept; otherwise the panel is restored from Pc and
// orthonormalised vector by vector (cgs2_vec).  Writes the panel's columns
// of R either way.
template <typename T>
__device__ void panel_cholqr(T* V, int k0, int b, int nvec, int len, int ld, T* Rout, T* red, T* Racc, T* Pc,
                             T* cs) {
  T* G = cs;
  T* L1 = G + QR_PB * QR_PB;
  T* L2 = L1 + QR_PB * QR_PB;
  T* inv = L2 + QR_PB * QR_PB;
  T* ref2 = inv + QR_PB;
  int* flag = reinterpret_cast<int*>(ref2 + QR_PB);
  const int tid = threadIdx.x, nt = blockDim.x;
  const T tol_c = T(3e-4), tol_d = qr_tol<T>();
  for (int e = tid; e < b * len; e += nt) Pc[e] = V[(k0 + e / len) * ld + e % len];
  panel_gram(V, k0, b, len, ld, G);
  // squared norm of every column before the projections (Pythagoras)
  for (int j = tid; j < b; j += nt) {
    T r2 = G[j * QR_PB + j];
    for (int c = 0; c < k0; ++c) r2 += Racc[c * QR_PB + j] * Racc[c * QR_PB + j];
    ref2[j] = r2;
  }
  if (tid == 0) *flag = 1;
  __syncthreads();
  panel_cholesky(G, b, ref2, tol_c, tol_d, L1, inv);
  if (tid == 0) {  // the panel's cancellation: first pivots against the columns' norms
    T m = red[42];
    for (int k = 0; k < b; ++k)
      if (L1[k * QR_PB + k] != T(0) && ref2[k] > T(0)) m = min(m, L1[k * QR_PB + k] / sqrt(ref2[k]));
    red[42] = m;
  }
  panel_solve(V, k0, b, len, ld, L1, inv);
  panel_gram(V, k0, b, len, ld, G);
  for (int e = tid; e < b * b; e += nt) {
    const int i = e / b, j = e % b;
    if (L1[i * QR_PB + i] != T(0) && L1[j * QR_PB + j] != T(0) &&
        !(fabs(G[i * QR_PB + j] - (i == j ? T(1) : T(0))) <= T(0.1)))
      *flag = 0;
  }
  __syncthreads();
  if (*flag) {
    panel_cholesky(G, b, (const T*)nullptr, tol_c, tol_d, L2, inv);
    panel_solve(V, k0, b, len, ld, L2, inv);
    panel_gram(V, k0, b, len, ld, G);
    for (int e = tid; e < b * b; e += nt) {
      const int i = e / b, j = e % b;
      if (L2[i * QR_PB + i] != T(0) && L2[j * QR_PB + j] != T(0) &&
          !(fabs(G[i * QR_PB + j] - (i == j ? T(1) : T(0))) <= T(1e-5)))
        *flag = 0;
      // a column the first pass kept but the second found dependent: Q1 was
      // too ill-conditioned for the Gram to resolve it, and that direction
      // would be lost (the columns compared above exclude it)
      if (i == j && L1[i * QR_PB + i] != T(0) && L2[i * QR_PB + i] == T(0)) *flag = 0;
    }
    __syncthreads();
  }
  if (*flag) {
    // R column k0 + j: the earlier panels' coefficients, then (L2^T L1^T)[c][j]
    if (Rout)
      for (int e = tid; e < nvec * b; e += nt) {
        const int c = e / b, j = e % b;
        T v = T(0);
        if (c < k0) {
          v = Racc[c * QR_PB + j];
        } else if (c < k0 + b) {
          const int ci = c - k0;
          // (L2^T L1^T)[ci][j] = sum_m L2[m][ci] L1[j][m], m from ci to j
          for (int m = ci; m <= j; ++m) v += L2[m * QR_PB + ci] * L1[j * QR_PB + m];
        }
        Rout[(size_t)c * nvec + k0 + j] = v;
      }
    __syncthreads();
    return;
  }
  for (int e = tid; e < b * len; e += nt) V[(k0 + e / len) * ld + e % len] = Pc[e];
  __syncthreads();
  for (int j = 0; j < b; ++j) cgs2_vec(V, k0 + j, k0, nvec, len, ld, Rout, red, Racc + j, QR_PB);
}

// Scratch: red (64 + 2 SMAX), Cs and Racc (SMAX * QR_PB each).  Offsets into
// V are int: nvec * ld stays below 2^31 for every caller (staged blocks and
// zipper blocks of at most SMAX vectors).  With Pc (QR_PB * len) and cs
// (chol_scratch_elems) given, FP32 panels go through panel_cholqr.
// The second pass of panel k0 .. k0+b-1 (orthonormal, R's columns of the
// panel written: S1 above the panel, R1 on it): S2 = Q_prev^T Q1 and Q1 -=
// Q_prev S2 (one projection; Cs = S2), then CGS2 inside the panel of these
// nearly unit vectors (R2; a vector keeping at most a tenth of its length
// was within the span of the earlier vectors and is zeroed).  X = Q_prev S1
// + Q1 R1 and Q1 = Q_prev S2 + Q2 R2 give R's panel columns [S1 + S2 R1;
// R2 R1] (Racc holds them on the way; R2 in cs).
template <typename T>
__device__ void panel_second_pass(T* V, int k0, int b, int nvec, int len, int ld, T* Rout, T* red, T* Cs, T* Racc,
                                  T* R2) {
  const int tid = threadIdx.x, nt = blockDim.x;
  bgs_project(V, k0, b, len, ld, Cs, Racc, true);
  for (int j = 0; j < b; ++j)
    cgs2_vec(V, k0 + j, k0, nvec, len, ld, (T*)nullptr, red, (const T*)nullptr, 0, R2, T(0.1));
  if (!Rout) return;
  // new columns into Racc ([(k0 + b) rows][QR_PB]), then back into Rout
  for (int e = tid; e < (k0 + b) * b; e += nt) {
    const int c = e / b, j = e % b;
    T v;
    if (c < k0) {
      v = Rout[(size_t)c * nvec + k0 + j];
      for (int i = 0; i <= j; ++i) v += Cs[c * QR_PB + i] * Rout[(size_t)(k0 + i) * nvec + k0 + j];
    } else {
      const int i = c - k0;
      v = T(0);
      for (int m = i; m <= j; ++m) v += R2[i * QR_PB + m] * Rout[(size_t)(k0 + m) * nvec + k0 + j];
    }
    Racc[c * QR_PB + j] = v;
  }
  __syncthreads();
  for (int e = tid; e < (k0 + b) * b; e += nt) {
    const int c = e / b, j = e % b;
    Rout[(size_t)c * nvec + k0 + j] = Racc[c * QR_PB + j];
  }
  __syncthreads();
}

// reorth_eta > 0: panels (after the first) whose smallest kept nk / n0 falls
// below it take panel_second_pass, with r2 (QR_PB^2 T) as scratch.
template <typename T>
__device__ void bcgs2_core(T* V, int nvec, int len, int ld, T* Rout, T* red, T* Cs, T* Racc, T* Pc = nullptr,
                           T* cs = nullptr, T reorth_eta = T(0), T* r2 = nullptr) {
  for (int k0 = 0; k0 < nvec; k0 += QR_PB) {
    const int b = min(QR_PB, nvec - k0);
    if (k0 > 0) {
      bgs_project(V, k0, b, len, ld, Cs, Racc, true);
      bgs_project(V, k0, b, len, ld, Cs, Racc, false);
    }
    if (threadIdx.x == 0) red[42] = T(1);
    __syncthreads();
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (Pc && cs) {
        panel_cholqr(V, k0, b, nvec, len, ld, Rout, red, Racc, Pc, cs);
        done = true;
      }
    }
    if (!done)
      for (int j = 0; j < b; ++j) cgs2_vec(V, k0 + j, k0, nvec, len, ld, Rout, red, Racc + j, QR_PB);
    __syncthreads();
    if (k0 > 0 && reorth_eta > T(0) && r2 && red[42] < reorth_eta)
      panel_second_pass(V, k0, b, nvec, len, ld, Rout, red, Cs, Racc, r2);
  }
}

// CGS2 on the ROWS of X (nvec vectors of length len, row stride ld), each
// vector contiguous so every access is coalesced; the vectors are staged in
// shared memory when they fit.  R (nvec x nvec, row-major) as in cgs2_core:
// x_k = sum_{c <= k} R[c][k] q_c.
// Cancellation below which a panel takes the second pass: its direction
// errors stay near eps / eta (2e-14 in FP64, 6e-5 in FP32).
template <typename T>
__host__ __device__ constexpr T reorth_eta() {
  return sizeof(T) == 8 ? T(1e-2) : T(1e-3);
}

template <typename T>
__global__ void __launch_bounds__(512, 1) k_cgs2_rows(T* X, int nvec, int len, int ld, T* Rout, int use_smem,
                                                      int use_chol, int reorth, size_t zs) {
  X = zp(X, zs);
  Rout = zp(Rout, zs);
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);  // 64 + 2 SMAX
  T* Cs = red + 64 + 2 * SMAX;              // SMAX * QR_PB
  T* Racc = Cs + SMAX * QR_PB;              // SMAX * QR_PB
  T* cs = Racc + SMAX * QR_PB;              // chol_scratch_elems
  T* V = use_smem ? cs + chol_scratch_elems<T>() : X;
  T* Pc = use_chol ? V + (size_t)nvec * len : nullptr;  // QR_PB * len (use_smem only)
  const int vld = use_smem ? len : ld;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (use_smem)
    for (int e = tid; e < nvec * len; e += nt) V[e] = X[(size_t)(e / len) * ld + e % len];
  __syncthreads();
  bcgs2_core(V, nvec, len, vld, Rout, red, Cs, Racc, Pc, use_chol ? cs : (T*)nullptr,
             reorth ? reorth_eta<T>() : T(0), cs);
  if (use_smem)
    for (int e = tid; e < nvec * len; e += nt) X[(size_t)(e / len) * ld + e % len] = V[e];
}

// ---------------------------------------------------------------- tall QR (TSQR)
// QR of nvec long vectors (rows of X, length len, row stride len) across
// many CTAs: the entries are cut into nb blocks of bl (the last one
// shorter); (1) k_tsqr_leaf: CGS2 of every block in its own CTA, its R_b
// written as the block's slice of the stacked factor S (nvec vectors of
// length nb * nvec, S[k][b * nvec + c] = R_b[c][k]); (2) QR of S, whose R is
// the R of X; (3) k_tsqr_apply: every block's Q_b times its slice of S's Q,
// x_k[block b] = sum_c S[k][b * nvec + c] q_c[block b].  A block with fewer
// entries than vectors leaves the dependent ones zero, with zero rows in
// R_b, which the stacked QR carries through.
template <typename T>
__global__ void __launch_bounds__(512) k_tsqr_leaf(T* X, int nvec, int len, int bl, T* S, int use_smem, size_t zs) {
  X = zp(X, zs);
  S = zp(S, zs);
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);  // 64 + 2 SMAX
  T* R = red + 64 + 2 * SMAX;               // nvec * nvec
  T* Vs = R + (size_t)nvec * nvec;          // nvec * bl (use_smem)
  const int b = blockIdx.x, nb = gridDim.x;
  const int i0 = b * bl, w = min(bl, len - i0);
  const int tid = threadIdx.x, nt = blockDim.x;
  T* V = use_smem ? Vs : X + i0;
  const int ld = use_smem ? w : len;
  if (use_smem)
    for (int e = tid; e < nvec * w; e += nt) Vs[e] = X[(size_t)(e / w) * len + i0 + e % w];
  __syncthreads();
  cgs2_core(V, nvec, w, ld, R, red);
  if (use_smem)
    for (int e = tid; e < nvec * w; e += nt) X[(size_t)(e / w) * len + i0 + e % w] = Vs[e];
  const size_t sl = (size_t)nb * nvec;
  for (int e = tid; e < nvec * nvec; e += nt) {
    const int c = e / nvec, k = e % nvec;
    S[(size_t)k * sl + (size_t)b * nvec + c] = R[e];
  }
}

// Step (3), 64 entries of the block at a time through shared memory (the
// outputs of a chunk depend only on that chunk's entries, so X is updated in
// place).
template <typename T>
__global__ void k_tsqr_apply(T* X, int nvec, int len, int bl, const T* __restrict__ S, size_t zs) {
  X = zp(X, zs);
  S = zp(S, zs);
  constexpr int CH = 64;
  extern __shared__ unsigned char smem_raw[];
  T* Sb = reinterpret_cast<T*>(smem_raw);  // [k][c] nvec * nvec
  T* Qs = Sb + (size_t)nvec * nvec;        // [c][i] nvec * CH
  const int b = blockIdx.x, nb = gridDim.x;
  const int i0 = b * bl, w = min(bl, len - i0);
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t sl = (size_t)nb * nvec;
  for (int e = tid; e < nvec * nvec; e += nt) Sb[e] = S[(size_t)(e / nvec) * sl + (size_t)b * nvec + e % nvec];
  for (int c0 = 0; c0 < w; c0 += CH) {
    const int cw = min(CH, w - c0);
    __syncthreads();
    for (int e = tid; e < nvec * cw; e += nt) Qs[(e / cw) * CH + e % cw] = X[(size_t)(e / cw) * len + i0 + c0 + e % cw];
    __syncthreads();
    for (int e = tid; e < nvec * cw; e += nt) {
      const int k = e / cw, i = e % cw;
      const T* sk = Sb + (size_t)k * nvec;
      T a0 = T(0), a1 = T(0);
      int c = 0;
      for (; c + 1 < nvec; c += 2) {
        a0 += sk[c] * Qs[c * CH + i];
        a1 += sk[c + 1] * Qs[(c + 1) * CH + i];
      }
      if (c < nvec) a0 += sk[c] * Qs[c * CH + i];
      X[(size_t)k * len + i0 + c0 + i] = a0 + a1;
    }
  }
}

// ---------------------------------------------------------------- left-canonical sweep
// Sites of row r: [p][chiL][chiR] = matrix (p*chiL) x chiR.  For j < cols-1:
// QR of site j, then site j+1 <- R site j+1.  The last site is normalised.
// The chiR columns of a site are staged as contiguous vectors in `work`
// (shared memory when they fit, else the global scratch) for the CGS2.
// With Panels (FP32, staged in shared memory, 512 threads for the panel
// products' registers) sites of >= 32 columns of >= 256 entries go through
// the block Gram-Schmidt with guarded Cholesky-QR panels of k_cgs2_rows;
// the others through per-vector CGS2.
template <typename T, bool Panels>
__global__ void __launch_bounds__(Panels ? 512 : 1024) k_left_canonical(DevMPS<T> mps, int r, int cols, T* gwork,
                                                                        int use_smem, size_t zs) {
  mps = zp(mps, zs);
  gwork = zp(gwork, zs);
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);  // 64 + 2 SMAX
  T* R = red + 64 + 2 * SMAX;               // MAXCHI * MAXCHI
  T* Cs = R + MAXCHI * MAXCHI;              // Panels: SMAX * QR_PB
  T* Racc = Cs + (Panels ? SMAX * QR_PB : 0);
  T* cs = Racc + (Panels ? SMAX * QR_PB : 0);  // chol_scratch_elems
  T* W = use_smem ? cs + (Panels ? chol_scratch_elems<T>() : 0) : gwork;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t wmax = (size_t)mps.site_stride;  // staged site, then the panel copy
  for (int j = 0; j < cols - 1; ++j) {
    const int* dA = mps.dimA + (r * cols + j) * 3;
    const int p = dA[0], chiL = dA[1], chiR = dA[2];
    const int len = p * chiL;
    T* A = mps.A + (size_t)(r * cols + j) * mps.site_stride;
    for (int e = tid; e < len * chiR; e += nt) W[(size_t)(e % chiR) * len + e / chiR] = A[e];
    __syncthreads();
    if (Panels && chiR >= 32 && len >= 256)
      bcgs2_core(W, chiR, len, len, R, red, Cs, Racc, W + wmax, cs, reorth_eta<T>(), cs);
    else
      cgs2_core(W, chiR, len, len, R, red);
    for (int e = tid; e < len * chiR; e += nt) A[e] = W[(size_t)(e % chiR) * len + e / chiR];
    __syncthreads();
    const int* dB = mps.dimA + (r * cols + j + 1) * 3;
    const int p2 = dB[0], chiL2 = dB[1], chiR2 = dB[2];  // chiL2 == chiR
    T* Bn = mps.A + (size_t)(r * cols + j + 1) * mps.site_stride;
    // new[s][a][b] = sum_{g >= a} R[a][g] old[s][g][b], in place, a ascending
    for (int c = tid; c < p2 * chiR2; c += nt) {
      const int s = c / chiR2, b = c % chiR2;
      T* col = Bn + (size_t)s * chiL2 * chiR2 + b;
      for (int a = 0; a < chiL2; ++a) {
        T v = T(0);
        for (int g = a; g < chiL2; ++g) v += R[a * chiL2 + g] * col[(size_t)g * chiR2];
        col[(size_t)a * chiR2] = v;
      }
    }
    __syncthreads();
  }
  const int* dA = mps.dimA + (r * cols + cols - 1) * 3;
  const int n = dA[0] * dA[1] * dA[2];
  T* A = mps.A + (size_t)(r * cols + cols - 1) * mps.site_stride;
  T part = T(0);
  for (int i = tid; i < n; i += nt) part += A[i] * A[i];
  const T nrm = sqrt(block_sum(part, red));
  const T inv = nrm > T(0) ? T(1) / nrm : T(0);
  for (int i = tid; i < n; i += nt) A[i] *= inv;
  if (tid == 0) mps.lognorm[r] += log((double)nrm);
}

// ---------------------------------------------------------------- zipper matrix
// T1[a][s][rr][k] = sum_a' B[s][a][a'] C[rr][a'][k]
template <typename T>
__global__ void k_zip_T1(const T* __restrict__ B, int chiL, int p, int chiR, const T* __restrict__ C,
                         int DR, int K, T* __restrict__ T1, size_t zs) {
  B = zp(B, zs);
  C = zp(C, zs);
  T1 = zp(T1, zs);
  const size_t total = (size_t)chiL * p * DR * K;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int k = e % K;
    size_t t = e / K;
    const int rr = t % DR;
    t /= DR;
    const int s = t % p;
    const int a = (int)(t / p);
    const T* b = B + ((size_t)s * chiL + a) * chiR;
    const T* c = C + (size_t)rr * chiR * K + k;
    T acc = T(0);
    for (int q = 0; q < chiR; ++q) acc += b[q] * c[(size_t)q * K];
    T1[e] = acc;
  }
}

// M[(l*chiL + a)][(u*K + k)] = bA[l / Gin][u] sum_h bL[l][h] Y_u[h],
//   Y_u[h] = sum_{x: PL x = h} bU[u][PU x] w(x) T1[a][PD x][PR x * Gout + gD_up[u]][k]
// (gD_up: the upper site's PD -> PG map; 0 in row 0).  One block per
// (a, chunk of k); dynamic shared memory holds the k-slice of T1 [p][DR] and
// the site's bL [DL][NL].
template <typename T>
__global__ void k_zip_M(DevTables tb, DevWeights<T> wt, int site, const T* __restrict__ T1, int chiL,
                        int p, int DR, int K, int DL, int DU, int kchunk, T* __restrict__ M, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  T1 = zp(T1, zs);
  M = zp(M, zs);
  extern __shared__ unsigned char smem_raw[];
  T* sT = reinterpret_cast<T*>(smem_raw);  // [p][DR]
  T* sbL = sT + (size_t)p * DR;            // [DL][NL]
  __shared__ T sw[MAXS];
  __shared__ uint8_t sPU[MAXS], sPD[MAXS], sPR[MAXS];
  __shared__ int16_t sx[MAXS];
  __shared__ int soff[MAXP + 1];
  __shared__ T sbU[256], sbA[256];
  __shared__ T sY[MAXP * MAXP];
  __shared__ int sg[MAXP];
  const int a = blockIdx.x;
  const int k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  const int d = tb.d[site];
  const int* dm = tb.dims + site * DIMW;
  const int NL = dm[D_NL], Gin = dm[D_GIN], Gout = dm[D_GOUT];
  const int cols = tb.cols;
  const int tid = threadIdx.x;
  for (int x = tid; x < d; x += blockDim.x) {
    sw[x] = wt.w[(size_t)site * tb.dmax + x];
    sPU[x] = tb.PU[(size_t)site * tb.dmax + x];
    sPD[x] = tb.PD[(size_t)site * tb.dmax + x];
    sPR[x] = tb.PR[(size_t)site * tb.dmax + x];
    sx[x] = tb.xsL[(size_t)site * tb.dmax + x];
  }
  for (int e = tid; e < 256; e += blockDim.x) {
    sbU[e] = wt.bU[(size_t)site * 256 + e];
    sbA[e] = wt.bA[(size_t)site * 256 + e];
  }
  for (int e = tid; e < DL * NL; e += blockDim.x)
    sbL[e] = wt.bL[(size_t)site * tb.lstride + (e / NL) * MAXP + e % NL];
  for (int e = tid; e <= MAXP; e += blockDim.x) soff[e] = tb.xoffL[site * (MAXP + 1) + e];
  for (int u = tid; u < MAXP; u += blockDim.x) sg[u] = (site >= cols && u < DU) ? tb.gD[(size_t)(site - cols) * MAXP + u] : 0;
  __syncthreads();
  const size_t ldM = (size_t)DU * K;
  for (int k = k0; k < k1; ++k) {
    for (int e = tid; e < p * DR; e += blockDim.x) sT[e] = T1[((size_t)a * p * DR + e) * K + k];
    __syncthreads();
    for (int e = tid; e < DU * NL; e += blockDim.x) {
      const int u = e / NL, h = e % NL;
      const int g = sg[u];
      T acc = T(0);
      for (int q = soff[h]; q < soff[h + 1]; ++q) {
        const int x = sx[q];
        acc += sbU[u * 16 + sPU[x]] * sw[x] * sT[sPD[x] * DR + sPR[x] * Gout + g];
      }
      sY[u * MAXP + h] = acc;
    }
    __syncthreads();
    for (int e = tid; e < DL * DU; e += blockDim.x) {
      const int l = e / DU, u = e % DU;
      T acc = T(0);
      for (int h = 0; h < NL; ++h) acc += sbL[l * NL + h] * sY[u * MAXP + h];
      M[((size_t)l * chiL + a) * ldM + (size_t)u * K + k] = sbA[(l / Gin) * 16 + u] * acc;
    }
    __syncthreads();
  }
}

// The same zipper matrix with one block per bond index a and every k at
// once (the launch shape of a lockstep group, where the GPU is full): the
// block stages T1[a] ([p][DR][K], contiguous) and the site's tables, forms
// every Y_u[h] for all k (k fastest: conflict-free reads of the slab), then
// every M entry of rows (l, a) with k fastest (coalesced writes).  Each
// entry's sums run in the order of k_zip_M, so the results are the same.
template <typename T>
__global__ void __launch_bounds__(256) k_zip_M_rows(DevTables tb, DevWeights<T> wt, int site, const T* __restrict__ T1,
                                                    int chiL, int p, int DR, int K, int DL, int DU,
                                                    T* __restrict__ M, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  T1 = zp(T1, zs);
  M = zp(M, zs);
  extern __shared__ unsigned char smem_raw[];
  T* sT = reinterpret_cast<T*>(smem_raw);  // [p][DR][K]
  T* sY = sT + (size_t)p * DR * K;         // [DU][NL][K]
  T* sbL = sY + (size_t)DU * MAXP * K;     // [DL][NL]
  __shared__ T sw[MAXS];
  __shared__ uint8_t sPU[MAXS], sPD[MAXS], sPR[MAXS];
  __shared__ int16_t sx[MAXS];
  __shared__ int soff[MAXP + 1];
  __shared__ T sbU[256], sbA[256];
  __shared__ int sg[MAXP];
  const int a = blockIdx.x;
  const int d = tb.d[site];
  const int* dm = tb.dims + site * DIMW;
  const int NL = dm[D_NL], Gin = dm[D_GIN], Gout = dm[D_GOUT];
  const int cols = tb.cols;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int x = tid; x < d; x += nt) {
    sw[x] = wt.w[(size_t)site * tb.dmax + x];
    sPU[x] = tb.PU[(size_t)site * tb.dmax + x];
    sPD[x] = tb.PD[(size_t)site * tb.dmax + x];
    sPR[x] = tb.PR[(size_t)site * tb.dmax + x];
    sx[x] = tb.xsL[(size_t)site * tb.dmax + x];
  }
  for (int e = tid; e < 256; e += nt) {
    sbU[e] = wt.bU[(size_t)site * 256 + e];
    sbA[e] = wt.bA[(size_t)site * 256 + e];
  }
  for (int e = tid; e < DL * NL; e += nt) sbL[e] = wt.bL[(size_t)site * tb.lstride + (e / NL) * MAXP + e % NL];
  for (int e = tid; e <= MAXP; e += nt) soff[e] = tb.xoffL[site * (MAXP + 1) + e];
  for (int u = tid; u < MAXP; u += nt) sg[u] = (site >= cols && u < DU) ? tb.gD[(size_t)(site - cols) * MAXP + u] : 0;
  const T* Ta = T1 + (size_t)a * p * DR * K;
  for (int e = tid; e < p * DR * K; e += nt) sT[e] = Ta[e];
  __syncthreads();
  for (int e = tid; e < DU * NL * K; e += nt) {
    const int k = e % K, h = (e / K) % NL, u = e / (K * NL);
    const int g = sg[u];
    T acc = T(0);
    for (int q = soff[h]; q < soff[h + 1]; ++q) {
      const int x = sx[q];
      acc += sbU[u * 16 + sPU[x]] * sw[x] * sT[((size_t)sPD[x] * DR + sPR[x] * Gout + g) * K + k];
    }
    sY[((size_t)u * MAXP + h) * K + k] = acc;
  }
  __syncthreads();
  const size_t ldM = (size_t)DU * K;
  for (int e = tid; e < DL * DU * K; e += nt) {
    const int k = e % K, u = (e / K) % DU, l = e / (K * DU);
    T acc = T(0);
    for (int h = 0; h < NL; ++h) acc += sbL[l * NL + h] * sY[((size_t)u * MAXP + h) * K + k];
    M[((size_t)l * chiL + a) * ldM + (size_t)u * K + k] = sbA[(l / Gin) * 16 + u] * acc;
  }
}

// ---------------------------------------------------------------- GEMM
// C[m x n] = op(A) op(B), row-major; op(A) = A (m x k, lda) or A^T (A stored
// k x m); op(B) = B (k x n, ldb) or B^T (B stored n x k).  32x32 tile,
// MT x MT outputs per thread ((32 / MT)^2 threads); each output is one chain
// of fused multiply-adds over k in order, whatever MT is.
template <typename T, bool TA, bool TB, int MT>
__global__ void __launch_bounds__((32 / MT) * (32 / MT)) k_gemm(int m, int n, int k, const T* __restrict__ A, int lda,
                                                                const T* __restrict__ B, int ldb, T* __restrict__ C,
                                                                int ldc, size_t zs) {
  A = zp(A, zs);
  B = zp(B, zs);
  C = zp(C, zs);
  constexpr int BM = 32, BN = 32, BK = 32, TPR = 32 / MT, NT = TPR * TPR;
  __shared__ T sA[BK][BM + 1];
  __shared__ T sB[BK][BN + 1];
  const int tx = threadIdx.x % TPR, ty = threadIdx.x / TPR;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  T acc[MT][MT] = {};
  for (int kk = 0; kk < k; kk += BK) {
    for (int e = threadIdx.x; e < BK * BM; e += NT) {
      int kq, i;
      if (TA) {  // contiguous along m
        kq = e / BM;
        i = e % BM;
      } else {  // contiguous along k
        i = e / BK;
        kq = e % BK;
      }
      const int gi = row0 + i, gk = kk + kq;
      T v = T(0);
      if (gi < m && gk < k) v = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
      sA[kq][i] = v;
    }
    for (int e = threadIdx.x; e < BK * BN; e += NT) {
      int kq, j;
      if (TB) {  // contiguous along k
        j = e / BK;
        kq = e % BK;
      } else {  // contiguous along n
        kq = e / BN;
        j = e % BN;
      }
      const int gj = col0 + j, gk = kk + kq;
      T v = T(0);
      if (gj < n && gk < k) v = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
      sB[kq][j] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kq = 0; kq < BK; ++kq) {
      T a[MT], b[MT];
#pragma unroll
      for (int r = 0; r < MT; ++r) {
        a[r] = sA[kq][ty * MT + r];
        b[r] = sB[kq][tx * MT + r];
      }
#pragma unroll
      for (int r = 0; r < MT; ++r)
#pragma unroll
        for (int c = 0; c < MT; ++c) acc[r][c] += a[r] * b[c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const int gi = row0 + ty * MT + i;
    if (gi >= m) continue;
#pragma unroll
    for (int j = 0; j < MT; ++j) {
      const int gj = col0 + tx * MT + j;
      if (gj < n) C[(size_t)gi * ldc + gj] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------- one-sided Jacobi
// On the s x s matrix R (row-major in global), accumulating V (s x s).
// Columns are rotated pairwise in round-robin order until every pair is
// orthogonal to tol; then columns are sorted by norm (descending) and
// written as RV (= U Sigma) and V, row-major s x s, plus sigma[s].
// s1_dev = sigma[0]; flag_dev |= degenerate cut at `keep`.
template <typename T>
__global__ void __launch_bounds__(1024) k_jacobi(const T* __restrict__ Rin, int s, T* __restrict__ RVout, T* __restrict__ Vout,
                         T* __restrict__ sig_out, int keep, double* s1_dev, int* flag_dev,
                         T* __restrict__ gbuf, int use_smem, size_t zs) {
  Rin = zp(Rin, zs);
  RVout = zp(RVout, zs);
  Vout = zp(Vout, zs);
  sig_out = zp(sig_out, zs);
  s1_dev = zp(s1_dev, zs);
  flag_dev = zp(flag_dev, zs);
  gbuf = zp(gbuf, zs);
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);  // 64
  T* sig = red + 64;                        // SMAX
  int* rank = reinterpret_cast<int*>(sig + SMAX);  // SMAX
  T* buf = use_smem ? reinterpret_cast<T*>(rank + SMAX) : gbuf;
  // column-major: Rc[c*s + i], Vc[c*s + i]
  T* Rc = buf;
  T* Vc = buf + (size_t)s * s;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < s * s; e += nt) {
    const int i = e / s, c = e % s;
    Rc[(size_t)c * s + i] = Rin[e];
    Vc[(size_t)c * s + i] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  T* nrm = sig;  // squared column norms, kept current by every rotation
  for (int c = wid_of(); c < s; c += (int)(blockDim.x >> 5)) {
    T a = T(0);
    for (int q = (int)(threadIdx.x & 31); q < s; q += 32) a += Rc[(size_t)c * s + q] * Rc[(size_t)c * s + q];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) nrm[c] = a;
  }
  __syncthreads();
  // columns below zero_rel of ||R||_F are numerically zero (R is often rank
  // deficient): pairs that involve one carry no information and are skipped
  __shared__ T s_fro2;
  if (tid == 0) {
    T f = T(0);
    for (int c = 0; c < s; ++c) f += nrm[c];
    s_fro2 = f;
  }
  __syncthreads();
  const T zero2 = (sizeof(T) == 8 ? T(1e-28) : T(1e-12)) * s_fro2;
  const int se = s + (s & 1);
  // rotate while |gamma| > tol * sqrt(alpha beta): s * eps in FP64; in FP32
  // rounding noise of ill-conditioned pairs stays above s * eps, so the bound
  // is 1e-5 (below the ~1e-4 accuracy of an FP32 truncation)
  const T tol = sizeof(T) == 8 ? T(2.22e-16) * T(s > 8 ? s : 8) : T(1e-5);
  const int max_sweeps = sizeof(T) == 8 ? 60 : 30;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  __shared__ int s_conv;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_conv = 1;
    // exact squared column norms once per sweep (the per-rotation updates
    // below follow the Hestenes recurrence and would otherwise drift)
    for (int c = wid; c < s; c += nw) {
      T a = T(0);
      for (int q = lane; q < s; q += 32) a += Rc[(size_t)c * s + q] * Rc[(size_t)c * s + q];
      a = warp_sum(a);
      if (lane == 0) nrm[c] = a;
    }
    __syncthreads();
    for (int r = 0; r < se - 1; ++r) {
      for (int pk = wid; pk < se / 2; pk += nw) {
        int i = pk == 0 ? 0 : ((pk + r - 1) % (se - 1)) + 1;
        int j = ((se - 1 - pk + r - 1) % (se - 1)) + 1;
        if (i >= s || j >= s) continue;
        if (i > j) {
          int t = i;
          i = j;
          j = t;
        }
        const T al = nrm[i], be = nrm[j];
        if (al <= zero2 || be <= zero2) continue;
        T* ci = Rc + (size_t)i * s;
        T* cj = Rc + (size_t)j * s;
        T ga = T(0);
        for (int q = lane; q < s; q += 32) ga += ci[q] * cj[q];
        ga = warp_sum(ga);
        if (fabs(ga) <= tol * sqrt(al) * sqrt(be)) continue;
        if (lane == 0) s_conv = 0;
        const T zeta = (be - al) / (T(2) * ga);
        const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t);
        const T sn = c * t;
        T* vi = Vc + (size_t)i * s;
        T* vj = Vc + (size_t)j * s;
        for (int q = lane; q < s; q += 32) {
          const T x = ci[q], y = cj[q];
          ci[q] = c * x - sn * y;
          cj[q] = sn * x + c * y;
          const T u = vi[q], v = vj[q];
          vi[q] = c * u - sn * v;
          vj[q] = sn * u + c * v;
        }
        if (lane == 0) {
          nrm[i] = al - t * ga;
          nrm[j] = be + t * ga;
        }
      }
      __syncthreads();
    }
    if (s_conv) {
      if (tid == 0 && flag_dev) atomicMax(flag_dev + 1, sweep + 1);
      break;
    }
    if (sweep == max_sweeps - 1 && tid == 0 && flag_dev) atomicMax(flag_dev + 1, max_sweeps);
    __syncthreads();
  }
  // singular values and descending order (ties by index)
  for (int c = wid; c < s; c += nw) {
    T a = T(0);
    for (int q = lane; q < s; q += 32) a += Rc[(size_t)c * s + q] * Rc[(size_t)c * s + q];
    a = warp_sum(a);
    if (lane == 0) sig[c] = sqrt(a);
  }
  __syncthreads();
  for (int c = tid; c < s; c += nt) {
    int rk = 0;
    for (int o = 0; o < s; ++o) rk += (sig[o] > sig[c]) || (sig[o] == sig[c] && o < c);
    rank[c] = rk;
  }
  __syncthreads();
  for (int e = tid; e < s * s; e += nt) {
    const int c = e / s, i = e % s;
    RVout[(size_t)i * s + rank[c]] = Rc[e];
    Vout[(size_t)i * s + rank[c]] = Vc[e];
  }
  for (int c = tid; c < s; c += nt) sig_out[rank[c]] = sig[c];
  __syncthreads();
  if (tid == 0) {
    T s1 = T(0);
    for (int c = 0; c < s; ++c)
      if (rank[c] == 0) s1 = sig[c];
    *s1_dev = (double)s1;
    if (keep < s && flag_dev) {
      T sk = T(0), sk1 = T(0);
      for (int c = 0; c < s; ++c) {
        if (rank[c] == keep - 1) sk = sig[c];
        if (rank[c] == keep) sk1 = sig[c];
      }
      if ((double)(sk - sk1) <= 1e-12 * (double)s1) atomicAdd(flag_dev, 1);
    }
  }
}

// deterministic pseudo-random block in (-1, 1): splitmix64 of (seed, index)
__device__ __forceinline__ double hash_unit(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9e3779b97f4a7c15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z = z ^ (z >> 31);
  return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

// Zt [s x n]: identity rows (direct case, s == n) or the pseudo-random block.
template <typename T>
__global__ void k_fill_start(T* Zt, int n, int s, uint64_t seed, int identity, size_t zs) {
  Zt = zp(Zt, zs);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * s; e += gridDim.x * blockDim.x) {
    const int c = e / n, i = e % n;
    Zt[e] = identity ? (i == c ? T(1) : T(0)) : (T)hash_unit(seed, (uint64_t)e);
  }
}

// dst[e] = (To) src[e]: a contiguous block changes precision (the FP64
// truncation of the final boundary rows in the mixed mode).
template <typename From, typename To>
__global__ void k_convert(const From* __restrict__ src, To* __restrict__ dst, size_t count, size_t zs) {
  src = zp(src, zs);
  dst = zp(dst, zs);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (To)src[e];
}

template <typename T>
__global__ void k_set_strided(T* base, size_t stride, int count, T v, size_t zs) {
  base = zp(base, zs);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) base[e * stride] = v;
}

// site[u][kp][k] = V[(u*K + k)][kp];  carry[l][a][kp] = US[(l*chiL + a)][kp] / s1
template <typename T>
__global__ void k_zip_write(const T* __restrict__ V, const T* __restrict__ US, int DL, int chiL, int DU,
                            int K, int keep, T* __restrict__ site, T* __restrict__ carry, const double* s1,
                            double* lognorm_r, size_t zs) {
  V = zp(V, zs);
  US = zp(US, zs);
  site = zp(site, zs);
  carry = zp(carry, zs);
  s1 = zp(s1, zs);
  lognorm_r = zp(lognorm_r, zs);
  const double sv = *s1;
  const T inv = sv > 0 ? (T)(1.0 / sv) : T(0);
  const int nsite = DU * keep * K, ncar = DL * chiL * keep;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nsite + ncar; e += gridDim.x * blockDim.x) {
    if (e < nsite) {
      const int k = e % K, kp = (e / K) % keep, u = e / (K * keep);
      site[e] = V[(size_t)(u * K + k) * keep + kp];
    } else {
      const int f = e - nsite;
      const int kp = f % keep, la = f / keep;
      carry[f] = US[(size_t)la * keep + kp] * inv;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *lognorm_r += log(sv);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_zip_site0(const T* __restrict__ M, int n, T* __restrict__ site, double* lognorm_r, size_t zs) {
  M = zp(M, zs);
  site = zp(site, zs);
  lognorm_r = zp(lognorm_r, zs);
  __shared__ T red[64];
  T part = T(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) part += M[i] * M[i];
  const T nrm = sqrt(block_sum(part, red));
  const T inv = nrm > T(0) ? T(1) / nrm : T(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) site[i] = M[i] * inv;
  if (threadIdx.x == 0) *lognorm_r += log((double)nrm);
}

template <typename T>
__global__ void k_mps_value(DevMPS<T> mps, int r, int cols, double* out) {
  __shared__ T v[MAXCHI], nv[MAXCHI];
  const int tid = threadIdx.x;
  if (tid == 0) v[0] = T(1);
  __syncthreads();
  int chi = 1;
  for (int j = 0; j < cols; ++j) {
    const int* dA = mps.dimA + (r * cols + j) * 3;
    const int chiL = dA[1], chiR = dA[2];
    const T* A = mps.A + (size_t)(r * cols + j) * mps.site_stride;  // p == 1
    for (int b = tid; b < chiR; b += blockDim.x) {
      T acc = T(0);
      for (int a = 0; a < chiL && a < chi; ++a) acc += v[a] * A[(size_t)a * chiR + b];
      nv[b] = acc;
    }
    __syncthreads();
    for (int b = tid; b < chiR; b += blockDim.x) v[b] = nv[b];
    chi = chiR;
    __syncthreads();
  }
  if (tid == 0) *out = (double)v[0];
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
cudaError_t launch_weights(const DevTables& tb, DevWeights<T> wt, double beta_u, cudaStream_t st) {
  count_launches("k_weights", st);
  ZOK(tb, wt);
  k_weights<T><<<dim3(tb.n, 1, zn()), 256, 0, st>>>(tb, wt, beta_u, zs());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_left_canonical(DevMPS<T> mps, int r, int cols, const int*, T* scratch, cudaStream_t st) {
  // staged site: (MAXP * chi) x chi elements
  const size_t chi = (size_t)std::sqrt((double)(mps.site_stride / MAXP));
  const size_t base = sizeof(T) * (64 + 2 * SMAX + MAXCHI * MAXCHI);
  const size_t full = base + sizeof(T) * MAXP * chi * chi;
  const int use_smem = full <= 200 * 1024 ? 1 : 0;
  // FP32 sites staged with room for the panels' scratch and one panel copy
  // (QR_PB vectors of up to MAXP * chi entries)
  const size_t with_panels = full + sizeof(T) * (2 * SMAX * QR_PB + chol_scratch_elems<T>() + QR_PB * MAXP * chi);
  const bool panels = sizeof(T) == 4 && use_smem && with_panels <= 200 * 1024;
  static std::once_flag attr_once;  // thread-safe: batches enqueue from several threads
  std::call_once(attr_once, [&] {
    cudaFuncSetAttribute(k_left_canonical<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096);
    cudaFuncSetAttribute(k_left_canonical<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096);
  });
  ZOK(mps, scratch);
  count_launches("k_left_canonical", st);
  if (panels)
    k_left_canonical<T, true><<<dim3(1, 1, zn()), 512, with_panels, st>>>(mps, r, cols, scratch, use_smem, zs());
  else
    k_left_canonical<T, false><<<dim3(1, 1, zn()), 1024, use_smem ? full : base, st>>>(mps, r, cols, scratch,
                                                                                     use_smem, zs());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zip_matrix(const DevTables& tb, DevWeights<T> wt, const T* B, int chiL, int p, int chiR,
                              const T* C, int DR, int K, int site, int DL, int DU, T* T1, T* M,
                              cudaStream_t st) {
  const size_t total = (size_t)chiL * p * DR * K;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  ZOK(tb, wt, B, C, T1, M);
  count_launches("k_zip_T1", st, 2.0 * chiL * p * DR * K * chiR);
  k_zip_T1<T><<<dim3(blocks, 1, zn()), 256, 0, st>>>(B, chiL, p, chiR, C, DR, K, T1, zs());
  const int kchunk = K >= 8 ? 4 : 1;
  dim3 grid(chiL, (K + kchunk - 1) / kchunk, zn());
  const size_t smem = sizeof(T) * ((size_t)p * DR + (size_t)DL * MAXP);
  // a lockstep group fills the GPU: one block per bond index with every k
  // (when the slab and the Y tables fit), else the per-k-chunk kernel
  const size_t smem_rows = sizeof(T) * ((size_t)p * DR * K + (size_t)DU * MAXP * K + (size_t)DL * MAXP);
  const bool rows = zn() > 1 && smem_rows <= 160 * 1024;
  static std::once_flag attr_once;  // thread-safe: batches enqueue from several threads
  std::call_once(attr_once, [&] {
    cudaFuncSetAttribute(k_zip_M<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(T) * 2 * (size_t)MAXP * MAXBOND));
    cudaFuncSetAttribute(k_zip_M_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  });
  count_launches("k_zip_M", st);
  if (rows)
    k_zip_M_rows<T><<<dim3(chiL, 1, zn()), 256, smem_rows, st>>>(tb, wt, site, T1, chiL, p, DR, K, DL, DU, M, zs());
  else
    k_zip_M<T><<<grid, 256, smem, st>>>(tb, wt, site, T1, chiL, p, DR, K, DL, DU, kchunk, M, zs());
  return cudaGetLastError();
}

template <typename T>
cudaError_t gemm(bool transA, int m, int n, int k, const T* A, int lda, const T* B, int ldb, T* C, int ldc,
                 cudaStream_t st) {
  return gemm2<T>(transA, false, m, n, k, A, lda, B, ldb, C, ldc, st);
}

// One k_gemm variant: MT x MT outputs per thread (32 / MT threads along each
// tile edge).
template <typename T, bool TA, bool TB>
void gemm_variant(int v, dim3 grid, int m, int n, int k, const T* A, int lda, const T* B, int ldb, T* C, int ldc,
                  size_t z, cudaStream_t st) {
  switch (v) {
    case 0: k_gemm<T, TA, TB, 1><<<grid, 1024, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, z); break;
    case 1: k_gemm<T, TA, TB, 2><<<grid, 256, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, z); break;
    case 2: k_gemm<T, TA, TB, 4><<<grid, 64, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, z); break;
    default: k_gemm<T, TA, TB, 8><<<grid, 16, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, z); break;
  }
}

template <typename T>
cudaError_t gemm2(bool transA, bool transB, int m, int n, int k, const T* A, int lda, const T* B, int ldb, T* C,
                  int ldc, cudaStream_t st) {
  ZOK(A, B, C);
  dim3 grid((n + 31) / 32, (m + 31) / 32, zn());
  const size_t z = zs();
  auto run = [&](int v) {
    if (transA && transB)
      gemm_variant<T, true, true>(v, grid, m, n, k, A, lda, B, ldb, C, ldc, z, st);
    else if (transA)
      gemm_variant<T, true, false>(v, grid, m, n, k, A, lda, B, ldb, C, ldc, z, st);
    else if (transB)
      gemm_variant<T, false, true>(v, grid, m, n, k, A, lda, B, ldb, C, ldc, z, st);
    else
      gemm_variant<T, false, false>(v, grid, m, n, k, A, lda, B, ldb, C, ldc, z, st);
  };
  // built-in choice: a lockstep group fills the GPU, 4 x 4 outputs per
  // thread (64 threads per tile, more multiply-adds per shared-memory read);
  // alone, 2 x 2 on 256 threads (shorter chains for the small, latency-bound
  // products).  Every variant sums each output over k in the same order (the
  // same fused multiply-adds), so the autotuner may pick any of them.
  const long long shape[] = {(long long)sizeof(T), transA, transB, m, n, k, lda, ldb, ldc};
  const int v = tune_pick("k_gemm", shape, 9, st, 4, 0xfu, zn() > 1 ? 2 : 1, run);
  count_launches("k_gemm", st, 2.0 * m * n * k);
  run(v);
  return cudaGetLastError();
}

template <typename From, typename To>
cudaError_t launch_convert(const From* src, To* dst, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const size_t blocks = std::min<size_t>((count + 255) / 256, 152 * 8);
  ZOK(src, dst);
  count_launches("k_convert", st);
  k_convert<From, To><<<dim3((unsigned)blocks, 1, zn()), 256, 0, st>>>(src, dst, count, zs());
  return cudaGetLastError();
}
template cudaError_t launch_convert<float, double>(const float*, double*, size_t, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, size_t, cudaStream_t);

template <typename T>
cudaError_t launch_set_strided(T* base, size_t stride, int count, T v, cudaStream_t st) {
  ZOK(base);
  count_launches("k_set_strided", st);
  k_set_strided<T><<<dim3((count + 255) / 256, 1, zn()), 256, 0, st>>>(base, stride, count, v, zs());
  return cudaGetLastError();
}

// Columns of the subspace-iteration block: FP64 keeps a wide block (fast
// convergence, reference accuracy); FP32 resolves ~1e-7 relative anyway, so a
// narrower block of keep + 16 columns suffices and halves the work.
template <typename T>
static int block_cols(int n, int keep) {
  if (n <= SMAX) return n;
  int s = sizeof(T) == 8 ? std::max(2 * keep, keep + 8) : keep + 16;
  return std::min(std::min(s, n), SMAX);
}

// Vectors this long or longer go through the multi-CTA TSQR.
constexpr int TSQR_MIN_LEN = 2048;

// Stacked R factors of a TSQR of vectors of length len and of its recursion
// (blocks of >= 256 entries; every level at most half the previous).
size_t tsqr_scratch_elems(int len) { return 2 * (size_t)SMAX * SMAX * ((size_t)len / 256 + 2); }

size_t truncated_svd_work(int m, int n, int) {
  const size_t s = (size_t)SMAX;  // upper bound of block_cols for any call
  // Z (n s), Y (m s), R (s s), RV (s s), VJ (s s), sig (s), jacobi global buf
  // (2 s s), then the TSQR scratch when a dimension is long
  const int mx = std::max(m, n);
  return s * n + s * m + 5 * s * s + s + 64 + (mx >= TSQR_MIN_LEN ? tsqr_scratch_elems(mx) : 0);
}

size_t truncated_svd_sigma_offset(int m, int n, int keep) {
  const size_t s = (size_t)block_cols<double>(n, keep);
  return s * n + s * m + 3 * s * s;
}

template <typename T>
static void cgs2_rows(T* X, int nvec, int len, T* Rout, cudaStream_t st, int reorth);

// Entries per TSQR block: staged in shared memory when it fits (FP32), else
// 1024 entries worked on in global memory (L2); never fewer than nvec.
template <typename T>
static int tsqr_block(int nvec, int* use_smem) {
  const size_t room = (200 * 1024) / sizeof(T) - (64 + 2 * SMAX) - (size_t)nvec * nvec;
  int bl = (int)(room / nvec) / 32 * 32;
  if (bl >= 256 && bl >= nvec) {
    *use_smem = 1;
    return std::min(bl, 1024);
  }
  *use_smem = 0;
  return 1024;
}

template <typename T>
static void tall_qr(T* X, int nvec, int len, T* Rout, T* S, cudaStream_t st, int reorth) {
  int use_smem = 0;
  const int bl = tsqr_block<T>(nvec, &use_smem);
  const int nb = (len + bl - 1) / bl;
  const size_t leaf_smem = sizeof(T) * ((64 + 2 * SMAX) + (size_t)nvec * nvec + (use_smem ? (size_t)nvec * bl : 0));
  const size_t apply_smem = sizeof(T) * ((size_t)nvec * nvec + (size_t)nvec * 64);
  static std::once_flag attr_once;  // thread-safe: batches enqueue from several threads
  std::call_once(attr_once, [&] {
    cudaFuncSetAttribute(k_tsqr_leaf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096);
    cudaFuncSetAttribute(k_tsqr_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096);
  });
  if (!zok(X, S, Rout)) return;
  count_launches("k_tsqr_leaf", st, 4.0 * len * nvec * nvec);
  k_tsqr_leaf<T><<<dim3(nb, 1, zn()), 512, leaf_smem, st>>>(X, nvec, len, bl, S, use_smem, zs());
  const int slen = nb * nvec;
  if (slen >= TSQR_MIN_LEN && slen < len)
    tall_qr<T>(S, nvec, slen, Rout, S + (size_t)nvec * slen, st, reorth);
  else
    cgs2_rows<T>(S, nvec, slen, Rout, st, reorth);
  count_launches("k_tsqr_apply", st, 2.0 * len * nvec * nvec);
  k_tsqr_apply<T><<<dim3(nb, 1, zn()), 512, apply_smem, st>>>(X, nvec, len, bl, S, zs());
}

// reorth: the result must be orthonormal to rounding (a QR whose R is used,
// or whose Q is a site of an MPS), so panels with strong cancellation take
// the second pass; the power steps of the subspace iteration only need a
// basis of the span and skip it.
template <typename T>
static void cgs2_rows(T* X, int nvec, int len, T* Rout, cudaStream_t st, int reorth) {
  const size_t base = sizeof(T) * (64 + 2 * SMAX + 2 * SMAX * QR_PB + chol_scratch_elems<T>());
  const size_t full = base + sizeof(T) * (size_t)nvec * len;
  const int use_smem = full <= 200 * 1024 ? 1 : 0;
  // FP32 panels by guarded Cholesky-QR when a copy of one panel fits too and
  // the block is large (>= 32 vectors of >= 256 entries), where the
  // per-vector chain costs most; small blocks keep per-vector CGS2 (with
  // Cholesky panels on them the mixed log Z of a 3 x 3 king's Ising lattice
  // at beta 2 moved beyond 1e-3 of the FP64 value)
  const size_t with_copy = full + sizeof(T) * (size_t)QR_PB * len;
  const int use_chol = (sizeof(T) == 4 && use_smem && with_copy <= 200 * 1024 && nvec >= 32 && len >= 256) ? 1 : 0;
  static std::once_flag attr_once;  // thread-safe: batches enqueue from several threads
  std::call_once(attr_once, [&] { cudaFuncSetAttribute(k_cgs2_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096); });
  // one thread per element up to 512 (the register budget of the panel
  // products), at least 4 warps
  const int threads = std::max(128, std::min(512, (len + 31) / 32 * 32));
  if (!zok(X, Rout)) return;
  count_launches("k_cgs2_rows", st, 4.0 * len * nvec * nvec);
  k_cgs2_rows<T><<<dim3(1, 1, zn()), threads, use_chol ? with_copy : (use_smem ? full : base), st>>>(
      X, nvec, len, len, Rout, use_smem, use_chol, reorth, zs());
}

template <typename T>
void launch_cgs2_rows(T* X, int nvec, int len, T* Rout, cudaStream_t st) {
  cgs2_rows<T>(X, nvec, len, Rout, st, 1);
}

// QR of the rows of X: one CTA for short vectors, TSQR for long ones (tsq:
// tsqr_scratch_elems(len) elements).
template <typename T>
static void qr_rows(T* X, int nvec, int len, T* Rout, T* tsq, cudaStream_t st, int reorth) {
  if (len >= TSQR_MIN_LEN)
    tall_qr<T>(X, nvec, len, Rout, tsq, st, reorth);
  else
    cgs2_rows<T>(X, nvec, len, Rout, st, reorth);
}

// Work layout: Zt [s x n], Yt [s x m] (rows = the block's column vectors),
// R, RV, VJ [s x s], sig [s], Jacobi spill buffer [2 s s].
template <typename T>
cudaError_t truncated_svd(const T* M, int m, int n, int keep, int iters, uint64_t seed, T* V, T* US, T* work,
                          size_t, double* s1_dev, int* flag_dev, cudaStream_t st, float* tcw, size_t tcw_elems) {
  const int s = block_cols<T>(n, keep);
  T* Zt = work;
  T* Yt = Zt + (size_t)n * s;
  T* R = Yt + (size_t)m * s;
  T* RV = R + (size_t)s * s;
  T* VJ = RV + (size_t)s * s;
  T* sig = VJ + (size_t)s * s;
  T* jbuf = sig + s + 64;
  T* tsq = jbuf + 2 * (size_t)s * s;
  const bool direct = n <= SMAX;
  // FP32 products on the tensor cores when the matrix is large
  std::optional<TcGemm> tc;
  if constexpr (std::is_same<T, float>::value) {
    if (!direct && tcw && tc_gemm_eligible(m, n, s) && tcw_elems >= tc_gemm_elems(m, n, s))
      tc.emplace(tcw, tcw_elems, M, m, n, flag_dev + 2, st);
  }
  // Yt = (M Z)^T and Zt = (M^T Y)^T
  auto prod_y = [&]() -> cudaError_t {
    if constexpr (std::is_same<T, float>::value)
      if (tc) return tc->run(false, Zt, s, Yt);
    return gemm2<T>(false, true, s, m, n, Zt, n, M, n, Yt, m, st);
  };
  auto prod_z = [&]() -> cudaError_t {
    if constexpr (std::is_same<T, float>::value)
      if (tc) return tc->run(true, Yt, s, Zt);
    return gemm2<T>(false, false, s, n, m, Yt, m, M, n, Zt, n, st);
  };
  ZOK(M, V, US, work, s1_dev, flag_dev, tcw);
  count_launches("k_fill_start", st);
  k_fill_start<T><<<dim3((n * s + 255) / 256, 1, zn()), 256, 0, st>>>(Zt, n, s, seed, direct ? 1 : 0, zs());
  if (!direct) {
    // the pseudo-random start block is well conditioned, so the power steps
    // need no orthonormalisation of it; the Rayleigh-Ritz step below does
    // need an orthonormal Z, hence the QR when there are no power steps
    if (iters == 0) qr_rows(Zt, s, n, (T*)nullptr, tsq, st, 1);
    for (int it = 0; it < iters; ++it) {
      cudaError_t e = prod_y();  // Y = M Z
      if (e != cudaSuccess) return e;
      qr_rows(Yt, s, m, (T*)nullptr, tsq, st, 0);
      e = prod_z();  // Z = M^T Y
      if (e != cudaSuccess) return e;
      qr_rows(Zt, s, n, (T*)nullptr, tsq, st, 0);
    }
  }
  // P = M Z = Q R (rows of Yt become the columns of Q); R = U_R Sigma V_J^T
  if (direct) {
    gemm2<T>(false, true, s, m, n, Zt, n, M, n, Yt, m, st);
  } else {
    const cudaError_t e = prod_y();
    if (e != cudaSuccess) return e;
  }
  qr_rows(Yt, s, m, R, tsq, st, 1);
  const size_t jsm_base = sizeof(T) * (64 + SMAX) + sizeof(int) * SMAX;
  const size_t jsm_full = jsm_base + sizeof(T) * 2 * (size_t)s * s;
  const int use_smem = jsm_full <= 200 * 1024 ? 1 : 0;
  const size_t jsm = use_smem ? jsm_full : jsm_base;
  static std::once_flag attr_once;  // thread-safe: batches enqueue from several threads
  std::call_once(attr_once, [&] { cudaFuncSetAttribute(k_jacobi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096); });
  count_launches("k_jacobi", st);
  k_jacobi<T><<<dim3(1, 1, zn()), 1024, jsm, st>>>(R, s, RV, VJ, sig, keep, s1_dev, flag_dev, jbuf, use_smem, zs());
  // V = Z VJ[:, :keep] = Zt^T VJ,  US = Q RV[:, :keep] = Yt^T RV
  gemm2<T>(true, false, n, keep, s, Zt, n, VJ, s, V, keep, st);
  gemm2<T>(true, false, m, keep, s, Yt, m, RV, s, US, keep, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zip_write(const T* V, const T* US, int DL, int chiL, int DU, int K, int keep, T* site_out,
                             T* carry_out, const double* s1_dev, double* lognorm_r, cudaStream_t st) {
  const int tot = DU * keep * K + DL * chiL * keep;
  ZOK(V, US, site_out, carry_out, s1_dev, lognorm_r);
  count_launches("k_zip_write", st);
  k_zip_write<T><<<dim3(std::min((tot + 255) / 256, 1024), 1, zn()), 256, 0, st>>>(
      V, US, DL, chiL, DU, K, keep, site_out, carry_out, s1_dev, lognorm_r, zs());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zip_site0(const T* M, int DU, int K, T* site_out, double* lognorm_r, cudaStream_t st) {
  ZOK(M, site_out, lognorm_r);
  count_launches("k_zip_site0", st);
  k_zip_site0<T><<<dim3(1, 1, zn()), 1024, 0, st>>>(M, DU * K, site_out, lognorm_r, zs());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mps_value(DevMPS<T> mps, int r, int cols, double* out, cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;  // not part of a grouped solve
  count_launches("k_mps_value", st);
  k_mps_value<T><<<1, 64, 0, st>>>(mps, r, cols, out);
  return cudaGetLastError();
}

#define SPG_INST(T)                                                                                       \
  template cudaError_t launch_weights<T>(const DevTables&, DevWeights<T>, double, cudaStream_t);        \
  template cudaError_t launch_left_canonical<T>(DevMPS<T>, int, int, const int*, T*, cudaStream_t);     \
  template cudaError_t launch_zip_matrix<T>(const DevTables&, DevWeights<T>, const T*, int, int, int,   \
                                            const T*, int, int, int, int, int, T*, T*, cudaStream_t);   \
  template cudaError_t truncated_svd<T>(const T*, int, int, int, int, uint64_t, T*, T*, T*, size_t,     \
                                        double*, int*, cudaStream_t, float*, size_t);                   \
  template cudaError_t launch_zip_write<T>(const T*, const T*, int, int, int, int, int, T*, T*,         \
                                           const double*, double*, cudaStream_t);                       \
  template cudaError_t launch_zip_site0<T>(const T*, int, int, T*, double*, cudaStream_t);              \
  template cudaError_t launch_mps_value<T>(DevMPS<T>, int, int, double*, cudaStream_t);                 \
  template cudaError_t gemm<T>(bool, int, int, int, const T*, int, const T*, int, T*, int, cudaStream_t);   \
  template cudaError_t gemm2<T>(bool, bool, int, int, int, const T*, int, const T*, int, T*, int,         \
                                cudaStream_t);                                                          \
  template cudaError_t launch_set_strided<T>(T*, size_t, int, T, cudaStream_t);                          \
  template void launch_cgs2_rows<T>(T*, int, int, T*, cudaStream_t);

SPG_INST(double)
SPG_INST(float)

}  // namespace spg
