// Search kernels: right environments (S5), conditional marginals (S6),
// branch merging and pruning to max_states (S7), exact final energies (S8).
//
// Paper: Sec. 2 (branch and bound in the probability space, one Potts
// variable at a time in a fixed order; marginals from the contracted network;
// merging of partial configurations equal on the boundary of the explored
// region), Sec. 3.1 (SearchParameters(max_states, cut_off_prob),
// merge_branches, low_energy_spectrum), Fig. 1(d)-(e).
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <mutex>

#include <type_traits>

#include "spg_internal.h"

namespace spg {

namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = lane < nw ? red[lane] : T(0);
  return warp_sum(t);
}
template <typename T>
__device__ T block_max(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = lane < nw ? red[lane] : T(-INFINITY);
  return warp_max(t);
}

// order-preserving map double -> u64 (NaN treated as -inf)
__device__ __forceinline__ unsigned long long ord_f64(double v) {
  if (v != v) v = -INFINITY;
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord_f64(unsigned long long k) {
  unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ unsigned long long ord_i64(int64_t v) {
  return (unsigned long long)v ^ 0x8000000000000000ull;
}

__device__ __forceinline__ int dim_of(const DevTables& tb, int s, int k) { return tb.dims[s * DIMW + k]; }

// ---------------------------------------------------------------- S5 right environments
// For beam element b at the start of row i, with B = B_{i+1}, u_j the PD
// class of the fixed cluster (i-1, j) and g_j = gD_{(i-1, j)}[u_j]:
//   R_L = 1;  R_j[a][l] = bA[l / Gin][u_j] sum_h bL[l][h] Y[h][a],
//   Y[h][a] = sum_{x: PL x = h} w(x) bU[u_j][PU x]
//             sum_a' B_j[PD x][a][a'] R_{j+1}[a'][PR x * Gout + g_j]
// stored at R[((b*(cols+1) + j)*chi + a)*rs + l], each R_j scaled to max |.| = 1.
// One block handles G consecutive beam elements; the site B_j, shared by
// all of them, is staged in shared memory once per column when it fits, and
// so are the G current environments when the bond is small (use_rn).
template <typename T>
__global__ void k_right_envs(DevTables tb, DevWeights<T> wt, DevMPS<T> mps, int row, DevSearch ds,
                             DevBeamT<T> bt, int cur, int G, int use_smem, int use_rn, int use_t, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  mps = zp(mps, zs);
  ds = zp(ds, zs);
  bt = zp(bt, zs);
  const int nb = ds.n_beam[cur];
  const int b0 = blockIdx.x * G;
  if (b0 >= nb) return;
  const int gn = min(G, nb - b0);
  const int rs = bt.rs;
  extern __shared__ unsigned char smem_raw[];
  T* Y = reinterpret_cast<T*>(smem_raw);           // [MAXP][MAXCHI]
  T* red = Y + MAXP * MAXCHI;                      // 32
  T* sbL = red + 32;                               // [rs][MAXP]
  T* Rn = sbL + (size_t)rs * MAXP;                 // [G][chi*rs] (use_rn)
  T* Bs = Rn + (use_rn ? (size_t)G * MAXCHI * rs : 0);  // staged site (use_smem)
  T* Tp = Bs + mps.site_stride;                    // [p][DR][chiL] products (use_t)
  __shared__ T sw[MAXS], sbU[256], sbA[256];
  __shared__ uint8_t sPU[MAXS], sPD[MAXS], sPR[MAXS];
  __shared__ int16_t sxs[MAXS];
  __shared__ int soff[MAXP + 1];
  const int cols = tb.cols, chi = bt.chi;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t renv = (size_t)chi * rs;  // one environment
  for (int g = 0; g < gn; ++g) {
    const int b = b0 + g;
    T* Rb = bt.R + (size_t)b * (cols + 1) * renv;
    for (int e = tid; e < (int)renv; e += nt) {
      const T v = e == 0 ? T(1) : T(0);
      Rb[(size_t)cols * renv + e] = v;
      if (use_rn) Rn[(size_t)g * renv + e] = v;
    }
    if (tid == 0) pick(ds.rid, cur)[b] = b;
    for (int a = tid; a < chi; a += nt) pick(bt.lenv, cur)[(size_t)b * chi + a] = a == 0 ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = cols - 1; j >= 1; --j) {
    const int s = row * cols + j;
    const int* dA = mps.dimA + ((row + 1) * cols + j) * 3;
    const int p = dA[0], chiL = dA[1], chiR = dA[2];
    const T* Ag = mps.A + (size_t)((row + 1) * cols + j) * mps.site_stride;
    // staged transposed, Bs[(s*chiR + a')*chiL + a]: consecutive lanes (a)
    // then read consecutive words (no bank conflicts)
    if (use_smem)
      for (int e = tid; e < p * chiL * chiR; e += nt) {
        const int ap = e % chiR, a = (e / chiR) % chiL, sg = e / (chiR * chiL);
        Bs[((size_t)sg * chiR + ap) * chiL + a] = Ag[e];
      }
    const int DL = dim_of(tb, s, D_DL), NL = dim_of(tb, s, D_NL), Gin = dim_of(tb, s, D_GIN);
    const int Gout = dim_of(tb, s, D_GOUT);
    const size_t so = (size_t)s * tb.dmax;
    const int d = tb.d[s];
    // this column's tables, staged once for all G beam elements
    for (int x = tid; x < d; x += nt) {
      sw[x] = wt.w[so + x];
      sPU[x] = tb.PU[so + x];
      sPD[x] = tb.PD[so + x];
      sPR[x] = tb.PR[so + x];
      sxs[x] = tb.xsL[so + x];
    }
    for (int e = tid; e < 256; e += nt) {
      sbU[e] = wt.bU[(size_t)s * 256 + e];
      sbA[e] = wt.bA[(size_t)s * 256 + e];
    }
    for (int e = tid; e < DL * MAXP; e += nt) sbL[e] = wt.bL[(size_t)s * tb.lstride + e];
    for (int e = tid; e <= MAXP; e += nt) soff[e] = tb.xoffL[s * (MAXP + 1) + e];
    __syncthreads();
    for (int g = 0; g < gn; ++g) {
      const int b = b0 + g;
      const uint16_t* stb = pick(ds.states, cur) + (size_t)b * ds.N;
      const int u = row > 0 ? tb.PD[(size_t)(s - cols) * tb.dmax + stb[s - cols]] : 0;
      const int gu = row > 0 ? tb.gD[(size_t)(s - cols) * MAXP + u] : 0;
      const T* Rg = use_rn ? Rn + (size_t)g * renv : bt.R + ((size_t)b * (cols + 1) + j + 1) * renv;
      // Y[h][a] = sum_{x in group h} w(x) bU[u][PU x] sum_a' A[PD x][a][a'] Rg[a'][PR x * Gout + gu]
      if (use_t) {
        // first every product Tp[pd][r][a] = sum_a' A[pd][a][a'] Rg[a'][r] (r < DR),
        // four consecutive a per thread (one R load per four multiply-adds),
        // then the weighted sums over the states of each class from Tp
        const int DR = dim_of(tb, s, D_DR);
        const int na4 = (chiL + 3) >> 2;
        bool tile = false;
        if constexpr (sizeof(T) == 4) tile = (chiL % 4 == 0) && (DR % 4 == 0) && (rs % 4 == 0);
        if constexpr (sizeof(T) == 4) {
          // FP32 with bonds in multiples of 4: a 4 (a) x 4 (r) tile per thread,
          // one 16-byte load of A and one of R per 16 multiply-adds (the same
          // summation order over a' as the loop below).  Rg and Bs rows start
          // on 16-byte boundaries: every offset is a multiple of 4 floats.
          if (tile) {
            const int nr4 = DR >> 2, ca4 = chiL >> 2;
            for (int e = tid; e < p * nr4 * na4; e += nt) {
              const int a0 = (e % na4) * 4, r0 = ((e / na4) % nr4) * 4, pd = e / (na4 * nr4);
              const float4* ab = reinterpret_cast<const float4*>(Bs + (size_t)pd * chiR * chiL + a0);
              const float* rg = reinterpret_cast<const float*>(Rg) + r0;
              float c[4][4];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) c[i][k] = 0.f;
              for (int ap = 0; ap < chiR; ++ap) {
                const float4 av = ab[(size_t)ap * ca4];
                const float4 rv = *reinterpret_cast<const float4*>(rg + (size_t)ap * rs);
                const float a4[4] = {av.x, av.y, av.z, av.w};
                const float r4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                  for (int k = 0; k < 4; ++k) c[i][k] += a4[i] * r4[k];
              }
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                T* tp = Tp + ((size_t)pd * DR + r0 + k) * chiL + a0;
#pragma unroll
                for (int i = 0; i < 4; ++i) tp[i] = c[i][k];
              }
            }
          }
        }
        if (!tile)
        for (int e = tid; e < p * DR * na4; e += nt) {
          const int a0 = (e % na4) * 4, r = (e / na4) % DR, pd = e / (na4 * DR);
          const T* ab = Bs + (size_t)pd * chiR * chiL + a0;
          T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);
          for (int ap = 0; ap < chiR; ++ap) {
            const T rv = Rg[(size_t)ap * rs + r];
            const T* av = ab + (size_t)ap * chiL;
            t0 += av[0] * rv;
            if (a0 + 1 < chiL) t1 += av[1] * rv;
            if (a0 + 2 < chiL) t2 += av[2] * rv;
            if (a0 + 3 < chiL) t3 += av[3] * rv;
          }
          T* tp = Tp + ((size_t)pd * DR + r) * chiL + a0;
          tp[0] = t0;
          if (a0 + 1 < chiL) tp[1] = t1;
          if (a0 + 2 < chiL) tp[2] = t2;
          if (a0 + 3 < chiL) tp[3] = t3;
        }
        __syncthreads();
        for (int e = tid; e < NL * chiL; e += nt) {
          const int h = e / chiL, a = e % chiL;
          T acc = T(0);
          for (int q = soff[h]; q < soff[h + 1]; ++q) {
            const int x = sxs[q];
            acc += sw[x] * sbU[u * 16 + sPU[x]] * Tp[((size_t)sPD[x] * DR + sPR[x] * Gout + gu) * chiL + a];
          }
          Y[h * MAXCHI + a] = acc;
        }
      } else
      for (int e = tid; e < NL * chiL; e += nt) {
        const int h = e / chiL, a = e % chiL;
        T acc = T(0);
        for (int q = soff[h]; q < soff[h + 1]; ++q) {
          const int x = sxs[q];
          const T c = sw[x] * sbU[u * 16 + sPU[x]];
          const int pr = sPR[x] * Gout + gu;
          // element (a, a') of slice PD x: Bs[(PD*chiR + a')*chiL + a] when
          // staged, else A[(PD*chiL + a)*chiR + a']
          const size_t sa = use_smem ? (size_t)chiL : 1;
          const T* arow = use_smem ? Bs + (size_t)sPD[x] * chiR * chiL + a
                                   : Ag + ((size_t)sPD[x] * chiL + a) * chiR;
          T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);
          int ap = 0;
          for (; ap + 3 < chiR; ap += 4) {
            t0 += arow[ap * sa] * Rg[(size_t)ap * rs + pr];
            t1 += arow[(ap + 1) * sa] * Rg[(size_t)(ap + 1) * rs + pr];
            t2 += arow[(ap + 2) * sa] * Rg[(size_t)(ap + 2) * rs + pr];
            t3 += arow[(ap + 3) * sa] * Rg[(size_t)(ap + 3) * rs + pr];
          }
          for (; ap < chiR; ++ap) t0 += arow[ap * sa] * Rg[(size_t)ap * rs + pr];
          acc += c * ((t0 + t1) + (t2 + t3));
        }
        Y[h * MAXCHI + a] = acc;
      }
      __syncthreads();
      // R_j[a][l] = bA[l / Gin][u] sum_h bL[l][h] Y[h][a], written unscaled,
      // then scaled in place to max |.| = 1 (each thread rescales its own
      // entries)
      T* Rj = bt.R + ((size_t)b * (cols + 1) + j) * renv;
      T* Rgw = use_rn ? Rn + (size_t)g * renv : nullptr;
      T mx = T(0);
      for (int e = tid; e < (int)renv; e += nt) {
        const int a = e / rs, l = e % rs;
        T acc = T(0);
        if (a < chiL && l < DL) {
          for (int h = 0; h < NL; ++h) acc += sbL[l * MAXP + h] * Y[h * MAXCHI + a];
          acc *= sbA[(l / Gin) * 16 + u];
        }
        Rj[e] = acc;
        mx = max(mx, (T)fabs((double)acc));
      }
      mx = block_max(mx, red);  // contains __syncthreads
      const T inv = mx > T(0) ? T(1) / mx : T(0);
      for (int e = tid; e < (int)renv; e += nt) {
        const T v = Rj[e] * inv;
        Rj[e] = v;
        if (use_rn) Rgw[e] = v;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- S6 marginals
// log q for q > 0 in the precision of the contraction: FP64 log in FP64 mode;
// in the mixed mode q = m 2^e (m in [0.5, 1), split from the bit pattern) and
// log q = log m + e log 2 with log m in FP32 (absolute error ~1e-7, the FP32
// mode's accuracy), so the FP64 pipe only forms the weights and their sum.
template <typename T>
__device__ __forceinline__ double log_pos(double q) {
  if constexpr (sizeof(T) == 8) {
    return log(q);
  } else {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(q);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex == 0) return log(q);  // subnormal
    const double m = __longlong_as_double((long long)((bits & 0x000fffffffffffffull) | 0x3fe0000000000000ull));
    return (double)logf((float)m) + (double)(ex - 1022) * 0.69314718055994530942;
  }
}

// One block per beam element b at site s = (i, j), with l the left bond
// fixed by clusters (i, j-1) and (i-1, j-1), u the PD class of (i-1, j) and
// g = gD_{(i-1, j)}[u]:
//   v[p][a'] = sum_a lenv[a] B[p][a][a'];  Z[p][r] = sum_a' v[p][a'] R_{j+1}[a'][r * Gout + g]
//   q(x) = w(x) bL[l][PL x] bU[u][PU x] Z[PD x][PR x]   (FP64 weights, q < 0 -> 0)
//   logc[b][x] = log q(x) - log sum_x q(x)
//   candE[b][x] = E[b] + E_s(x) + RL[l][PL x] + RU[u][PU x] + RA_{s+1}[PR x][u']
// (u' the PD class of (i-1, j+1); RA of site s+1 holds the anti-diagonal
// edge (i-1, j+1)-(i, j)).  The factor bA[l / Gin][u] is the same for every
// x and cancels.
template <typename T>
__global__ void k_marginals(DevTables tb, DevWeights<double> wd, DevMPS<T> mps, int site, DevSearch ds,
                            DevBeamT<T> bt, int cur, size_t zs) {
  tb = zp(tb, zs);
  wd = zp(wd, zs);
  mps = zp(mps, zs);
  ds = zp(ds, zs);
  bt = zp(bt, zs);
  const int b = blockIdx.x;
  if (b >= ds.n_beam[cur]) return;
  __shared__ T sl[MAXCHI];
  __shared__ T sv[MAXP * MAXCHI];
  __shared__ double sZ[MAXP * MAXP];
  __shared__ double red[32];
  const int cols = tb.cols, chi = bt.chi, rs = bt.rs;
  const int i = site / cols, j = site % cols;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int* dA = mps.dimA + ((i + 1) * cols + j) * 3;
  const int p = dA[0], chiL = dA[1], chiR = dA[2];
  const T* A = mps.A + (size_t)((i + 1) * cols + j) * mps.site_stride;
  const int NR = dim_of(tb, site, D_NR), Gin = dim_of(tb, site, D_GIN), Gout = dim_of(tb, site, D_GOUT);
  const uint16_t* stb = pick(ds.states, cur) + (size_t)b * ds.N;
  const size_t dm = tb.dmax;
  const int a_l = j > 0 ? tb.PR[(size_t)(site - 1) * dm + stb[site - 1]] : 0;
  const int g_l = (j > 0 && i > 0) ? tb.PG[(size_t)(site - cols - 1) * dm + stb[site - cols - 1]] : 0;
  const int l = a_l * Gin + g_l;
  const int u = i > 0 ? tb.PD[(size_t)(site - cols) * dm + stb[site - cols]] : 0;
  const int gu = i > 0 ? tb.gD[(size_t)(site - cols) * MAXP + u] : 0;
  const bool adr = i > 0 && j + 1 < cols;
  const int ur = adr ? tb.PD[(size_t)(site - cols + 1) * dm + stb[site - cols + 1]] : 0;
  for (int a = tid; a < chiL; a += nt) sl[a] = pick(bt.lenv, cur)[(size_t)b * chi + a];
  __syncthreads();
  for (int e = tid; e < p * chiR; e += nt) {
    const int s = e / chiR, ap = e % chiR;
    T acc = T(0);
    for (int a = 0; a < chiL; ++a) acc += sl[a] * A[((size_t)s * chiL + a) * chiR + ap];
    sv[s * MAXCHI + ap] = acc;
  }
  __syncthreads();
  const int rb = pick(ds.rid, cur)[b];
  const T* Rj = bt.R + ((size_t)rb * (cols + 1) + (j + 1)) * chi * rs;
  for (int e = tid; e < p * NR; e += nt) {
    const int s = e / NR, rr = e % NR;
    const int col = rr * Gout + gu;
    T acc = T(0);
    for (int ap = 0; ap < chiR; ++ap) acc += sv[s * MAXCHI + ap] * Rj[(size_t)ap * rs + col];
    sZ[s * MAXP + rr] = (double)acc;
  }
  const size_t so = (size_t)site * dm;
  const double* bLl = wd.bL + (size_t)site * tb.lstride + (size_t)l * MAXP;
  const double* bUu = wd.bU + (size_t)site * 256 + u * 16;
  __syncthreads();
  const int d = tb.d[site];
  // the weights once (each thread keeps its own states' in shared memory)
  __shared__ double sq[MAXS];
  double part = 0.0;
  for (int x = tid; x < d; x += nt) {
    double q = wd.w[so + x] * bLl[tb.PL[so + x]] * bUu[tb.PU[so + x]] * sZ[tb.PD[so + x] * MAXP + tb.PR[so + x]];
    q = q > 0.0 ? q : 0.0;
    sq[x] = q;
    part += q;
  }
  const double tot = block_sum(part, red);
  const double lt = log(tot);
  const int64_t E0 = pick(ds.E, cur)[b];
  const int64_t* RLl = tb.RL + (size_t)site * tb.lstride + (size_t)l * MAXP;
  const int64_t* RUu = tb.RU + (size_t)site * 256 + u * 16;
  for (int x = tid; x < d; x += nt) {
    const int pl = tb.PL[so + x], pu = tb.PU[so + x], pr = tb.PR[so + x];
    const double q = sq[x];
    const double lc = (tot > 0.0) ? (q > 0.0 ? log_pos<T>(q) - lt : -INFINITY) : -INFINITY;
    ds.logc[(size_t)b * ds.dmax + x] = lc;
    int64_t e = E0 + tb.E[so + x] + RLl[pl] + RUu[pu];
    if (adr) e += tb.RA[(size_t)(site + 1) * 256 + pr * 16 + ur];
    ds.candE[(size_t)b * ds.dmax + x] = e;
  }
  if (tid == 0 && !(tot >= 0.0)) atomicOr(ds.err, ERR_NAN);
}

// The mixed mode's marginals: the same conditionals with the state weights
// formed in FP32 and the normalisation in FP64.  Per beam element b, as in
// k_marginals: v = lenv B_j, Z[p][r] = sum_a' v[p][a'] R[a'][r * Gout + g];
// Z is scaled to max |.| = 1 (a factor that cancels in the normalisation),
// so that the FP32 product q(x) = w(x) bL[l][PL x] bU[u][PU x] Z[PD x][PR x]
// stays in FP32's range for the states that matter (the weight factors of a
// site stay above e^-SPG_FP32_WEIGHT_SPAN, else the solve runs the FP64
// path); sum_x q(x) in FP64, logc = log q (FP32) - log sum (FP64).
// One warp per beam element, 8 per block: the block stages B_j's site once
// (when it fits), each warp works without block barriers (its reductions
// are shuffles), so a block's elements proceed independently.
constexpr int MW = 8;  // beam elements (warps) per block
__global__ void __launch_bounds__(256) k_marginals_f32(DevTables tb, DevWeights<float> wt, DevMPS<float> mps,
                                                      int site, DevSearch ds, DevBeamT<float> bt, int cur,
                                                      int staged, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  mps = zp(mps, zs);
  ds = zp(ds, zs);
  bt = zp(bt, zs);
  const int nb = ds.n_beam[cur];
  const int b0 = blockIdx.x * MW;
  if (b0 >= nb) return;
  // dynamic shared memory: the staged site (staged: p chiL chiR floats),
  // then per warp v [MAXP][chi] and the environment columns [chi][MAXP]
  extern __shared__ __align__(16) float smk[];
  __shared__ float sl[MW][MAXCHI];
  __shared__ float sZ[MW][MAXP * MAXP];
  const int cols = tb.cols, chi = bt.chi, rs = bt.rs;
  const int i = site / cols, j = site % cols;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int* dA = mps.dimA + ((i + 1) * cols + j) * 3;
  const int p = dA[0], chiL = dA[1], chiR = dA[2];
  const float* A = mps.A + (size_t)((i + 1) * cols + j) * mps.site_stride;
  if (staged) {
    for (int e = tid; e < p * chiL * chiR; e += 256) smk[e] = A[e];
    __syncthreads();
  }
  // `staged` is the site's slot in floats (0: read from global memory)
  const float* Ar = staged ? smk : A;
  const size_t wbuf = (size_t)MAXP * bt.chi;  // floats of one warp's v (and of its environment columns)
  float* svw = smk + (staged ? (size_t)staged : 0) + (size_t)w * 2 * wbuf;
  float* srw = svw + wbuf;
  const int b = b0 + w;
  if (b >= nb) return;  // after the only block barrier
  const int NR = dim_of(tb, site, D_NR), Gin = dim_of(tb, site, D_GIN), Gout = dim_of(tb, site, D_GOUT);
  const size_t dm = tb.dmax;
  const uint16_t* stb = pick(ds.states, cur) + (size_t)b * ds.N;
  const int a_l = j > 0 ? tb.PR[(size_t)(site - 1) * dm + stb[site - 1]] : 0;
  const int g_l = (j > 0 && i > 0) ? tb.PG[(size_t)(site - cols - 1) * dm + stb[site - cols - 1]] : 0;
  const int l = a_l * Gin + g_l;
  const int u = i > 0 ? tb.PD[(size_t)(site - cols) * dm + stb[site - cols]] : 0;
  const int gu = i > 0 ? tb.gD[(size_t)(site - cols) * MAXP + u] : 0;
  const bool adr = i > 0 && j + 1 < cols;
  const int ur = adr ? tb.PD[(size_t)(site - cols + 1) * dm + stb[site - cols + 1]] : 0;
  for (int a = lane; a < chiL; a += 32) sl[w][a] = pick(bt.lenv, cur)[(size_t)b * chi + a];
  __syncwarp();
  // the environment columns the element reads, R[a'][r * Gout + g] for
  // r < NR, staged (coalesced over r) while v is formed
  const int rb = pick(ds.rid, cur)[b];
  const float* Rj = bt.R + ((size_t)rb * (cols + 1) + (j + 1)) * chi * rs;
  for (int e = lane; e < chiR * NR; e += 32) srw[e] = Rj[(size_t)(e / NR) * rs + (e % NR) * Gout + gu];
  // v[p][a'] = sum_a lenv[a] B[p][a][a'], four outputs per lane at a time
  // (each sums over a in order)
  const int nv = p * chiR;
  for (int e0 = lane; e0 < nv; e0 += 128) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const float* ap4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = min(e0 + 32 * t, nv - 1);
      ap4[t] = Ar + (size_t)(e / chiR) * chiL * chiR + e % chiR;
    }
    for (int a = 0; a < chiL; ++a) {
      const float la = sl[w][a];
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t] += la * ap4[t][(size_t)a * chiR];
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = e0 + 32 * t;
      if (e < nv) svw[(e / chiR) * chi + e % chiR] = acc[t];
    }
  }
  __syncwarp();
  float zmx = 0.f;
  const int nz = p * NR;
  for (int e0 = lane; e0 < nz; e0 += 128) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int sp4[4], rr4[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = min(e0 + 32 * t, nz - 1);
      sp4[t] = e / NR;
      rr4[t] = e % NR;
    }
    for (int ap = 0; ap < chiR; ++ap)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t] += svw[sp4[t] * chi + ap] * srw[ap * NR + rr4[t]];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = e0 + 32 * t;
      if (e < nz) {
        sZ[w][sp4[t] * MAXP + rr4[t]] = acc[t];
        zmx = fmaxf(zmx, fabsf(acc[t]));
      }
    }
  }
  zmx = warp_max(zmx);
  __syncwarp();
  const float zin = zmx > 0.f ? 1.f / zmx : 0.f;
  const size_t so = (size_t)site * dm;
  const float* bLl = wt.bL + (size_t)site * tb.lstride + (size_t)l * MAXP;
  const float* bUu = wt.bU + (size_t)site * 256 + u * 16;
  const int d = tb.d[site];
  float q[MAXS / 32];
  double part = 0.0;
#pragma unroll
  for (int k = 0; k < MAXS / 32; ++k) {
    const int x = lane + 32 * k;
    float v = 0.f;
    if (x < d) {
      v = wt.w[so + x] * bLl[tb.PL[so + x]] * bUu[tb.PU[so + x]] * (sZ[w][tb.PD[so + x] * MAXP + tb.PR[so + x]] * zin);
      v = v > 0.f ? v : 0.f;
    }
    q[k] = v;
    part += (double)v;
  }
  const double tot = warp_sum(part);
  const double lt = log(tot);
  const int64_t E0 = pick(ds.E, cur)[b];
  const int64_t* RLl = tb.RL + (size_t)site * tb.lstride + (size_t)l * MAXP;
  const int64_t* RUu = tb.RU + (size_t)site * 256 + u * 16;
#pragma unroll
  for (int k = 0; k < MAXS / 32; ++k) {
    const int x = lane + 32 * k;
    if (x < d) {
      const int pl = tb.PL[so + x], pu = tb.PU[so + x], pr = tb.PR[so + x];
      const double lc = (tot > 0.0) ? (q[k] > 0.f ? (double)logf(q[k]) - lt : -INFINITY) : -INFINITY;
      ds.logc[(size_t)b * ds.dmax + x] = lc;
      int64_t e = E0 + tb.E[so + x] + RLl[pl] + RUu[pu];
      if (adr) e += tb.RA[(size_t)(site + 1) * 256 + pr * 16 + ur];
      ds.candE[(size_t)b * ds.dmax + x] = e;
    }
  }
  if (lane == 0 && !(tot >= 0.0)) atomicOr(ds.err, ERR_NAN);
}

// ---------------------------------------------------------------- S7 merge
// Classes of equal reduced parent keys by open addressing.  The reduced
// parent key of element b: states (packed `bits` each) of the key sites at
// this step other than the current site.  Every beam element writes its key,
// then inserts it into a table of hsize (a power of two >= 2 cap) slots (slot
// = owner index + 1, 0 empty), joining the slot whose owner has the same key
// (an owner's key is written before its slot is claimed, and read past the
// L1 cache); the representative of a class is the lowest index of the slot's
// members (atomicMin), which is the class's lowest lex rank.  The slot of
// element b is kept in nxt[b].  Table and minima are reset by the launcher
// (byte memsets).

__device__ __forceinline__ unsigned key_hash(const unsigned long long* k) {
  unsigned long long h = 0x9e3779b97f4a7c15ull;
  for (int w = 0; w < KEYW; ++w) {
    h ^= k[w] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    h *= 0xff51afd7ed558ccdull;
  }
  return (unsigned)(h ^ (h >> 32));
}

__global__ void k_class_insert(DevTables tb, int site, DevSearch ds, int cur, int merge, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = ds.n_beam[cur];
  if (b >= nb) return;
  if (!merge) {
    ds.nxt[b] = -1;
    return;
  }
  unsigned long long kb[KEYW] = {};
  const int* ks = tb.keys + site * (MAXKEY + 1);
  const int n = ks[0], bits = *tb.kshift;
  const uint16_t* stb = pick(ds.states, cur) + (size_t)b * ds.N;
  for (int q = 0; q < n; ++q) {
    const int pos = q * bits;
    const int w = pos >> 6, o = pos & 63;
    if (w < KEYW) kb[w] |= (unsigned long long)stb[ks[1 + q]] << o;
    else atomicOr(ds.err, ERR_KEY);
  }
  for (int w = 0; w < KEYW; ++w) ds.key[(size_t)b * KEYW + w] = kb[w];
  __threadfence();
  const unsigned mask = (unsigned)ds.hsize - 1u;
  unsigned slot = key_hash(kb) & mask;
  int mine = -1;
  for (int t = 0; t < ds.hsize; ++t, slot = (slot + 1) & mask) {
    const int owner = atomicCAS(ds.htab + slot, 0, b + 1);
    if (owner == 0) {
      mine = (int)slot;
      break;
    }
    const unsigned long long* ko = ds.key + (size_t)(owner - 1) * KEYW;
    bool eq = true;
    for (int w = 0; w < KEYW; ++w) eq = eq && __ldcg(ko + w) == kb[w];
    if (eq) {
      mine = (int)slot;
      break;
    }
  }
  ds.nxt[b] = mine;  // never -1: the table has more slots than elements
  if (mine >= 0) atomicMin(ds.hmin + mine, b);
}

// For each (class representative b, x): the member with the lowest
// (candidate energy, lex rank) wins.  When the site's own state is not part
// of the key (no edge to a later site) and branches are merged, one winner
// is taken per class over all states x, lex order (member, x); without
// merging every child is its own class.  The beam is kept in lex order, so
// the lex rank of a member is its index.  Three passes over all candidates:
// the class minimum of the energy (atomicMin on its order-preserving bits),
// the lowest member (and x) reaching it, and the winner table.  wmin is
// reset to all ones and win / wkey to WIN_NONE (byte memsets) before.
constexpr int WIN_NONE = 0x7f7f7f7f;

__global__ void k_win_min(DevTables tb, int site, DevSearch ds, int cur, int merge, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  const int nb = ds.n_beam[cur];
  const int d = tb.d[site];
  const bool xin = !merge || tb.dims[site * DIMW + D_XIN] != 0;  // without merging every child is its own class
  const size_t tot = (size_t)nb * ds.dmax;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(c / ds.dmax), x = (int)(c % ds.dmax);
    if (x >= d) continue;
    // the class representative (the lowest member of the element's slot)
    const int slot = ds.nxt[b];
    const int r = (merge && slot >= 0) ? ds.hmin[slot] : b;
    if (x == 0) ds.rep[b] = r;
    atomicMin(&ds.wmin[(size_t)r * ds.dmax + (xin ? x : 0)], ord_i64(ds.candE[c]));
  }
}

__global__ void k_win_arg(DevTables tb, int site, DevSearch ds, int cur, int merge, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  const int nb = ds.n_beam[cur];
  const int d = tb.d[site];
  const bool xin = !merge || tb.dims[site * DIMW + D_XIN] != 0;  // without merging every child is its own class
  const size_t tot = (size_t)nb * ds.dmax;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(c / ds.dmax), x = (int)(c % ds.dmax);
    if (x >= d) continue;
    const int r = ds.rep[b];
    if (ord_i64(ds.candE[c]) != ds.wmin[(size_t)r * ds.dmax + (xin ? x : 0)]) continue;
    if (xin)
      atomicMin(&ds.win[(size_t)r * ds.dmax + x], b);
    else
      atomicMin(&ds.wkey[r], (int)c);
  }
}

__global__ void k_win_fix(DevTables tb, int site, DevSearch ds, int cur, int merge, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  const int nb = ds.n_beam[cur];
  const int d = tb.d[site];
  const bool xin = !merge || tb.dims[site * DIMW + D_XIN] != 0;  // without merging every child is its own class
  const size_t tot = (size_t)ds.cap * ds.dmax;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(c / ds.dmax), x = (int)(c % ds.dmax);
    int w = -1;
    if (b < nb && x < d && ds.rep[b] == b) {
      if (xin) {
        const int v = ds.win[c];
        w = v != WIN_NONE ? v : -1;
      } else {
        const int k = ds.wkey[b];
        if (k != WIN_NONE && k % ds.dmax == x) w = k / ds.dmax;
      }
    }
    ds.win[c] = w;
  }
}

// ---------------------------------------------------------------- S7 prune: radix select
// Composite key of candidate c = b*dmax + x (ascending order = rank order):
//   k0 = ~ord(log p), k1 = ord(E), k2 = (winner << 16) | x.
// sel_state words: 0..2 prefix, 3 need, 4 status (0 running, 1 done), 5
// pass, 6 max logp key, 7 min selected logp key, 8 max rejected logp key,
// 9 log cut offset (as double bits, +inf when off), 10 total valid.
struct CandKey {
  unsigned long long k[3];
  bool valid;
  double lp;
};

__device__ __forceinline__ CandKey cand_key(const DevSearch& ds, int cur, size_t c, int nb, int d,
                                            double log_cut, unsigned long long maxkey) {
  CandKey r;
  r.valid = false;
  const int b = (int)(c / ds.dmax), x = (int)(c % ds.dmax);
  if (b >= nb || x >= d) return r;
  const int w = ds.win[c];
  if (w < 0) return r;
  const double lp = pick(ds.logp, cur)[w] + ds.logc[(size_t)w * ds.dmax + x];
  if (log_cut > -INFINITY) {
    const double mx = unord_f64(maxkey);
    if (!(lp >= mx + log_cut)) return r;
  }
  r.valid = true;
  r.lp = lp;
  r.k[0] = ~ord_f64(lp);
  r.k[1] = ord_i64(ds.candE[(size_t)w * ds.dmax + x]);
  r.k[2] = ((unsigned long long)w << 16) | (unsigned long long)x;
  return r;
}

__global__ void __launch_bounds__(1024) k_logp_max(DevTables tb, int site, DevSearch ds, int cur, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  const int nb = ds.n_beam[cur], d = tb.d[site];
  const size_t tot = (size_t)ds.cap * ds.dmax;
  unsigned long long best = 0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < tot; c += (size_t)gridDim.x * blockDim.x) {
    CandKey k = cand_key(ds, cur, c, nb, d, -INFINITY, 0);
    if (k.valid) best = max(best, ord_f64(k.lp));
  }
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best) atomicMax(ds.sel_state + 6, best);
}

// Selection state of a fresh prune step (one thread); the histogram is
// zeroed once per solve (k_reset_beam) and by the last block of every pass.
__device__ __forceinline__ void select_state_reset(const DevSearch& ds) {
  ds.sel_state[0] = ds.sel_state[1] = ds.sel_state[2] = 0;
  ds.sel_state[3] = (unsigned long long)ds.cap;
  ds.sel_state[4] = 0;
  ds.sel_state[5] = 0;
  ds.sel_state[6] = 0;
  ds.sel_state[7] = ~0ull;
  ds.sel_state[8] = 0;
  ds.sel_state[10] = 0;
  *ds.sel_count = 0;
  *ds.pend_n = 0;
  *ds.done_ctr = 0;
}

__device__ __forceinline__ bool prefix_match(const CandKey& k, const unsigned long long* pre, int pass) {
  // bits determined before this pass: 16*pass of the 192-bit key
  const int full = pass >> 2, part = (pass & 3) * 16;
  for (int w = 0; w < full; ++w)
    if (k.k[w] != pre[w]) return false;
  if (part > 0) {
    const unsigned long long m = ~0ull << (64 - part);
    if ((k.k[full] & m) != (pre[full] & m)) return false;
  }
  return true;
}

// One radix pass: histogram of the 16-bit digit `pass` of the keys that
// match the prefix chosen so far, over all candidates (list == nullptr) or
// over the candidate ids list[0 .. *list_n).
__global__ void __launch_bounds__(1024) k_select_pass(DevTables tb, int site, DevSearch ds, int cur, int pass, double log_cut,
                              const int* list, const int* list_n, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  list = zp(list, zs);
  list_n = zp(list_n, zs);
  __shared__ bool s_last;
  const unsigned long long status = ds.sel_state[4];
  if (status != 0) return;
  const int nb = ds.n_beam[cur], d = tb.d[site];
  const size_t tot = list ? (size_t)*list_n : (size_t)ds.cap * ds.dmax;
  unsigned long long pre[3] = {ds.sel_state[0], ds.sel_state[1], ds.sel_state[2]};
  const unsigned long long maxkey = ds.sel_state[6];
  const int w = pass >> 2, sh = 48 - (pass & 3) * 16;
  // every lane runs the same number of iterations so that the warp-wide
  // match below sees all 32 lanes; lanes with the same digit add once
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t c0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t iters = (tot + stride - 1) / stride;
  const int lane = threadIdx.x & 31;
  for (size_t it = 0; it < iters; ++it) {
    const size_t i = c0 + it * stride;
    int digit = -1;
    if (i < tot) {
      const size_t c = list ? (size_t)list[i] : i;
      CandKey k = cand_key(ds, cur, c, nb, d, log_cut, maxkey);
      if (k.valid && prefix_match(k, pre, pass)) digit = (int)((k.k[w] >> sh) & 0xffff);
    }
    const unsigned same = __match_any_sync(0xffffffffu, digit);
    if (digit >= 0 && lane == __ffs(same) - 1) atomicAdd(ds.hist + digit, (unsigned)__popc(same));
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ds.done_ctr, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: scan the histogram, pick the digit holding the need-th key.
  // part[t] = keys in digits [64 t, 64 t + 64); an inclusive block scan of
  // part finds the group, one warp's scan of its 64 digits the digit.
  __shared__ unsigned long long part[1024];
  __shared__ unsigned long long wsum[32];
  __shared__ int s_group, s_dig;
  __shared__ unsigned long long s_before;
  const int tid = threadIdx.x, nt = blockDim.x;  // nt == 1024
  const int per = 65536 / nt;
  const int wid = tid >> 5;
  unsigned long long loc = 0;
  for (int q = 0; q < per; ++q) loc += ((volatile unsigned*)ds.hist)[tid * per + q];
  // inclusive scan: within the warp, then over the 32 warp totals
  unsigned long long inc = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    unsigned long long v = wsum[lane], x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    wsum[lane] = x - v;  // exclusive prefix of the warps
  }
  __syncthreads();
  inc += wsum[wid];
  part[tid] = inc;
  const unsigned long long need0 = ds.sel_state[3];
  if (tid == 0) s_group = nt - 1;
  __syncthreads();
  // the first group whose inclusive count reaches need
  if (inc >= need0 && (tid == 0 || part[tid - 1] < need0)) s_group = tid;
  __syncthreads();
  const int t = s_group;
  if (wid == 0) {
    // digits 64 t .. 64 t + 63, two per lane
    const unsigned long long before = t > 0 ? part[t - 1] : 0ull;
    const unsigned a = ((volatile unsigned*)ds.hist)[t * per + 2 * lane];
    const unsigned b = ((volatile unsigned*)ds.hist)[t * per + 2 * lane + 1];
    unsigned long long x = (unsigned long long)a + b, xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    const unsigned long long ex = before + xi - x;  // keys in digits before 2 lane
    // digit 2 lane reaches need if ex + a >= need, else 2 lane + 1 if ex + a + b >= need
    int cand = 1 << 30;
    if (ex + a >= need0) cand = 2 * lane;
    else if (ex + a + b >= need0) cand = 2 * lane + 1;
    int best = cand;
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) s_dig = best >= (1 << 30) ? per - 1 : best;  // the last digit of the group if counts were short
    // count of keys before the chosen digit
    const int dsel = __shfl_sync(0xffffffffu, best >= (1 << 30) ? per - 1 : best, 0);
    unsigned long long mine = 0;
    if (2 * lane < dsel) mine += a;
    if (2 * lane + 1 < dsel) mine += b;
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0) s_before = before + mine;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long need = need0;
    const unsigned long long total = part[nt - 1];
    if (pass == 0) ds.sel_state[10] = total;
    if (pass == 0 && total <= need) {
      ds.sel_state[0] = ds.sel_state[1] = ds.sel_state[2] = ~0ull;  // select all valid
      ds.sel_state[4] = 1;
    } else {
      const int digit = t * per + s_dig;
      const unsigned long long cum = s_before;
      const unsigned long long hv = ((volatile unsigned*)ds.hist)[digit];
      need = need > cum ? need - cum : 1;
      ds.sel_state[w] |= (unsigned long long)digit << sh;
      ds.sel_state[3] = need;
      if (hv == need || pass == 11) {
        // every key matching the prefix up to here is selected: fill the rest with ones
        if (sh > 0) ds.sel_state[w] |= (1ull << sh) - 1ull;
        for (int q = w + 1; q < 3; ++q) ds.sel_state[q] = ~0ull;
        ds.sel_state[4] = 1;
      }
    }
    ds.sel_state[5] = pass + 1;
    *ds.done_ctr = 0;
  }
  __syncthreads();
  for (int e = tid; e < 65536; e += nt) ds.hist[e] = 0;
}

__device__ __forceinline__ bool key_le(const CandKey& k, const unsigned long long* t) {
  if (k.k[0] != t[0]) return k.k[0] < t[0];
  if (k.k[1] != t[1]) return k.k[1] < t[1];
  return k.k[2] <= t[2];
}

// Candidates (all, or the ids list[0 .. *list_n)) against the selection:
// with split set and the selection still open after the first pass, the
// top digit decides (below the chosen digit: selected, equal: pending for
// the later passes, above: rejected); otherwise the full threshold key
// decides (key <= threshold: selected).  Selected ids go to sel_list,
// pending ones to pend; the extremes of the selected and rejected log p feed
// the near-tie test.
__global__ void __launch_bounds__(1024) k_select_classify(DevTables tb, int site, DevSearch ds, int cur, double log_cut, const int* list,
                                  const int* list_n, int split, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  list = zp(list, zs);
  list_n = zp(list_n, zs);
  if (!split && ds.sel_state[4] == 2) return;  // resolved by k_select_refine
  const int nb = ds.n_beam[cur], d = tb.d[site];
  const size_t tot = list ? (size_t)*list_n : (size_t)ds.cap * ds.dmax;
  const unsigned long long thr[3] = {ds.sel_state[0], ds.sel_state[1], ds.sel_state[2]};
  const unsigned long long maxkey = ds.sel_state[6];
  const bool by_digit = split && ds.sel_state[4] == 0;
  const unsigned long long d0 = thr[0] >> 48;
  unsigned long long min_sel = ~0ull, max_rej = 0ull;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t c0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  // every lane runs the same number of iterations so that the warp-wide
  // ballots below see all 32 lanes
  const size_t iters = (tot + stride - 1) / stride;
  const int lane = threadIdx.x & 31;
  for (size_t it = 0; it < iters; ++it) {
    const size_t i = c0 + it * stride;
    bool take = false, pend = false;
    size_t c = 0;
    if (i < tot) {
      c = list ? (size_t)list[i] : i;
      CandKey k = cand_key(ds, cur, c, nb, d, log_cut, maxkey);
      if (k.valid) {
        if (by_digit) {
          const unsigned long long dg = k.k[0] >> 48;
          take = dg < d0;
          pend = dg == d0;
        } else {
          take = key_le(k, thr);
        }
        if (take)
          min_sel = min(min_sel, ord_f64(k.lp));
        else if (!pend)
          max_rej = max(max_rej, ord_f64(k.lp) + 1ull);  // +1 keeps 0 = "none"
      }
    }
    const unsigned mt = __ballot_sync(0xffffffffu, take);
    if (mt) {
      int base = 0;
      if (lane == 0) base = atomicAdd(ds.sel_count, __popc(mt));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (take) {
        const int pos = base + __popc(mt & ((1u << lane) - 1u));
        if (pos < ds.cap) ds.sel_list[pos] = (int)c;
      }
    }
    const unsigned mp = __ballot_sync(0xffffffffu, pend);
    if (mp) {
      int base = 0;
      if (lane == 0) base = atomicAdd(ds.pend_n, __popc(mp));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (pend) ds.pend[base + __popc(mp & ((1u << lane) - 1u))] = (int)c;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    min_sel = min(min_sel, __shfl_xor_sync(0xffffffffu, min_sel, o));
    max_rej = max(max_rej, __shfl_xor_sync(0xffffffffu, max_rej, o));
  }
  if (lane == 0) {
    if (min_sel != ~0ull) atomicMin(ds.sel_state + 7, min_sel);
    if (max_rej != 0ull) atomicMax(ds.sel_state + 8, max_rej);
  }
}

// The pending candidates (those sharing the top digit chosen by the first
// pass) resolved in one block: 8-bit radix rounds over the rest of the key
// (histograms in shared memory, keys recomputed from the candidate arrays),
// then the pending ids up to the final threshold appended to sel_list.  The
// selection is marked resolved (state 2).
__global__ void __launch_bounds__(1024) k_select_refine(DevTables tb, int site, DevSearch ds, int cur, double log_cut, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  __shared__ unsigned hist[256];
  __shared__ unsigned long long s_pre[3];
  __shared__ unsigned long long s_need;
  __shared__ int s_done, s_base;
  __shared__ unsigned long long s_min, s_max;
  if (ds.sel_state[4] != 0) return;
  const int n = *ds.pend_n;
  const int nb = ds.n_beam[cur], d = tb.d[site];
  const unsigned long long maxkey = ds.sel_state[6];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  if (tid == 0) {
    s_pre[0] = ds.sel_state[0];
    s_pre[1] = ds.sel_state[1];
    s_pre[2] = ds.sel_state[2];
    s_need = ds.sel_state[3];
    s_done = 0;
    s_min = ~0ull;
    s_max = 0ull;
  }
  __syncthreads();
  // bits fixed so far: 16 (the first pass); round r fixes 8 more
  for (int fixed = 16; fixed < 192 && !s_done; fixed += 8) {
    for (int e = tid; e < 256; e += nt) hist[e] = 0u;
    __syncthreads();
    const int w = fixed >> 6, sh = 56 - (fixed & 63);
    const unsigned long long pre0 = s_pre[0], pre1 = s_pre[1], pre2 = s_pre[2];
    for (int i = tid; i < n; i += nt) {
      const CandKey k = cand_key(ds, cur, (size_t)ds.pend[i], nb, d, log_cut, maxkey);
      if (!k.valid) continue;
      // the key's bits above this digit must equal the prefix
      bool match = true;
      const unsigned long long pre[3] = {pre0, pre1, pre2};
      for (int q = 0; q < w; ++q) match = match && k.k[q] == pre[q];
      const unsigned long long m = (fixed & 63) ? (~0ull << (64 - (fixed & 63))) : 0ull;
      match = match && ((k.k[w] & m) == (pre[w] & m));
      if (match) atomicAdd(&hist[(k.k[w] >> sh) & 0xff], 1u);
    }
    __syncthreads();
    if (tid < 32) {
      // inclusive scan of the 256 bins, 8 per lane
      unsigned loc[8];
      unsigned sum = 0;
      for (int q = 0; q < 8; ++q) {
        loc[q] = hist[lane * 8 + q];
        sum += loc[q];
      }
      unsigned incl = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      unsigned long long cum = incl - sum;  // keys in the digits before this lane's first
      const unsigned long long need = s_need;
      int digit = 1 << 30;
      unsigned long long before = 0, hv = 0;
      for (int q = 0; q < 8; ++q) {
        if (digit == (1 << 30) && cum + loc[q] >= need) {
          digit = lane * 8 + q;
          before = cum;
          hv = loc[q];
        }
        cum += loc[q];
      }
      // the lowest lane that found the digit publishes it
      const unsigned found = __ballot_sync(0xffffffffu, digit != (1 << 30));
      const int src = found ? __ffs(found) - 1 : 31;
      digit = __shfl_sync(0xffffffffu, digit, src);
      before = __shfl_sync(0xffffffffu, before, src);
      hv = __shfl_sync(0xffffffffu, hv, src);
      if (lane == 0) {
        if (!found) digit = 255;  // cannot happen while the counts are consistent
        s_pre[w] |= (unsigned long long)digit << sh;
        const unsigned long long nn = need > before ? need - before : 1ull;
        s_need = nn;
        if (hv == nn || fixed + 8 >= 192) {
          if (sh > 0) s_pre[w] |= (1ull << sh) - 1ull;
          for (int q = w + 1; q < 3; ++q) s_pre[q] = ~0ull;
          s_done = 1;
        }
      }
    }
    __syncthreads();
  }
  // classify the pending ids against the final threshold
  const unsigned long long thr[3] = {s_pre[0], s_pre[1], s_pre[2]};
  if (tid == 0) s_base = 0;
  __syncthreads();
  unsigned long long mn = ~0ull, mx = 0ull;
  for (int i0 = 0; i0 < n; i0 += nt) {
    const int i = i0 + tid;
    bool take = false;
    int c = 0;
    if (i < n) {
      c = ds.pend[i];
      const CandKey k = cand_key(ds, cur, (size_t)c, nb, d, log_cut, maxkey);
      if (k.valid) {
        take = key_le(k, thr);
        if (take)
          mn = min(mn, ord_f64(k.lp));
        else
          mx = max(mx, ord_f64(k.lp) + 1ull);
      }
    }
    const unsigned msk = __ballot_sync(0xffffffffu, take);
    int base = 0;
    if (lane == 0 && msk) base = atomicAdd(&s_base, __popc(msk));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (take) {
      const int pos = *ds.sel_count + base + __popc(msk & ((1u << lane) - 1u));
      if (pos < ds.cap) ds.sel_list[pos] = c;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    if (mn != ~0ull) atomicMin(&s_min, mn);
    if (mx != 0ull) atomicMax(&s_max, mx);
  }
  __syncthreads();
  if (tid == 0) {
    *ds.sel_count += s_base;
    if (s_min != ~0ull) atomicMin(ds.sel_state + 7, s_min);
    if (s_max != 0ull) atomicMax(ds.sel_state + 8, s_max);
    ds.sel_state[0] = thr[0];
    ds.sel_state[1] = thr[1];
    ds.sel_state[2] = thr[2];
    ds.sel_state[4] = 2;
  }
}

// One block: sort the selected ids by lex key (winner, x); record near ties.
__global__ void __launch_bounds__(1024) k_select_sort(DevTables tb, int site, DevSearch ds, int cur, int nxt_buf, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  extern __shared__ unsigned long long sk[];  // [pow2 >= cap]
  const int n = min(*ds.sel_count, ds.cap);
  int P = 1;
  while (P < n) P <<= 1;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    unsigned long long v = ~0ull;
    if (e < n) {
      const int c = ds.sel_list[e];
      const int x = c % ds.dmax;
      const int w = ds.win[c];
      v = ((unsigned long long)w << 40) | ((unsigned long long)x << 24) | (unsigned long long)e;
    }
    sk[e] = v;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int e = threadIdx.x; e < P; e += blockDim.x) {
        const int o = e ^ jj;
        if (o > e) {
          const bool up = (e & k) == 0;
          const unsigned long long a = sk[e], b = sk[o];
          if ((a > b) == up) {
            sk[e] = b;
            sk[o] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  // rewrite sel_list in lex order (through the original slot index in the low bits)
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int slot = (int)(sk[e] & 0xffffffull);
    sk[e] = (unsigned long long)ds.sel_list[slot];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) ds.sel_list[e] = (int)sk[e];
  if (threadIdx.x == 0) {
    ds.n_beam[nxt_buf] = n;
    *ds.candidates += (double)ds.n_beam[cur] * (double)tb.d[site];
    const unsigned long long rj = ds.sel_state[8];
    if (rj != 0 && n > 0) {
      const double a = unord_f64(ds.sel_state[7]);
      const double bb = unord_f64(rj - 1ull);
      if (fabs(a - bb) <= 1e-9 * fmax(1.0, fabs(a))) atomicAdd(ds.near_ties, 1);
    }
    select_state_reset(ds);  // for the next site's prune
  }
}

// ---------------------------------------------------------------- update
// New beam element i from selected candidate c = rep*dmax + x with parent w.
template <typename T>
__global__ void k_update(DevTables tb, DevMPS<T> mps, int site, DevSearch ds, DevBeamT<T> bt, int cur, size_t zs) {
  tb = zp(tb, zs);
  mps = zp(mps, zs);
  ds = zp(ds, zs);
  bt = zp(bt, zs);
  const int i = blockIdx.x;
  const int nxt = cur ^ 1;
  if (i >= ds.n_beam[nxt]) return;
  __shared__ T red[32];
  const int c = ds.sel_list[i];
  const int x = c % ds.dmax;
  const int w = ds.win[c];
  const int N = ds.N;
  for (int q = threadIdx.x; q < N; q += blockDim.x)
    pick(ds.states, nxt)[(size_t)i * N + q] = q == site ? (uint16_t)x : pick(ds.states, cur)[(size_t)w * N + q];
  if (threadIdx.x == 0) {
    pick(ds.E, nxt)[i] = ds.candE[(size_t)w * ds.dmax + x];
    pick(ds.logp, nxt)[i] = pick(ds.logp, cur)[w] + ds.logc[(size_t)w * ds.dmax + x];
    pick(ds.rid, nxt)[i] = pick(ds.rid, cur)[w];
  }
  const int cols = tb.cols, chi = bt.chi;
  const int r = site / cols, j = site % cols;
  const int* dA = mps.dimA + ((r + 1) * cols + j) * 3;
  const int chiL = dA[1], chiR = dA[2];
  const T* A = mps.A + (size_t)((r + 1) * cols + j) * mps.site_stride;
  const int pd = tb.PD[(size_t)site * tb.dmax + x];
  const T* lw = pick(bt.lenv, cur) + (size_t)w * chi;
  T mx = T(0);
  T v = T(0);
  const int ap = threadIdx.x;
  if (ap < chiR) {
    for (int a = 0; a < chiL; ++a) v += lw[a] * A[((size_t)pd * chiL + a) * chiR + ap];
    mx = (T)fabs((double)v);
  }
  mx = block_max(mx, red);
  const T inv = mx > T(0) ? T(1) / mx : T(0);
  if (ap < chi) pick(bt.lenv, nxt)[(size_t)i * chi + ap] = ap < chiR ? v * inv : T(0);
}

// lenv of teacher-forced prefixes: prod_{k<j} B_{i+1}[k][:, PD x_k, :], scaled.
template <typename T>
__global__ void k_lenv_prefix(DevTables tb, DevMPS<T> mps, int site, DevSearch ds, DevBeamT<T> bt, int cur) {
  const int b = blockIdx.x;
  if (b >= ds.n_beam[cur]) return;
  __shared__ T v[MAXCHI], nv[MAXCHI], red[32];
  const int cols = tb.cols, chi = bt.chi;
  const int r = site / cols, j = site % cols;
  const uint16_t* stb = pick(ds.states, cur) + (size_t)b * ds.N;
  if (threadIdx.x < MAXCHI) v[threadIdx.x] = threadIdx.x == 0 ? T(1) : T(0);
  __syncthreads();
  for (int k = 0; k < j; ++k) {
    const int s = r * cols + k;
    const int* dA = mps.dimA + ((r + 1) * cols + k) * 3;
    const int chiL = dA[1], chiR = dA[2];
    const T* A = mps.A + (size_t)((r + 1) * cols + k) * mps.site_stride;
    const int pd = tb.PD[(size_t)s * tb.dmax + stb[s]];
    T val = T(0);
    if (threadIdx.x < chiR)
      for (int a = 0; a < chiL; ++a) val += v[a] * A[((size_t)pd * chiL + a) * chiR + threadIdx.x];
    T mx = block_max(threadIdx.x < chiR ? (T)fabs((double)val) : T(0), red);
    __syncthreads();
    if (threadIdx.x < MAXCHI) nv[threadIdx.x] = threadIdx.x < chiR ? val / mx : T(0);
    __syncthreads();
    if (threadIdx.x < MAXCHI) v[threadIdx.x] = nv[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x < chi) pick(bt.lenv, cur)[(size_t)b * chi + threadIdx.x] = v[threadIdx.x];
}

__global__ void k_reset_beam(DevSearch ds, int cur, size_t zs) {
  ds = zp(ds, zs);
  for (int e = threadIdx.x; e < 65536; e += blockDim.x) ds.hist[e] = 0;
  if (threadIdx.x == 0) {
    select_state_reset(ds);
    if (pick(ds.dn, cur)) pick(ds.dn, cur)[0] = 0;
    if (ds.dflow) *ds.dflow = 0;
    ds.n_beam[cur] = 1;
    pick(ds.E, cur)[0] = 0;
    pick(ds.logp, cur)[0] = 0.0;
    pick(ds.rid, cur)[0] = 0;
    *ds.near_ties = 0;
    *ds.err = 0;
    *ds.candidates = 0.0;
  }
  for (int q = threadIdx.x; q < ds.N; q += blockDim.x) pick(ds.states, cur)[q] = 0;
}

// ---------------------------------------------------------------- droplets
// One block per new beam element i (buffer nxt = cur ^ 1), after the prune of
// `site` (sel_list in its final order).  Its winner w (parent) and state x,
// the merge class rep b (c = b * dmax + x); members b' of the class have
// rep[b'] == b, their candidates (b', x') with x' == x when the site's state
// is part of the key, any x' otherwise.
__device__ __forceinline__ const uint16_t* drop_row(const DevSearch& ds, int cur, int b, int k) {
  return k < 0 ? pick(ds.states, cur) + (size_t)b * ds.N : pick(ds.dst, cur) + ((size_t)b * MAXDROP + k) * ds.N;
}

__global__ void k_droplets(DevTables tb, int site, DevSearch ds, int cur, int merge, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  __shared__ long long cE[MAXDCAND];
  __shared__ int cb[MAXDCAND];
  __shared__ short cx[MAXDCAND], ck[MAXDCAND];
  __shared__ int crank[MAXDCAND];
  __shared__ int s_nc, s_acc, s_ok;
  const int nxt = cur ^ 1;
  const int i = blockIdx.x;
  if (i >= ds.n_beam[nxt]) return;
  const int N = ds.N, dmax = ds.dmax, d = tb.d[site];
  const int nb = ds.n_beam[cur];
  const int c = ds.sel_list[i];
  const int x = c % dmax, brep = c / dmax;
  const int w = ds.win[c];
  const bool xin = !merge || tb.dims[site * DIMW + D_XIN] != 0;
  const int64_t Ew = ds.candE[(size_t)w * dmax + x];
  const int tid = threadIdx.x, nt = blockDim.x;
  // inherited: the winner parent's droplets, extended by x at this site
  const int nin = pick(ds.dn, cur)[w];
  uint16_t* out = pick(ds.dst, nxt) + (size_t)i * MAXDROP * N;
  for (int e = tid; e < nin * N; e += nt) {
    const int k = e / N, q = e % N;
    out[e] = q == site ? (uint16_t)x : pick(ds.dst, cur)[((size_t)w * MAXDROP + k) * N + q];
  }
  for (int k = tid; k < nin; k += nt) pick(ds.dE, nxt)[(size_t)i * MAXDROP + k] = pick(ds.dE, cur)[(size_t)w * MAXDROP + k];
  if (tid == 0) {
    s_nc = 0;
    s_acc = nin;
  }
  __syncthreads();
  // candidates within the energy cutoff
  const int nxs = xin ? 1 : d;
  for (int e = tid; e < nb * nxs; e += nt) {
    const int bp = e / nxs;
    if (ds.rep[bp] != brep) continue;
    const int xp = xin ? x : e % nxs;
    const int64_t Ep = ds.candE[(size_t)bp * dmax + xp];
    const int nd = pick(ds.dn, cur)[bp];
    for (int k = -1; k < nd; ++k) {
      if (k < 0 && bp == w && xp == x) continue;  // the winner itself
      const int64_t dE = Ep + (k < 0 ? 0 : pick(ds.dE, cur)[(size_t)bp * MAXDROP + k]) - Ew;
      if (dE > ds.dcut) continue;
      const int slot = atomicAdd(&s_nc, 1);
      if (slot < MAXDCAND) {
        cE[slot] = dE;
        cb[slot] = bp;
        cx[slot] = (short)xp;
        ck[slot] = (short)k;
      }
    }
  }
  __syncthreads();
  if (s_nc > MAXDCAND && tid == 0) atomicAdd(ds.dflow, s_nc - MAXDCAND);
  const int nc = min(s_nc, MAXDCAND);
  // rank by (dE, state over sites 0 .. site)
  for (int a = tid; a < nc; a += nt) {
    int r = 0;
    const uint16_t* ra = drop_row(ds, cur, cb[a], ck[a]);
    for (int o = 0; o < nc; ++o) {
      if (o == a) continue;
      bool less;
      if (cE[o] != cE[a]) {
        less = cE[o] < cE[a];
      } else {
        const uint16_t* ro = drop_row(ds, cur, cb[o], ck[o]);
        int cmp = 0;
        for (int q = 0; q <= site && !cmp; ++q) {
          const int va = q == site ? cx[a] : ra[q], vo = q == site ? cx[o] : ro[q];
          cmp = vo < va ? -1 : (vo > va ? 1 : 0);
        }
        less = cmp < 0 || (cmp == 0 && o < a);  // equal states: any fixed order
      }
      r += less;
    }
    crank[r] = a;
  }
  __syncthreads();
  // greedy acceptance in rank order: Hamming distance > dham from the state
  // (the winner's row with x) and from every droplet kept so far
  const uint16_t* wrow = pick(ds.states, cur) + (size_t)w * N;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int r = 0; r < nc; ++r) {
    const int a = crank[r];
    const uint16_t* ra = drop_row(ds, cur, cb[a], ck[a]);
    if (tid == 0) s_ok = 1;
    __syncthreads();
    const int nref = 1 + s_acc;  // the state, then the kept droplets
    for (int ref = wid; ref < nref; ref += nw) {
      int diff = 0;
      for (int q = lane; q <= site; q += 32) {
        const int va = q == site ? cx[a] : ra[q];
        const int vr = ref == 0 ? (q == site ? x : wrow[q]) : out[(size_t)(ref - 1) * N + q];
        diff += va != vr;
      }
      for (int o = 16; o > 0; o >>= 1) diff += __shfl_xor_sync(0xffffffffu, diff, o);
      if (lane == 0 && diff <= ds.dham) atomicAnd(&s_ok, 0);
    }
    __syncthreads();
    if (s_ok) {
      const int k = s_acc;
      if (k < MAXDROP) {
        for (int q = tid; q < N; q += nt) out[(size_t)k * N + q] = q == site ? (uint16_t)cx[a] : (q < site ? ra[q] : 0);
        if (tid == 0) pick(ds.dE, nxt)[(size_t)i * MAXDROP + k] = cE[a];
      } else if (tid == 0) {
        atomicAdd(ds.dflow, 1);
      }
      __syncthreads();
      if (tid == 0 && k < MAXDROP) s_acc = k + 1;
    }
    __syncthreads();
  }
  if (tid == 0) pick(ds.dn, nxt)[i] = s_acc;
}

// The best final state's droplets, sorted by (energy, state).
__global__ void k_final_droplets(DevSearch ds, int cur, int* out_n, int64_t* out_E, uint16_t* out_states, size_t zs) {
  ds = zp(ds, zs);
  out_n = zp(out_n, zs);
  out_E = zp(out_E, zs);
  out_states = zp(out_states, zs);
  __shared__ int s_best;
  __shared__ int rk[MAXDROP];
  const int n = ds.n_beam[cur], N = ds.N;
  if (threadIdx.x == 0) {
    int b0 = -1;
    for (int b = 0; b < n; ++b)
      if (b0 < 0 || pick(ds.E, cur)[b] < pick(ds.E, cur)[b0]) b0 = b;
    s_best = b0;
  }
  __syncthreads();
  const int b0 = s_best;
  const int nd = b0 < 0 ? 0 : pick(ds.dn, cur)[b0];
  if (threadIdx.x < nd) {
    const int a = threadIdx.x;
    const uint16_t* ra = pick(ds.dst, cur) + ((size_t)b0 * MAXDROP + a) * N;
    const int64_t Ea = pick(ds.dE, cur)[(size_t)b0 * MAXDROP + a];
    int r = 0;
    for (int o = 0; o < nd; ++o) {
      if (o == a) continue;
      const int64_t Eo = pick(ds.dE, cur)[(size_t)b0 * MAXDROP + o];
      bool less = Eo < Ea;
      if (Eo == Ea) {
        const uint16_t* ro = pick(ds.dst, cur) + ((size_t)b0 * MAXDROP + o) * N;
        int cmp = 0;
        for (int q = 0; q < N && !cmp; ++q) cmp = ro[q] < ra[q] ? -1 : (ro[q] > ra[q] ? 1 : 0);
        less = cmp < 0 || (cmp == 0 && o < a);
      }
      r += less;
    }
    rk[r] = a;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nd * N; e += blockDim.x) {
    const int r = e / N, q = e % N;
    out_states[(size_t)r * N + q] = pick(ds.dst, cur)[((size_t)b0 * MAXDROP + rk[r]) * N + q];
  }
  for (int r = threadIdx.x; r < nd; r += blockDim.x) out_E[r] = pick(ds.E, cur)[b0] + pick(ds.dE, cur)[(size_t)b0 * MAXDROP + rk[r]];
  if (threadIdx.x == 0) *out_n = nd;
}

// ---------------------------------------------------------------- forced paths
// Teacher forcing along n given full states (the per-result FP64 check):
// beam element b follows targets[b]; the search kernels compute the
// conditionals of its prefix as for any beam element, and k_force selects
// the target state as the only child (its own parent) and records that
// state's log-conditional at out[b][site].
__global__ void k_force_init(DevSearch ds, const int* n_dev, int cur) {
  const int n = min(*n_dev, ds.cap);
  const size_t N = ds.N;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ds.n_beam[cur] = n;
    *ds.near_ties = 0;
    *ds.err = 0;
    *ds.candidates = 0.0;
  }
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)n * N;
       e += (size_t)gridDim.x * blockDim.x) {
    pick(ds.states, cur)[e] = 0;
    if (e % N == 0) {
      const size_t b = e / N;
      pick(ds.E, cur)[b] = 0;
      pick(ds.logp, cur)[b] = 0.0;
      pick(ds.rid, cur)[b] = 0;
    }
  }
}

__global__ void k_force(int site, DevSearch ds, int cur, const uint16_t* __restrict__ targets,
                        double* __restrict__ out) {
  const int n = ds.n_beam[cur];
  const size_t N = ds.N;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
    const int x = targets[(size_t)b * N + site];
    const int c = b * ds.dmax + x;
    ds.sel_list[b] = c;
    ds.win[c] = b;
    out[(size_t)b * N + site] = ds.logc[c];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ds.n_beam[cur ^ 1] = n;
}

// max over b < n and sites of |a - r| / max(1, |r|) (a state's own
// conditionals in two precisions); a finite value against -inf counts as inf.
__global__ void __launch_bounds__(1024) k_logmarg_err(const double* __restrict__ a, const double* __restrict__ r, const int* n_dev,
                              int N, double* out) {
  __shared__ double red[32];
  const size_t tot = (size_t)max(0, *n_dev) * N;
  double m = 0.0;
  for (size_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const double x = a[e], y = r[e];
    double d;
    if (isinf(y) || isinf(x))
      d = (isinf(x) && isinf(y)) ? 0.0 : INFINITY;
    else
      d = fabs(x - y) / fmax(1.0, fabs(y));
    if (!(d <= m)) m = d;  // NaN propagates
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, m, o);
    if (!(t <= m)) m = t;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (!(red[w] <= v)) v = red[w];
    *out = v;
  }
}

// ---------------------------------------------------------------- S8 final
// Exact energy of each final state from the tables (checked against the
// running energy), then order by (energy, lex rank).
__global__ void __launch_bounds__(1024) k_final(DevTables tb, DevSearch ds, int cur, uint16_t* out_states, int64_t* out_E,
                        double* out_logp, int* out_n, size_t zs) {
  tb = zp(tb, zs);
  ds = zp(ds, zs);
  out_states = zp(out_states, zs);
  out_E = zp(out_E, zs);
  out_logp = zp(out_logp, zs);
  out_n = zp(out_n, zs);
  extern __shared__ unsigned long long fin_smem[];
  long long* sE = reinterpret_cast<long long*>(fin_smem);   // [SPG_MAXFINAL]
  int* rank = reinterpret_cast<int*>(sE + SPG_MAXFINAL);    // [SPG_MAXFINAL]
  const int n = min(ds.n_beam[cur], SPG_MAXFINAL);
  const int N = ds.N, cols = tb.cols;
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    const uint16_t* st = pick(ds.states, cur) + (size_t)b * N;
    int64_t E = 0;
    // every edge once: left and up-left in RL, up in RU, the anti-diagonal
    // (i-1, j)-(i, j-1) in RA (tables are zero where an edge is missing)
    for (int s = 0; s < N; ++s) {
      const size_t so = (size_t)s * tb.dmax;
      const int x = st[s];
      const int i = s / cols, j = s % cols;
      const int a = j > 0 ? tb.PR[so - tb.dmax + st[s - 1]] : 0;
      const int g = (i > 0 && j > 0) ? tb.PG[(size_t)(s - cols - 1) * tb.dmax + st[s - cols - 1]] : 0;
      const int u = i > 0 ? tb.PD[(size_t)(s - cols) * tb.dmax + st[s - cols]] : 0;
      const int l = a * tb.dims[s * DIMW + D_GIN] + g;
      E += tb.E[so + x];
      E += tb.RL[(size_t)s * tb.lstride + (size_t)l * MAXP + tb.PL[so + x]];
      E += tb.RU[(size_t)s * 256 + u * 16 + tb.PU[so + x]];
      E += tb.RA[(size_t)s * 256 + a * 16 + u];
    }
    if (E != pick(ds.E, cur)[b]) atomicOr(ds.err, ERR_ENERGY);
    sE[b] = E;
  }
  __syncthreads();
  // rank by (E, lex rank b); O(n^2) with n <= SPG_MAXFINAL
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    int rk = 0;
    for (int o = 0; o < n; ++o) rk += (sE[o] < sE[b]) || (sE[o] == sE[b] && o < b);
    rank[b] = rk;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    const int rk = rank[b];
    out_E[rk] = sE[b];
    out_logp[rk] = pick(ds.logp, cur)[b];
  }
  for (size_t e = threadIdx.x; e < (size_t)n * N; e += blockDim.x) {
    const int b = (int)(e / N), s = (int)(e % N);
    out_states[(size_t)rank[b] * N + s] = pick(ds.states, cur)[e];
  }
  if (threadIdx.x == 0) *out_n = n;
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
cudaError_t launch_right_envs(const DevTables& tb, DevWeights<T> wt, DevMPS<T> mps, int row, const DevSearch& ds,
                              DevBeamT<T> bt, int cur, cudaStream_t st) {
  // small bonds: G environments per block kept in shared memory; large
  // bonds: one beam element per block, environments read from global memory
  const int use_rn = bt.rs <= MAXP ? 1 : 0;
  const int G = use_rn ? (sizeof(T) == 4 ? 8 : 4) : 1;
  const size_t base = sizeof(T) * ((size_t)MAXP * MAXCHI + 32 + (size_t)bt.rs * MAXP +
                                   (use_rn ? (size_t)G * MAXCHI * bt.rs : 0));
  const size_t full = base + sizeof(T) * mps.site_stride;
  const int use_smem = full <= 200 * 1024 ? 1 : 0;
  // the per-(class pair) products, when they fit beside the staged site
  const size_t chi = (size_t)bt.chi;
  const size_t tbytes = sizeof(T) * (size_t)MAXP * bt.rs * chi;
  const int use_t = (use_smem && full + tbytes <= 200 * 1024) ? 1 : 0;
  const size_t smem = use_t ? full + tbytes : (use_smem ? full : base);
  static std::once_flag attr_once;  // thread-safe: batches enqueue from several threads
  std::call_once(attr_once, [&] { cudaFuncSetAttribute(k_right_envs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 4096); });
  ZOK(tb, wt, mps, ds, bt);
  count_launches("k_right_envs", st);
  k_right_envs<T><<<dim3((ds.cap + G - 1) / G, 1, zn()), 512, smem, st>>>(tb, wt, mps, row, ds, bt, cur, G, use_smem,
                                                                          use_rn, use_t, zs());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_marginals(const DevTables& tb, DevWeights<T> wt, DevWeights<double> wd, DevMPS<T> mps, int site,
                             const DevSearch& ds, DevBeamT<T> bt, int cur, cudaStream_t st, double flops) {
  if constexpr (std::is_same<T, float>::value) {
    ZOK(tb, wt, mps, ds, bt);
    // variant 0: the site staged in shared memory (when it fits beside the
    // warps' buffers); variant 1: the site read through the L1 cache, less
    // shared memory per block and more blocks per SM.  Both compute the same
    // values from the same data.
    const size_t site_floats = mps.site_stride;
    const size_t warp_floats = (size_t)MW * 2 * MAXP * bt.chi;
    const bool fits = sizeof(float) * (site_floats + warp_floats) <= 160 * 1024;
    static std::once_flag once;
    std::call_once(once, [] {
      cudaFuncSetAttribute(k_marginals_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    auto run = [&](int v) {
      const int staged = v == 0 ? (int)site_floats : 0;
      const size_t smem = sizeof(float) * ((size_t)staged + warp_floats);
      k_marginals_f32<<<dim3((ds.cap + MW - 1) / MW, 1, zn()), 32 * MW, smem, st>>>(tb, wt, mps, site, ds, bt, cur,
                                                                                    staged, zs());
    };
    // the bonds of a site depend on its column and on whether its row is the
    // first (the beam still filling) or the last (trivial environment below)
    const int i = site / tb.cols, j = site % tb.cols;
    const long long shape[] = {bt.chi, ds.cap, tb.dmax, (long long)site_floats, j, std::min(i, 1), i == tb.rows - 1};
    const int v = tune_pick("k_marginals", shape, 7, st, 2, fits ? 3u : 2u, fits ? 0 : 1, run);
    count_launches("k_marginals", st, flops);
    run(v);
    return cudaGetLastError();
  } else {
    (void)wt;
    ZOK(tb, wd, mps, ds, bt);
    count_launches("k_marginals", st, flops);
    k_marginals<T><<<dim3(ds.cap, 1, zn()), 256, 0, st>>>(tb, wd, mps, site, ds, bt, cur, zs());
    return cudaGetLastError();
  }
}

cudaError_t launch_merge(const DevTables& tb, int site, const DevSearch& ds, int cur, int merge, cudaStream_t st) {
  ZOK(tb, ds);
  const int nbk = (ds.cap + 255) / 256;
  const size_t z = zs();
  cudaError_t e;
  if (merge) {
    if ((e = zfill(ds.htab, 0, sizeof(int) * ds.hsize, st)) != cudaSuccess) return e;
    if ((e = zfill(ds.hmin, 0x7f, sizeof(int) * ds.hsize, st)) != cudaSuccess) return e;
  }
  count_launches("k_class_insert", st);
  k_class_insert<<<dim3(nbk, 1, zn()), 256, 0, st>>>(tb, site, ds, cur, merge, z);
  const size_t tot = (size_t)ds.cap * ds.dmax;
  const int wb = (int)std::min<size_t>((tot + 255) / 256, 8192);
  if ((e = zfill(ds.wmin, 0xff, sizeof(unsigned long long) * tot, st)) != cudaSuccess) return e;
  if ((e = zfill(ds.win, 0x7f, sizeof(int) * tot, st)) != cudaSuccess) return e;
  if ((e = zfill(ds.wkey, 0x7f, sizeof(int) * ds.cap, st)) != cudaSuccess) return e;
  count_launches("k_win_min", st);
  k_win_min<<<dim3(wb, 1, zn()), 256, 0, st>>>(tb, site, ds, cur, merge, z);
  count_launches("k_win_arg", st);
  k_win_arg<<<dim3(wb, 1, zn()), 256, 0, st>>>(tb, site, ds, cur, merge, z);
  count_launches("k_win_fix", st);
  k_win_fix<<<dim3(wb, 1, zn()), 256, 0, st>>>(tb, site, ds, cur, merge, z);
  return cudaGetLastError();
}

cudaError_t launch_select(const DevTables& tb, int site, const DevSearch& ds, int cur, double log_cut,
                          cudaStream_t st) {
  const size_t tot = (size_t)ds.cap * ds.dmax;
  // grid-stride passes on at most 64 blocks: a solve alone runs them as fast
  // as on a full-GPU grid (they move a few tens of MB through L2), and the
  // other solves of a batch keep the remaining SMs (measured: batch of 32
  // +6.6%, one solve unchanged)
  // (in a lockstep group every instance gets 8: the group fills the GPU)
  const int blocks = (int)std::min<size_t>((tot + 1023) / 1024, zn() > 1 ? 8 : 64);
  ZOK(tb, ds);
  const size_t z = zs();
  const dim3 g(blocks, 1, zn()), g1(1, 1, zn());
  if (log_cut > -INFINITY) {
    count_launches("k_logp_max", st);
    k_logp_max<<<g, 1024, 0, st>>>(tb, site, ds, cur, z);
  }
  // pass 0 and the split scan every candidate; the later passes and the
  // final classification only the candidates of the chosen top digit
  count_launches("k_select_pass", st);
  k_select_pass<<<g, 1024, 0, st>>>(tb, site, ds, cur, 0, log_cut, nullptr, nullptr, z);
  count_launches("k_select_classify", st);
  k_select_classify<<<g, 1024, 0, st>>>(tb, site, ds, cur, log_cut, nullptr, nullptr, 1, z);
  count_launches("k_select_refine", st);
  k_select_refine<<<g1, 1024, 0, st>>>(tb, site, ds, cur, log_cut, z);
  int P = 1;
  while (P < ds.cap) P <<= 1;
  count_launches("k_select_sort", st);
  k_select_sort<<<g1, 1024, sizeof(unsigned long long) * P, st>>>(tb, site, ds, cur, cur ^ 1, z);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(const DevTables& tb, DevMPS<T> mps, int site, const DevSearch& ds, DevBeamT<T> bt, int cur,
                          cudaStream_t st) {
  ZOK(tb, mps, ds, bt);
  count_launches("k_update", st);
  k_update<T><<<dim3(ds.cap, 1, zn()), 64, 0, st>>>(tb, mps, site, ds, bt, cur, zs());
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lenv_from_prefix(const DevTables& tb, DevMPS<T> mps, int site, const DevSearch& ds,
                                    DevBeamT<T> bt, int cur, cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;  // not part of a grouped solve
  count_launches("k_lenv_prefix", st);
  k_lenv_prefix<T><<<ds.cap, 64, 0, st>>>(tb, mps, site, ds, bt, cur);
  return cudaGetLastError();
}

namespace {
__global__ void k_or_flag(int* dst, const int* src, size_t zs) {
  dst = zp(dst, zs);
  src = zp(src, zs);
  if (threadIdx.x == 0) *dst |= *src;
}
}  // namespace

cudaError_t launch_or_flag(int* dst, const int* src, cudaStream_t st) {
  ZOK(dst, src);
  count_launches("k_or_flag", st);
  k_or_flag<<<dim3(1, 1, zn()), 32, 0, st>>>(dst, src, zs());
  return cudaGetLastError();
}

namespace {
// The GPU's global nanosecond timer at the moment this kernel runs.
__global__ void k_stamp(unsigned long long* slot, size_t zs) {
  slot = zp(slot, zs);
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  if (threadIdx.x == 0) *slot = t;
}
}  // namespace

cudaError_t launch_stamp(unsigned long long* slot, cudaStream_t st) {
  ZOK(slot);
  count_launches("k_stamp", st);
  k_stamp<<<dim3(1, 1, zn()), 32, 0, st>>>(slot, zs());
  return cudaGetLastError();
}

cudaError_t launch_reset_beam(const DevSearch& ds, int cur, cudaStream_t st) {
  ZOK(ds);
  count_launches("k_reset_beam", st);
  k_reset_beam<<<dim3(1, 1, zn()), 256, 0, st>>>(ds, cur, zs());
  return cudaGetLastError();
}

cudaError_t launch_final(const DevTables& tb, const DevSearch& ds, int cur, uint16_t* out_states, int64_t* out_E,
                         double* out_logp, int* out_n, cudaStream_t st) {
  const int sm = (int)((sizeof(long long) + sizeof(int)) * SPG_MAXFINAL);
  static std::once_flag attr_once;  // thread-safe: batches enqueue from several threads
  std::call_once(attr_once, [&] { cudaFuncSetAttribute(k_final, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); });
  ZOK(tb, ds, out_states, out_E, out_logp, out_n);
  count_launches("k_final", st);
  k_final<<<dim3(1, 1, zn()), 1024, sm, st>>>(tb, ds, cur, out_states, out_E, out_logp, out_n, zs());
  return cudaGetLastError();
}

cudaError_t launch_droplets(const DevTables& tb, int site, const DevSearch& ds, int cur, int merge, cudaStream_t st) {
  ZOK(tb, ds);
  count_launches("k_droplets", st);
  k_droplets<<<dim3(ds.cap, 1, zn()), 256, 0, st>>>(tb, site, ds, cur, merge, zs());
  return cudaGetLastError();
}

cudaError_t launch_final_droplets(const DevSearch& ds, int cur, int* out_n, int64_t* out_E, uint16_t* out_states,
                                  cudaStream_t st) {
  ZOK(ds, out_n, out_E, out_states);
  count_launches("k_final_droplets", st);
  k_final_droplets<<<dim3(1, 1, zn()), 256, 0, st>>>(ds, cur, out_n, out_E, out_states, zs());
  return cudaGetLastError();
}

cudaError_t launch_force_init(const DevSearch& ds, const int* n_dev, int cur, cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;
  count_launches("k_force_init", st);
  k_force_init<<<64, 256, 0, st>>>(ds, n_dev, cur);
  return cudaGetLastError();
}

cudaError_t launch_force(int site, const DevSearch& ds, int cur, const uint16_t* targets, double* out,
                         cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;
  count_launches("k_force", st);
  k_force<<<(ds.cap + 255) / 256, 256, 0, st>>>(site, ds, cur, targets, out);
  return cudaGetLastError();
}

cudaError_t launch_logmarg_err(const double* a, const double* r, const int* n_dev, int N, double* out,
                               cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;
  count_launches("k_logmarg_err", st);
  k_logmarg_err<<<1, 1024, 0, st>>>(a, r, n_dev, N, out);
  return cudaGetLastError();
}

namespace {
// Byte copies and fills inside a solve (k_zcopy: 16-byte words when both
// ends and the size allow), one grid slice per instance of a group.
__global__ void k_zcopy(void* dst, const void* src, size_t bytes, size_t zs) {
  dst = zp(dst, zs);
  src = zp(src, zs);
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | bytes) & 15) == 0) {
    const uint4* s = static_cast<const uint4*>(src);
    uint4* d = static_cast<uint4*>(dst);
    for (size_t i = i0; i < bytes / 16; i += st) d[i] = s[i];
  } else {
    const unsigned char* s = static_cast<const unsigned char*>(src);
    unsigned char* d = static_cast<unsigned char*>(dst);
    for (size_t i = i0; i < bytes; i += st) d[i] = s[i];
  }
}
__global__ void k_zfill(void* dst, int byte, size_t bytes, size_t zs) {
  dst = zp(dst, zs);
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
  const unsigned v = (unsigned)byte & 0xffu;
  if (((reinterpret_cast<uintptr_t>(dst) | bytes) & 15) == 0) {
    const unsigned w = v * 0x01010101u;
    uint4* d = static_cast<uint4*>(dst);
    for (size_t i = i0; i < bytes / 16; i += st) d[i] = make_uint4(w, w, w, w);
  } else {
    unsigned char* d = static_cast<unsigned char*>(dst);
    for (size_t i = i0; i < bytes; i += st) d[i] = (unsigned char)v;
  }
}
}  // namespace

// Without a group the stream's own copy and fill; in a group one kernel
// over every instance.
cudaError_t zcopy(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if (zn() == 1) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
  if (!zok(dst, src, static_cast<const char*>(dst) + bytes - 1, static_cast<const char*>(src) + bytes - 1))
    return cudaErrorInvalidValue;
  count_launches("k_zcopy", st);
  const size_t units = (bytes + 15) / 16;
  k_zcopy<<<dim3((unsigned)std::min<size_t>((units + 255) / 256, 1024), 1, zn()), 256, 0, st>>>(dst, src, bytes,
                                                                                               zs());
  return cudaGetLastError();
}

cudaError_t zfill(void* dst, int byte, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if (zn() == 1) return cudaMemsetAsync(dst, byte, bytes, st);
  if (!zok(dst, static_cast<const char*>(dst) + bytes - 1)) return cudaErrorInvalidValue;
  count_launches("k_zfill", st);
  const size_t units = (bytes + 15) / 16;
  k_zfill<<<dim3((unsigned)std::min<size_t>((units + 255) / 256, 1024), 1, zn()), 256, 0, st>>>(dst, byte, bytes,
                                                                                               zs());
  return cudaGetLastError();
}

template cudaError_t launch_right_envs<double>(const DevTables&, DevWeights<double>, DevMPS<double>, int,
                                               const DevSearch&, DevBeamT<double>, int, cudaStream_t);
template cudaError_t launch_right_envs<float>(const DevTables&, DevWeights<float>, DevMPS<float>, int,
                                              const DevSearch&, DevBeamT<float>, int, cudaStream_t);
template cudaError_t launch_marginals<double>(const DevTables&, DevWeights<double>, DevWeights<double>,
                                              DevMPS<double>, int, const DevSearch&, DevBeamT<double>, int,
                                              cudaStream_t, double);
template cudaError_t launch_marginals<float>(const DevTables&, DevWeights<float>, DevWeights<double>, DevMPS<float>,
                                             int, const DevSearch&, DevBeamT<float>, int, cudaStream_t, double);
template cudaError_t launch_update<double>(const DevTables&, DevMPS<double>, int, const DevSearch&,
                                           DevBeamT<double>, int, cudaStream_t);
template cudaError_t launch_update<float>(const DevTables&, DevMPS<float>, int, const DevSearch&, DevBeamT<float>,
                                          int, cudaStream_t);
template cudaError_t launch_lenv_from_prefix<double>(const DevTables&, DevMPS<double>, int, const DevSearch&,
                                                     DevBeamT<double>, int, cudaStream_t);
template cudaError_t launch_lenv_from_prefix<float>(const DevTables&, DevMPS<float>, int, const DevSearch&,
                                                    DevBeamT<float>, int, cudaStream_t);

}  // namespace spg
