// Right environments of the beam search (S5) on the tensor cores, FP32 mode,
// for rows whose sites satisfy the square-lattice conditions below
// (Chimera-like and square lattices).  The contraction and its layout are
// those of k_right_envs (search.cu): for beam element b at the start of row
// i, with B = B_{i+1}, u_j the PD class of the fixed cluster (i-1, j):
//   R_L = 1;  R_j[a][l] = bA[l / Gin][u_j] sum_h bL[l][h] Y[h][a],
//   Y[h][a] = sum_{x: PL x = h} w(x) bU[u_j][PU x] sum_a' B_j[PD x][a][a'] R_{j+1}[a'][PR x],
// each R_j scaled to max |.| = 1.  Paper: Sec. 2 (environments of the
// conditional probabilities) and Sec. 3.1 (the contractions run on the GPU).
//
// The dominant part, T[pd][r][a] = sum_a' B_j[pd][a][a'] R_{j+1}[a'][r] for
// every (beam element, r) and (pd, a), is one dense product per column and
// beam tile: D[(b, r)][(pd, a)] = sum_a' R_b[a'][r] B_j[(pd, a)][a'], M = 128
// (8 beam elements x 16 right-bond entries), N = 512 (16 projected states x
// 32 bond entries), K = 32, on tcgen05 with split-TF32 operands (hi*hi +
// hi*lo + lo*hi, FP32-level accuracy; see umma_gemm.cu) and the accumulator
// in tensor memory (all 512 columns).  The sum over states is then
// thread-local: the thread of TMEM lane (b, r) reads the 16 column groups
// (pd, .) of its row and forms
//   Y_b[h(r)][a] = sum_pd C_u[pd][r] T[pd][r][a],
//   C_u[pd][r] = sum_{x: PD x = pd, PR x = r} w(x) bU[u][PU x],
// which needs every state with right class r to have one left class h(r),
// distinct for distinct r (square lattices: a cluster's left and right edges
// project it the same way).  The rightmost column needs no product (R_L is
// the unit environment: T[pd][0][a] = B[pd][a][0]) and is summed directly.
// Conditions of a row (checked on the host): at least 3 columns, Gout = 1,
// no up-index coupling of the MPO, DL, DR, NL <= 16, the bond of the
// environments <= 16, B_{i+1}'s sites of at most 16 x 32 x 32, and the class
// condition above on every column but the rightmost.
//
// One CTA of 8 warps per tile of 8 beam elements of one instance (grid.z:
// the instances of a lockstep group) runs the row's columns right to left:
// TMA loads the column's split site (prepared per row by k_renv_prep) and
// the tile's split R_{j+1} (written by the same CTA in the previous column),
// thread 0 issues the MMAs, warps w and w + 4 read accumulator lane quarter
// w & 3 (half of the state classes each).
// Every mbarrier wait is bounded: on a timeout ERR_TIMEOUT is recorded, the
// CTA waits (bounded) for its copies and products in flight, frees its
// tensor memory and returns.
#include <cuda.h>

#include "spg.h"
#include "spg_internal.h"
#include "tc_ptx.h"

namespace spg {

bool make_f32_tensor_map(void* map, const float* base, int rows, int kp, int box_rows);

namespace {

constexpr int RT_B = 8;      // beam elements per CTA
constexpr int RT_R = 16;     // right-bond rows per beam element
constexpr int RT_M = RT_B * RT_R;
constexpr int RT_PD = 16;    // projected states of a site
constexpr int RT_A = 32;     // bond entries per projected state (rows of B padded to 32)
constexpr int RT_N = RT_PD * RT_A;
constexpr int RT_K = 32;     // bond entries a' (one 128-byte swizzle row of FP32)
constexpr uint32_t A_BYTES = RT_M * RT_K * 4;   // 16 KB per TF32 part
constexpr uint32_t B_HALF = 256 * RT_K * 4;     // 32 KB: one TMA box of 256 rows
constexpr uint32_t B_BYTES = 2 * B_HALF;        // 64 KB per TF32 part
constexpr uint32_t TX_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr size_t RT_SMEM = 2 * (size_t)B_BYTES + 2 * (size_t)A_BYTES + 1024;
constexpr int RT_T = 256;    // threads: warps w and w + 4 share accumulator lane quarter w

// Per row and column j (1 .. cols-2) of the row: the split site B_j as a
// K-major [512][32] matrix (row pd * 32 + a, column a'; zeros beyond the
// site's dims), the state coefficients C_u[pd][r] for every u < 16, and the
// left class h(r) of each right class (-1: no state); for the rightmost
// column j = cols-1 the weights W_u[h][pd] of its direct sum.
//   layout: Bh, Bl [cols][512][32]; Cu [cols][16][16][16]; hr [cols][16]
__global__ void __launch_bounds__(256) k_renv_prep(DevTables tb, DevWeights<float> wt, DevMPS<float> mps, int row,
                                                   float* Bh, float* Bl, float* Cu, int* hr, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  mps = zp(mps, zs);
  Bh = zp(Bh, zs);
  Bl = zp(Bl, zs);
  Cu = zp(Cu, zs);
  hr = zp(hr, zs);
  const int cols = tb.cols;
  const int j = blockIdx.x + 1;
  const bool last = j == cols - 1;  // the rightmost column: only its W below
  const int s = row * cols + j;
  const int* dA = mps.dimA + ((row + 1) * cols + j) * 3;
  const int p = dA[0], chiL = dA[1], chiR = dA[2];
  const float* A = mps.A + (size_t)((row + 1) * cols + j) * mps.site_stride;
  const int tid = threadIdx.x, nt = blockDim.x;
  float* bh = Bh + (size_t)j * RT_N * RT_K;
  float* bl = Bl + (size_t)j * RT_N * RT_K;
  for (int e = tid; e < RT_N * RT_K && !last; e += nt) {
    const int n = e / RT_K, k = e % RT_K;
    const int pd = n / RT_A, a = n % RT_A;
    const float v = (pd < p && a < chiL && k < chiR) ? A[((size_t)pd * chiL + a) * chiR + k] : 0.f;
    float h, l;
    tc::split_tf32(v, h, l);
    bh[e] = h;
    bl[e] = l;
  }
  // C_u[pd][r]: thread (pd, r) sums over the states in index order (a fixed
  // order: the same values on every run)
  const size_t so = (size_t)s * tb.dmax;
  const int d = tb.d[s];
  __shared__ float sw[MAXS];
  __shared__ uint8_t sPD[MAXS], sPR[MAXS], sPU[MAXS], sPL[MAXS];
  __shared__ float sbU[256];
  for (int x = tid; x < d; x += nt) {
    sw[x] = wt.w[so + x];
    sPD[x] = tb.PD[so + x];
    sPR[x] = tb.PR[so + x];
    sPU[x] = tb.PU[so + x];
    sPL[x] = tb.PL[so + x];
  }
  for (int e = tid; e < 256; e += nt) sbU[e] = wt.bU[(size_t)s * 256 + e];
  __syncthreads();
  // the rightmost column (R_L = unit): W_u[h][pd] = sum_{x: PL x = h, PD x
  // = pd} w(x) bU[u][PU x] in C_u's slot, thread (h, pd)
  float* cu = Cu + (size_t)j * 16 * 256;
  for (int c = tid; c < 256; c += nt) {
    const int pd = last ? c % 16 : c / 16, r = c % 16, h = c / 16;
    float acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = 0.f;
    for (int x = 0; x < d; ++x)
      if (last ? (sPL[x] == h && sPD[x] == pd) : (sPD[x] == pd && sPR[x] == r)) {
        const float w = sw[x];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] += w * sbU[u * 16 + sPU[x]];
      }
#pragma unroll
    for (int u = 0; u < 16; ++u) cu[(size_t)u * 256 + c] = acc[u];
  }
  if (tid < 16 && !last) {
    int h = -1;
    for (int x = 0; x < d; ++x)
      if (sPR[x] == tid) {
        h = sPL[x];
        break;
      }
    hr[j * 16 + tid] = h;
  }
}

// The row's right environments for beam tile blockIdx.x of instance
// blockIdx.z.  Asp: the tiles' split R_{j+1} ([tiles][128][32] per part),
// Bh/Bl/Cu/hr from k_renv_prep.
__global__ void __launch_bounds__(RT_T, 1)
    k_renv_tc(const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
              const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl, DevTables tb,
              DevWeights<float> wt, DevMPS<float> mps, int row, DevSearch ds, DevBeamT<float> bt, int cur,
              const float* Cu, const int* hr, float* Ah, float* Al, size_t zs) {
  tb = zp(tb, zs);
  wt = zp(wt, zs);
  mps = zp(mps, zs);
  ds = zp(ds, zs);
  bt = zp(bt, zs);
  Cu = zp(Cu, zs);
  hr = zp(hr, zs);
  Ah = zp(Ah, zs);
  Al = zp(Al, zs);
  const int nb = ds.n_beam[cur];
  const int b0 = blockIdx.x * RT_B;
  if (b0 >= nb) return;
  const int gn = min(RT_B, nb - b0);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t base0 = tc::smem_u32(smem_raw);
  const uint32_t tiles = (base0 + 1023u) & ~1023u;
  const uint32_t sBh = tiles, sBl = tiles + B_BYTES, sAh = tiles + 2 * B_BYTES, sAl = sAh + A_BYTES;
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ float Ys[RT_B][16][RT_A + 1];  // padded: the writes of part 1 spread over the banks
  __shared__ float sbL[16 * MAXP];
  __shared__ float sbA[256];
  __shared__ int s_hr[16];
  __shared__ int s_abort;
  __shared__ uint8_t s_up[RT_B][SPG_MAX_COLS];  // PD class of the cluster above column j, per element
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t full = tc::smem_u32(&bars[0]), done = tc::smem_u32(&bars[1]);
  const int cols = tb.cols, chi = bt.chi, rs = bt.rs;
  const size_t renv = (size_t)chi * rs;
  float* Ath = Ah + (size_t)blockIdx.x * RT_M * RT_K;  // this tile's split R_{j+1}
  float* Atl = Al + (size_t)blockIdx.x * RT_M * RT_K;
  if (tid == 0) {
    tc::mbar_init(full, 1);
    tc::mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // R_L = unit and the row-start bookkeeping of the beam elements
  for (int g = 0; g < gn; ++g) {
    const int b = b0 + g;
    float* Rb = bt.R + ((size_t)b * (cols + 1) + cols) * renv;
    for (int e = tid; e < (int)renv; e += RT_T) Rb[e] = e == 0 ? 1.f : 0.f;
    if (tid == 0) pick(ds.rid, cur)[b] = b;
    for (int a = tid; a < chi; a += RT_T) pick(bt.lenv, cur)[(size_t)b * chi + a] = a == 0 ? 1.f : 0.f;
  }
  for (int e = tid; e < RT_B * 16 * (RT_A + 1); e += RT_T) (&Ys[0][0][0])[e] = 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // the PD class of the fixed cluster above column j for the block's
  // element g, for every column at once (the state and table loads of all
  // of them in flight together)
  for (int e = tid; e < RT_B * cols; e += RT_T) {
    const int g = e / cols, j = e % cols;
    int u = 0;
    if (row > 0 && g < gn) {
      const int s_up = (row - 1) * cols + j;
      u = tb.PD[(size_t)s_up * tb.dmax + pick(ds.states, cur)[(size_t)(b0 + g) * ds.N + s_up]];
    }
    s_up[g][j] = (uint8_t)u;
  }
  __syncthreads();
  auto up_class = [&](int g, int j) -> int { return s_up[g < RT_B ? g : 0][j]; };
  // R_j[a][l] = bA[l / Gin][u] sum_h bL[l][h] Y[h][a] from Ys: thread (bl2,
  // a), a warp per beam element, every l (Ys read along a, bL broadcast);
  // scaled to max |.| = 1; written to R and, split, as the next column's
  // operand; Ys cleared for the next column
  auto finish_column = [&](int j) {
    const int s = row * cols + j;
    const int* dA = mps.dimA + ((row + 1) * cols + j) * 3;
    const int chiL = dA[1];
    const int* dm = tb.dims + s * DIMW;
    const int DL = dm[D_DL], NL = dm[D_NL], Gin = dm[D_GIN];
    for (int e = tid; e < 16 * MAXP; e += RT_T) sbL[e] = (e / MAXP) < DL ? wt.bL[(size_t)s * tb.lstride + e] : 0.f;
    for (int e = tid; e < 256; e += RT_T) sbA[e] = wt.bA[(size_t)s * 256 + e];
    __syncthreads();
    const int bl2 = tid >> 5, a = tid & 31;
    const int u2 = up_class(bl2, j);
    const bool bok = bl2 < gn;
    float out[16];
    float mx = 0.f;
    float y[16];
#pragma unroll
    for (int hh = 0; hh < 16; ++hh) y[hh] = Ys[bl2][hh][a];
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      float t = 0.f;
      if (bok && l < DL && a < chiL) {
#pragma unroll
        for (int hh = 0; hh < 16; ++hh)
          if (hh < NL) t += sbL[l * MAXP + hh] * y[hh];
        t *= sbA[(l / Gin) * 16 + u2];
      }
      out[l] = t;
      mx = fmaxf(mx, fabsf(t));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float inv = mx > 0.f ? 1.f / mx : 0.f;
    if (bok && a < chi) {
      float* Rj = bt.R + ((size_t)(b0 + bl2) * (cols + 1) + j) * renv + (size_t)a * rs;
#pragma unroll
      for (int l = 0; l < 16; ++l)
        if (l < rs) Rj[l] = out[l] * inv;
    }
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      float hi, lo;
      tc::split_tf32(out[l] * inv, hi, lo);
      Ath[(size_t)(bl2 * RT_R + l) * RT_K + a] = hi;
      Atl[(size_t)(bl2 * RT_R + l) * RT_K + a] = lo;
    }
    __syncthreads();
    for (int e = tid; e < RT_B * 16 * (RT_A + 1); e += RT_T) (&Ys[0][0][0])[e] = 0.f;
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
  };
  {
    // column cols-1 against the unit R_L: T[pd][0][a] = B[pd][a][0], so
    // Y_b[h][a] = sum_{x: PL x = h} w(x) bU[u][PU x] B[PD x][a][0] directly
    // (thread (g, a) owns column a of Ys[g], states in index order)
    const int j = cols - 1;
    const int* dA = mps.dimA + ((row + 1) * cols + j) * 3;
    const int p = dA[0], chiL = dA[1], chiR = dA[2];
    const float* Bs = mps.A + (size_t)((row + 1) * cols + j) * mps.site_stride;
    for (int e = tid; e < RT_B * 16 * RT_A; e += RT_T) {
      const int g = e / (16 * RT_A), h = (e / RT_A) % 16, a = e % RT_A;
      if (g >= gn || a >= chiL) continue;
      const float* W = Cu + ((size_t)j * 16 + up_class(g, j)) * 256 + h * 16;
      float acc = 0.f;
      for (int pd = 0; pd < p; ++pd) acc += W[pd] * Bs[((size_t)pd * chiL + a) * chiR];
      Ys[g][h][a] = acc;
    }
    __syncthreads();
    finish_column(j);
  }
  // this thread's accumulator row: beam element bl, right-bond entry r
  // (warps w and w + 4 read lane quarter w & 3 and take the state classes
  // pd < 8 and pd >= 8 respectively)
  const int quarter = warp & 3, half = warp >> 2;
  const int bl = 2 * quarter + (lane >> 4), r = lane & 15;
  int it = 0;
  for (int j = cols - 2; j >= 1; --j, ++it) {
    const int s = row * cols + j;
    const int* dA = mps.dimA + ((row + 1) * cols + j) * 3;
    const int p = dA[0];
    const int DR = tb.dims[s * DIMW + D_DR];
    // copies: the column's split site (two boxes of 256 rows per part) and
    // the tile's split R_{j+1}
    if (tid == 0) {
      tc::mbar_expect_tx(full, TX_BYTES);
      const int z = (int)blockIdx.z;
      tc::tma_load_3d(sBh, &tBh, 0, j * RT_N, z, full);
      tc::tma_load_3d(sBh + B_HALF, &tBh, 0, j * RT_N + 256, z, full);
      tc::tma_load_3d(sBl, &tBl, 0, j * RT_N, z, full);
      tc::tma_load_3d(sBl + B_HALF, &tBl, 0, j * RT_N + 256, z, full);
      tc::tma_load_3d(sAh, &tAh, 0, blockIdx.x * RT_M, z, full);
      tc::tma_load_3d(sAl, &tAl, 0, blockIdx.x * RT_M, z, full);
    }
    if (tid < 16) s_hr[tid] = hr[j * 16 + tid];
    const bool landed = tc::mbar_wait(full, it & 1, ds.err);
    if (!landed) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr uint32_t idesc = tc::tf32_idesc(RT_M, 256);
      const uint64_t ah = tc::sw128_desc(sAh), al = tc::sw128_desc(sAl);
      for (int hf = 0; hf < 2; ++hf) {
        const uint64_t bh = tc::sw128_desc(sBh + hf * B_HALF), blo = tc::sw128_desc(sBl + hf * B_HALF);
        const uint32_t dt = tmem + (uint32_t)(hf * 256);
        for (int kk = 0; kk < RT_K / 8; ++kk) {
          const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 8 floats further along the row
          tc::umma_tf32(dt, ah + o, bh + o, idesc, kk > 0 ? 1u : 0u);
          tc::umma_tf32(dt, ah + o, blo + o, idesc, 1u);
          tc::umma_tf32(dt, al + o, bh + o, idesc, 1u);
        }
      }
      tc::umma_commit(done);
    }
    __syncwarp();
    const bool computed = tc::mbar_wait(done, it & 1, ds.err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!computed) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    // Y_b[h(r)][a] = sum_pd C_u[pd][r] T[pd][r][a] (lane (bl, r) of the warp's quarter)
    const bool valid = bl < gn && r < DR;
    const float* cu = Cu + ((size_t)j * 16 + up_class(bl, j)) * 256 + r;
    float acc[RT_A];
#pragma unroll
    for (int a = 0; a < RT_A; ++a) acc[a] = 0.f;
    // the coefficients first: the accumulator loads below are ordered
    // against every memory access
    constexpr int PH = RT_PD / 2;  // classes per half
    const int pd0 = half * PH;
    float cv[PH];
#pragma unroll
    for (int q = 0; q < PH; ++q) cv[q] = (valid && pd0 + q < p) ? cu[(pd0 + q) * 16] : 0.f;
#pragma unroll
    for (int q = 0; q < PH; ++q) {
      if (pd0 + q >= p) break;
      float v[RT_A];
      tc::tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((pd0 + q) * RT_A), v);
      const float c = cv[q];
#pragma unroll
      for (int a = 0; a < RT_A; ++a) acc[a] += c * v[a];
    }
    // the lower half's partial sum, then the upper half's added to it
    const int h = valid ? s_hr[r] : -1;
    if (half == 0 && h >= 0)
#pragma unroll
      for (int a = 0; a < RT_A; ++a) Ys[bl][h][a] = acc[a];
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (half == 1 && h >= 0)
#pragma unroll
      for (int a = 0; a < RT_A; ++a) Ys[bl][h][a] += acc[a];
    __syncthreads();
    finish_column(j);
  }
  if (s_abort && tid == 0) {
    // copies or products still in flight land before the CTA exits (bounded)
    tc::mbar_wait(full, it & 1, ds.err);
    tc::mbar_wait(done, it & 1, ds.err);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

}  // namespace

size_t renv_tc_elems(int cols, int cap) {
  // Bh, Bl, Cu, hr, Ah, Al
  const size_t tiles = ((size_t)cap + RT_B - 1) / RT_B;
  return 2 * (size_t)cols * RT_N * RT_K + (size_t)cols * 16 * 256 + (size_t)cols * 16 + 2 * tiles * RT_M * RT_K + 64;
}

cudaError_t launch_right_envs_tc(const DevTables& tb, DevWeights<float> wt, DevMPS<float> mps, int row,
                                 const DevSearch& ds, DevBeamT<float> bt, int cur, float* work, cudaStream_t st) {
  const int cols = tb.cols;
  const int tiles = (ds.cap + RT_B - 1) / RT_B;
  float* Bh = work;
  float* Bl = Bh + (size_t)cols * RT_N * RT_K;
  float* Cu = Bl + (size_t)cols * RT_N * RT_K;
  int* hr = reinterpret_cast<int*>(Cu + (size_t)cols * 16 * 256);
  float* Ah = reinterpret_cast<float*>(hr + (size_t)cols * 16);
  float* Al = Ah + (size_t)tiles * RT_M * RT_K;
  ZOK(tb, wt, mps, ds, bt, work, Al + (size_t)tiles * RT_M * RT_K - 1);
  // TMA needs 16-byte aligned bases: every part above is a multiple of 16
  // bytes from work (work itself 256-byte aligned)
  CUtensorMap maps[4];
  if (!make_f32_tensor_map(&maps[0], Bh, cols * RT_N, RT_K, 256) ||
      !make_f32_tensor_map(&maps[1], Bl, cols * RT_N, RT_K, 256) ||
      !make_f32_tensor_map(&maps[2], Ah, tiles * RT_M, RT_K, RT_M) ||
      !make_f32_tensor_map(&maps[3], Al, tiles * RT_M, RT_K, RT_M))
    return cudaErrorInvalidValue;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_renv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT_SMEM);
  });
  count_launches("k_renv_prep", st);
  k_renv_prep<<<dim3(cols - 1, 1, zn()), 256, 0, st>>>(tb, wt, mps, row, Bh, Bl, Cu, hr, zs());
  // algorithmic flops of the products (the three split-TF32 passes are the
  // way they are computed, not more work)
  count_launches("k_renv_tc", st, 2.0 * (double)tiles * RT_M * RT_N * RT_K * (cols - 2));
  k_renv_tc<<<dim3(tiles, 1, zn()), RT_T, RT_SMEM, st>>>(maps[0], maps[1], maps[2], maps[3], tb, wt, mps, row, ds, bt,
                                                        cur, Cu, hr, Ah, Al, zs());
  return cudaGetLastError();
}

}  // namespace spg
