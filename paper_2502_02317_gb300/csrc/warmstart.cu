// Learned warm start of the variational compression: the MLP that maps the
// couplings near a boundary row to that row's MPS sites (forward, backward,
// Adam, BF16 inference), and the kernels that move boundary-MPS rows between
// the solver's layout and the network's padded [16][chi][chi] sites.
//
// Paper: Sec. 3.1 (MpsParameters(bond_dim, num_sweeps): the variational
// compression the network initialises; the SVD zipper stays the default).
// The paper has no learned part; the network, its loss and the optimiser are
// this library's reading of "a warm start predicted from the couplings".
//
// Parameters live in one flat FP32 array [W1 | b1 | W2 | b2 | W3 | b3]
// (weights row-major [fan_out][fan_in]); gradients and the Adam moments use
// the same layout.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/spg.h"
#include "spg_internal.h"

namespace spg {

namespace {

// ---------------------------------------------------------------- GEMM
// C[i][j] = act(sum_k opA(i, k) opB(k, j) + bias[j]) for i < M, j < N:
//   opA(i, k) = TA ? A[k * lda + i] : A[i * lda + k]
//   opB(k, j) = TB ? B[j * ldb + k] : B[k * ldb + j]
// act 0: identity, 1: tanh.  RoundA rounds A's entries to BF16 when they are
// staged (with a BF16 B, the inference products of BF16 operands with FP32
// accumulation).  64 x 64 tile, K slices of 16, 256 threads, 4 x 4 outputs
// per thread.
constexpr int GBM = 64, GBN = 64, GBK = 16;

template <typename TW>
__device__ __forceinline__ float to_f(TW v) {
  return (float)v;
}
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <bool TA, bool TB, typename TW, bool RoundA>
__global__ void __launch_bounds__(256) k_mlp_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                                  const TW* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                                  const float* __restrict__ bias, int act) {
  __shared__ float sA[GBK][GBM + 4];
  __shared__ float sB[GBK][GBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * GBM, j0 = blockIdx.x * GBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256;
      int i, k;
      if (TA) {  // A[k][i]: i contiguous
        k = e / GBM;
        i = e % GBM;
      } else {  // A[i][k]: k contiguous
        i = e / GBK;
        k = e % GBK;
      }
      const int gi = i0 + i, gk = k0 + k;
      float v = 0.f;
      if (gi < M && gk < K) v = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
      if (RoundA) v = __bfloat162float(__float2bfloat16(v));
      sA[k][i] = v;
      int j, kb;
      if (TB) {  // B[j][k]: k contiguous
        j = e / GBK;
        kb = e % GBK;
      } else {  // B[k][j]: j contiguous
        kb = e / GBN;
        j = e % GBN;
      }
      const int gj = j0 + j, gkb = k0 + kb;
      float w = 0.f;
      if (gj < N && gkb < K) w = to_f<TW>(TB ? B[(size_t)gj * ldb + gkb] : B[(size_t)gkb * ldb + gj]);
      sB[kb][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GBK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = sA[k][ty * 4 + q];
        b[q] = sB[k][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int gi = i0 + ty * 4 + p;
    if (gi >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = j0 + tx * 4 + q;
      if (gj >= N) continue;
      float v = acc[p][q] + (bias ? bias[gj] : 0.f);
      if (act == 1) v = tanhf(v);
      C[(size_t)gi * ldc + gj] = v;
    }
  }
}

template <bool TA, bool TB, typename TW, bool RoundA>
cudaError_t gemm_mlp(int M, int N, int K, const float* A, int lda, const TW* B, int ldb, float* C, int ldc,
                     const float* bias, int act, cudaStream_t st, double flops_scale = 1.0) {
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  count_launches("k_mlp_gemm", st, 2.0 * M * N * K * flops_scale);
  k_mlp_gemm<TA, TB, TW, RoundA><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- elementwise
// counter-based uniform in [0, 1): splitmix64 of (seed, index)
__device__ __forceinline__ double unit_hash(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9e3779b97f4a7c15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// weights uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), biases zero
__global__ void k_mlp_init(float* p, int64_t count, int64_t oW1, int64_t ob1, int64_t oW2, int64_t ob2, int64_t oW3,
                           int64_t ob3, int n_in, int n_hidden, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    int fan = 0;
    if (e < ob1) fan = n_in;
    else if (e >= oW2 && e < ob2) fan = n_hidden;
    else if (e >= oW3 && e < ob3) fan = n_hidden;
    p[e] = fan ? (float)((2.0 * unit_hash(seed, (uint64_t)e) - 1.0) / sqrt((double)fan)) : 0.f;
  }
  (void)oW1;
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = __float2bfloat16(src[e]);
}

// dY = (Y - T) / n in place of Y; per-block partial sums of (Y - T)^2
__global__ void k_loss_dy(float* __restrict__ Y, const float* __restrict__ T, int64_t count, float inv_n,
                          double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    s += (double)d * (double)d;
    Y[e] = d * inv_n;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// out[slot] (+)= 0.5 * sum of the nb partial sums / n (deterministic order)
__global__ void k_loss_sum(const double* __restrict__ part, int nb, double inv_n, double* out, int accumulate) {
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[b];
    const double v = 0.5 * t * inv_n;
    *out = accumulate ? *out + v : v;
  }
}

// dA = dH * (1 - H^2) in place of dH (tanh backward)
__global__ void k_tanh_bwd(float* __restrict__ dH, const float* __restrict__ H, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float h = H[e];
    dH[e] *= 1.f - h * h;
  }
}

// db[j] = sum_i dY[i][j] (rows in order)
__global__ void k_colsum(const float* __restrict__ dY, int n, int N, float* __restrict__ db) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += dY[(size_t)i * N + j];
    db[j] = s;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t count, float lr, float c1, float c2) {
  constexpr float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    p[e] -= lr * (me * c1) / (sqrtf(ve * c2) + eps);
  }
}

// minibatch rows drawn with replacement: row i of the batch = sample
// floor(u(seed, step * batch + i) * n)
__global__ void k_gather_batch(const float* __restrict__ X, const float* __restrict__ T, int64_t n, int n_in,
                               int n_out, int batch, uint64_t seed, int64_t step, float* __restrict__ Xb,
                               float* __restrict__ Tb) {
  const int i = blockIdx.x;
  if (i >= batch) return;
  int64_t src = (int64_t)(unit_hash(seed, (uint64_t)(step * batch + i)) * (double)n);
  if (src >= n) src = n - 1;
  for (int k = threadIdx.x; k < n_in; k += blockDim.x) Xb[(size_t)i * n_in + k] = X[(size_t)src * n_in + k];
  for (int k = threadIdx.x; k < n_out; k += blockDim.x) Tb[(size_t)i * n_out + k] = T[(size_t)src * n_out + k];
}

inline int nblocks(int64_t count) { return (int)std::min<int64_t>((count + 255) / 256, 152 * 16); }

// ---------------------------------------------------------------- MPS rows
// padded network site [16][chi][chi] <-> solver site [p][chiL][chiR]
template <typename T, typename TO>
__global__ void k_export_row(DevMPS<T> mps, int row, int cols, int chi, TO* __restrict__ out) {
  const size_t per = (size_t)MAXP * chi * chi;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per * cols; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / per);
    const size_t f = e % per;
    const int s = (int)(f / ((size_t)chi * chi)), a = (int)((f / chi) % chi), ap = (int)(f % chi);
    const int* dA = mps.dimA + (row * cols + j) * 3;
    TO v = TO(0);
    if (s < dA[0] && a < dA[1] && ap < dA[2])
      v = (TO)mps.A[(size_t)(row * cols + j) * mps.site_stride + ((size_t)s * dA[1] + a) * dA[2] + ap];
    out[e] = v;
  }
}

template <typename T>
__global__ void k_ws_scatter(const float* __restrict__ Y, int chi, int cols, DevMPS<T> mps, int row) {
  const size_t per = (size_t)MAXP * chi * chi;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per * cols; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / per);
    const size_t f = e % per;
    const int s = (int)(f / ((size_t)chi * chi)), a = (int)((f / chi) % chi), ap = (int)(f % chi);
    const int* dA = mps.dimA + (row * cols + j) * 3;
    if (s < dA[0] && a < dA[1] && ap < dA[2])
      mps.A[(size_t)(row * cols + j) * mps.site_stride + ((size_t)s * dA[1] + a) * dA[2] + ap] = (T)Y[e];
  }
}

// Sign gauge of an exported row (padded layout, one block): for j = cols-1
// .. 1, every left-bond row a of site j whose largest-magnitude entry (first
// in (s, a') order on ties) is negative is negated with column a of site
// j-1.  One warp per row a.
template <typename TO>
__global__ void __launch_bounds__(1024) k_sign_fix(TO* __restrict__ out, const int* __restrict__ dims, int cols,
                                                   int chi) {
  const size_t per = (size_t)MAXP * chi * chi;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = cols - 1; j >= 1; --j) {
    const int p = dims[j * 3 + 0], chiL = dims[j * 3 + 1], chiR = dims[j * 3 + 2];
    const int pp = dims[(j - 1) * 3 + 0], chiLp = dims[(j - 1) * 3 + 1];
    TO* S = out + (size_t)j * per;
    TO* Sp = out + (size_t)(j - 1) * per;
    for (int a = wid; a < chiL; a += nw) {
      double best = -1.0;
      int bi = 1 << 30;
      double bv = 0.0;
      for (int e = lane; e < p * chiR; e += 32) {
        const int s = e / chiR, ap = e % chiR;
        const double v = (double)S[((size_t)s * chi + a) * chi + ap];
        const double m = fabs(v);
        if (m > best || (m == best && e < bi)) {
          best = m;
          bi = e;
          bv = v;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
          bv = ov;
        }
      }
      if (bv < 0.0) {
        for (int e = lane; e < p * chiR; e += 32) {
          const int s = e / chiR, ap = e % chiR;
          TO* x = S + ((size_t)s * chi + a) * chi + ap;
          *x = -*x;
        }
        for (int e = lane; e < pp * chiLp; e += 32) {
          const int s = e / chiLp, b = e % chiLp;
          TO* x = Sp + ((size_t)s * chi + b) * chi + a;
          *x = -*x;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------- internal API
size_t mlp_infer_elems(const spg_mlp* m, int n) { return (size_t)n * (2 * m->n_hidden + m->n_out); }

cudaError_t mlp_infer_bf16(const spg_mlp* m, const float* X, int n, float* work, float* Y, cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;  // not part of a grouped solve
  const __nv_bfloat16* pb = static_cast<const __nv_bfloat16*>(m->pbf);
  const int I = m->n_in, H = m->n_hidden, O = m->n_out;
  float* H1 = work;
  float* H2 = H1 + (size_t)n * H;
  cudaError_t e;
  if ((e = gemm_mlp<false, true, __nv_bfloat16, true>(n, H, I, X, I, pb + m->oW1, I, H1, H, m->p + m->ob1, 1, st)))
    return e;
  if ((e = gemm_mlp<false, true, __nv_bfloat16, true>(n, H, H, H1, H, pb + m->oW2, H, H2, H, m->p + m->ob2, 1, st)))
    return e;
  return gemm_mlp<false, true, __nv_bfloat16, true>(n, O, H, H2, H, pb + m->oW3, H, Y, O, m->p + m->ob3, 0, st);
}

template <typename T>
cudaError_t launch_ws_scatter(const float* Y, int chi, int cols, DevMPS<T> mps, int row, cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;  // not part of a grouped solve
  count_launches("k_ws_scatter", st);
  const int64_t cnt = (int64_t)MAXP * chi * chi * cols;
  k_ws_scatter<T><<<nblocks(cnt), 256, 0, st>>>(Y, chi, cols, mps, row);
  return cudaGetLastError();
}
template cudaError_t launch_ws_scatter<float>(const float*, int, int, DevMPS<float>, int, cudaStream_t);
template cudaError_t launch_ws_scatter<double>(const float*, int, int, DevMPS<double>, int, cudaStream_t);

template <typename T>
cudaError_t launch_export_row(DevMPS<T> mps, int row, int cols, int chi, T* out, const int* dims_dev, int fix_signs,
                              cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;  // not part of a grouped solve
  count_launches("k_export_row", st);
  const int64_t cnt = (int64_t)MAXP * chi * chi * cols;
  k_export_row<T, T><<<nblocks(cnt), 256, 0, st>>>(mps, row, cols, chi, out);
  if (fix_signs) {
    count_launches("k_sign_fix", st);
    k_sign_fix<T><<<1, 1024, 0, st>>>(out, dims_dev, cols, chi);
  }
  return cudaGetLastError();
}
template cudaError_t launch_export_row<float>(DevMPS<float>, int, int, int, float*, const int*, int, cudaStream_t);
template cudaError_t launch_export_row<double>(DevMPS<double>, int, int, int, double*, const int*, int,
                                               cudaStream_t);

int mlp_setup(spg_mlp* m) {
  const int64_t I = m->n_in, H = m->n_hidden, O = m->n_out;
  m->oW1 = 0;
  m->ob1 = m->oW1 + H * I;
  m->oW2 = m->ob1 + H;
  m->ob2 = m->oW2 + H * H;
  m->oW3 = m->ob2 + H;
  m->ob3 = m->oW3 + O * H;
  m->n_params = m->ob3 + O;
  const size_t np = (size_t)m->n_params;
  if (cudaMalloc(&m->p, 4 * np * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return SPG_ENOMEM;
  }
  m->g = m->p + np;
  m->m = m->g + np;
  m->v = m->m + np;
  if (cudaMalloc(&m->pbf, np * sizeof(__nv_bfloat16)) != cudaSuccess) {
    cudaGetLastError();
    return SPG_ENOMEM;
  }
  return SPG_OK;
}

static cudaError_t refresh_bf16(spg_mlp* m) {
  count_launches("k_to_bf16", m->stream);
  k_to_bf16<<<nblocks(m->n_params), 256, 0, m->stream>>>(m->p, static_cast<__nv_bfloat16*>(m->pbf), m->n_params);
  return cudaGetLastError();
}

int mlp_init_params(spg_mlp* m, uint64_t seed) {
  count_launches("k_mlp_init", m->stream);
  k_mlp_init<<<nblocks(m->n_params), 256, 0, m->stream>>>(m->p, m->n_params, m->oW1, m->ob1, m->oW2, m->ob2, m->oW3,
                                                          m->ob3, m->n_in, m->n_hidden, seed);
  if (cudaMemsetAsync(m->m, 0, 2 * sizeof(float) * (size_t)m->n_params, m->stream) != cudaSuccess) return SPG_ECUDA;
  if (refresh_bf16(m) != cudaSuccess) return SPG_ECUDA;
  m->t = 0;
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? SPG_OK : SPG_ECUDA;
}

// Scratch of one call on n samples (offsets in floats, 256-byte aligned):
// activations H1, H2 [n][H], outputs / output gradients Y [n][O], the
// loss's per-block partial sums (FP64), dH2, dH1 [n][H], the gathered
// minibatch Xb [n][I], Tb [n][O] (training only) and the loss slot (FP64).
struct BpLayout {
  size_t H1, H2, Y, part, dH2, dH1, Xb, Tb, loss, total;
};
static BpLayout bp_layout(const spg_mlp* m, int n, bool batch) {
  const size_t I = m->n_in, H = m->n_hidden, O = m->n_out, N = (size_t)n;
  auto al = [](size_t x) { return (x + 63) & ~size_t(63); };
  BpLayout L{};
  size_t o = 0;
  L.H1 = o;
  o = al(o + N * H);
  L.H2 = o;
  o = al(o + N * H);
  L.Y = o;
  o = al(o + N * O);
  L.part = o;
  o = al(o + 2 * 1024);
  L.dH2 = o;
  o = al(o + N * H);
  L.dH1 = o;
  o = al(o + N * H);
  if (batch) {
    L.Xb = o;
    o = al(o + N * I);
    L.Tb = o;
    o = al(o + N * O);
  }
  L.loss = o;
  o = al(o + 2);
  L.total = o;
  return L;
}

static float* mlp_scratch(spg_mlp* m, size_t need) {
  if (m->scratch_elems < need) {
    if (m->scratch) cudaFree(m->scratch);
    m->scratch = nullptr;
    m->scratch_elems = 0;
    if (cudaMalloc(&m->scratch, need * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    m->scratch_elems = need;
  }
  return m->scratch;
}

// forward (FP32, keeping H1, H2), loss and gradients of n samples into m->g;
// the loss (0.5/n sum of squares) is written (or added) to the loss slot
static cudaError_t mlp_backprop(spg_mlp* m, const float* X, const float* T, int n, float* w, const BpLayout& L,
                                int accumulate) {
  const int I = m->n_in, H = m->n_hidden, O = m->n_out;
  cudaStream_t st = m->stream;
  float* H1 = w + L.H1;
  float* H2 = w + L.H2;
  float* Y = w + L.Y;
  double* part = reinterpret_cast<double*>(w + L.part);
  float* dH2 = w + L.dH2;
  float* dH1 = w + L.dH1;
  double* loss_dev = reinterpret_cast<double*>(w + L.loss);
  cudaError_t e;
  if ((e = gemm_mlp<false, true, float, false>(n, H, I, X, I, m->p + m->oW1, I, H1, H, m->p + m->ob1, 1, st))) return e;
  if ((e = gemm_mlp<false, true, float, false>(n, H, H, H1, H, m->p + m->oW2, H, H2, H, m->p + m->ob2, 1, st))) return e;
  if ((e = gemm_mlp<false, true, float, false>(n, O, H, H2, H, m->p + m->oW3, H, Y, O, m->p + m->ob3, 0, st))) return e;
  const int64_t cnt = (int64_t)n * O;
  const int nb = std::min(nblocks(cnt), 1024);
  count_launches("k_loss_dy", st);
  k_loss_dy<<<nb, 256, 0, st>>>(Y, T, cnt, 1.f / (float)n, part);
  count_launches("k_loss_sum", st);
  k_loss_sum<<<1, 32, 0, st>>>(part, nb, 1.0 / n, loss_dev, accumulate);
  const float* dY = Y;
  // output layer: dW3 = dY^T H2, db3 = column sums of dY, dH2 = dY W3
  if ((e = gemm_mlp<true, false, float, false>(O, H, n, dY, O, H2, H, m->g + m->oW3, H, nullptr, 0, st))) return e;
  count_launches("k_colsum", st);
  k_colsum<<<(O + 255) / 256, 256, 0, st>>>(dY, n, O, m->g + m->ob3);
  if ((e = gemm_mlp<false, false, float, false>(n, H, O, dY, O, m->p + m->oW3, H, dH2, H, nullptr, 0, st))) return e;
  count_launches("k_tanh_bwd", st);
  k_tanh_bwd<<<nblocks((int64_t)n * H), 256, 0, st>>>(dH2, H2, (int64_t)n * H);
  // second layer
  if ((e = gemm_mlp<true, false, float, false>(H, H, n, dH2, H, H1, H, m->g + m->oW2, H, nullptr, 0, st))) return e;
  count_launches("k_colsum", st);
  k_colsum<<<(H + 255) / 256, 256, 0, st>>>(dH2, n, H, m->g + m->ob2);
  if ((e = gemm_mlp<false, false, float, false>(n, H, H, dH2, H, m->p + m->oW2, H, dH1, H, nullptr, 0, st))) return e;
  count_launches("k_tanh_bwd", st);
  k_tanh_bwd<<<nblocks((int64_t)n * H), 256, 0, st>>>(dH1, H1, (int64_t)n * H);
  // first layer
  if ((e = gemm_mlp<true, false, float, false>(H, I, n, dH1, H, X, I, m->g + m->oW1, I, nullptr, 0, st))) return e;
  count_launches("k_colsum", st);
  k_colsum<<<(H + 255) / 256, 256, 0, st>>>(dH1, n, H, m->g + m->ob1);
  return cudaGetLastError();
}

}  // namespace spg

using namespace spg;

#define WS_CK(call)                       \
  do {                                    \
    if ((call) != cudaSuccess) {          \
      cudaGetLastError();                 \
      return SPG_ECUDA;                   \
    }                                     \
  } while (0)

extern "C" {

void spg_mlp_destroy(spg_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaStreamSynchronize(m->stream);
  if (m->p) cudaFree(m->p);
  if (m->pbf) cudaFree(m->pbf);
  if (m->scratch) cudaFree(m->scratch);
  spg_ctx* ctx = m->ctx;
  delete m;
  if (ctx) ctx_release(ctx);
}

int64_t spg_mlp_num_params(const spg_mlp* m) { return m ? m->n_params : 0; }

int spg_mlp_params(spg_mlp* m, float* get_host, const float* set_host) {
  if (!m) return SPG_EINVAL;
  WS_CK(cudaSetDevice(m->device));
  const size_t bytes = sizeof(float) * (size_t)m->n_params;
  if (get_host) {
    WS_CK(cudaMemcpyAsync(get_host, m->p, bytes, cudaMemcpyDeviceToHost, m->stream));
    WS_CK(cudaStreamSynchronize(m->stream));
  }
  if (set_host) {
    WS_CK(cudaMemcpyAsync(m->p, set_host, bytes, cudaMemcpyHostToDevice, m->stream));
    WS_CK(cudaMemsetAsync(m->m, 0, 2 * bytes, m->stream));
    WS_CK(refresh_bf16(m));
    m->t = 0;
    WS_CK(cudaStreamSynchronize(m->stream));
  }
  return SPG_OK;
}

int spg_mlp_forward(spg_mlp* m, const float* X, int32_t n, float* Y, int32_t bf16) {
  if (!m || !X || !Y || n < 1 || n > 65536) return SPG_EINVAL;
  WS_CK(cudaSetDevice(m->device));
  const BpLayout L = bp_layout(m, n, false);
  float* w = mlp_scratch(m, L.total);
  if (!w) return SPG_ENOMEM;
  const int I = m->n_in, H = m->n_hidden, O = m->n_out;
  cudaStream_t st = m->stream;
  if (bf16) {
    WS_CK(mlp_infer_bf16(m, X, n, w, Y, st));
  } else {
    float* H1 = w + L.H1;
    float* H2 = w + L.H2;
    WS_CK((gemm_mlp<false, true, float, false>(n, H, I, X, I, m->p + m->oW1, I, H1, H, m->p + m->ob1, 1, st)));
    WS_CK((gemm_mlp<false, true, float, false>(n, H, H, H1, H, m->p + m->oW2, H, H2, H, m->p + m->ob2, 1, st)));
    WS_CK((gemm_mlp<false, true, float, false>(n, O, H, H2, H, m->p + m->oW3, H, Y, O, m->p + m->ob3, 0, st)));
  }
  WS_CK(cudaStreamSynchronize(st));
  return SPG_OK;
}

int spg_mlp_loss_grad(spg_mlp* m, const float* X, const float* T, int32_t n, double* loss, float* grad_host) {
  if (!m || !X || !T || n < 1 || n > 4096) return SPG_EINVAL;
  WS_CK(cudaSetDevice(m->device));
  const BpLayout L = bp_layout(m, n, false);
  float* w = mlp_scratch(m, L.total);
  if (!w) return SPG_ENOMEM;
  double* ldev = reinterpret_cast<double*>(w + L.loss);
  WS_CK(mlp_backprop(m, X, T, n, w, L, 0));
  double l = 0.0;
  WS_CK(cudaMemcpyAsync(&l, ldev, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  if (grad_host)
    WS_CK(cudaMemcpyAsync(grad_host, m->g, sizeof(float) * (size_t)m->n_params, cudaMemcpyDeviceToHost, m->stream));
  WS_CK(cudaStreamSynchronize(m->stream));
  if (loss) *loss = l;
  return SPG_OK;
}

int spg_mlp_train(spg_mlp* m, const float* X, const float* T, int64_t n, int32_t batch, int32_t steps, double lr,
                  uint64_t seed, double* loss) {
  if (!m || !X || !T || n < 1 || batch < 1 || batch > 4096 || steps < 0 || !(lr > 0.0)) return SPG_EINVAL;
  WS_CK(cudaSetDevice(m->device));
  const BpLayout L = bp_layout(m, batch, true);
  float* w = mlp_scratch(m, L.total);
  if (!w) return SPG_ENOMEM;
  float* Xb = w + L.Xb;
  float* Tb = w + L.Tb;
  double* ldev = reinterpret_cast<double*>(w + L.loss);
  cudaStream_t st = m->stream;
  WS_CK(cudaMemsetAsync(ldev, 0, sizeof(double), st));
  const int tail = std::min(steps, 50);
  for (int s = 0; s < steps; ++s) {
    count_launches("k_gather_batch", st);
    k_gather_batch<<<batch, 256, 0, st>>>(X, T, n, m->n_in, m->n_out, batch, seed, (int64_t)s, Xb, Tb);
    WS_CK(mlp_backprop(m, Xb, Tb, batch, w, L, s >= steps - tail ? 1 : 0));
    m->t += 1;
    const double c1 = 1.0 / (1.0 - std::pow(0.9, m->t)), c2 = 1.0 / (1.0 - std::pow(0.999, m->t));
    count_launches("k_adam", st);
    k_adam<<<nblocks(m->n_params), 256, 0, st>>>(m->p, m->g, m->m, m->v, m->n_params, (float)lr, (float)c1, (float)c2);
    WS_CK(cudaGetLastError());
  }
  WS_CK(refresh_bf16(m));
  double l = 0.0;
  WS_CK(cudaMemcpyAsync(&l, ldev, sizeof(double), cudaMemcpyDeviceToHost, st));
  WS_CK(cudaStreamSynchronize(st));
  if (loss) *loss = tail > 0 ? l / tail : 0.0;
  return SPG_OK;
}

}  // extern "C"
