// Tensor-core products of the truncated SVD (S3) on large zipper matrices:
// D = A B^T with A [M x K] and B [N x K] both K-major FP32, on the 5th-gen
// tensor cores (tcgen05.mma kind::tf32, accumulator in tensor memory,
// operands brought to shared memory by TMA with 128-byte swizzle).
//
// TF32 keeps 10 mantissa bits, too few for the truncation (a product with
// ~5e-4 relative error shifts the kept singular vectors).  Each operand is
// therefore split into a TF32 high part and the FP32 remainder, x = hi + lo
// (hi = x rounded to TF32, lo = x - hi exactly), and D accumulates
// hi*hi + hi*lo + lo*hi in FP32: the dropped lo*lo term and the TF32 reading
// of lo are below 2^-21 relative, i.e. FP32-level products at three tensor
// passes per multiply-add (the split-precision technique of Ootomo & Yokota,
// "Recovering single precision accuracy from Tensor Cores while surpassing
// the FP32 theoretical peak performance", IJHPCA 2022).
//
// Paper: Sec. 3.1 (MpsContractor(SVDTruncate, ...)) and Sec. 2 (boundary-MPS
// contraction); the paper runs these products through CUDA.jl / cuBLAS.
//
// One CTA of 4 warps computes a 128 x BN tile of D over a range of K:
// warp 0 (one thread) issues the TMA loads of a 3-stage ring, warp 1 (one
// thread) issues the MMAs and commits each stage back to the loader, warp 2
// owns the tensor-memory allocation, and all four warps drain the
// accumulator (warp w reads TMEM lanes 32w..32w+31 = rows of the tile).
// Every wait on an mbarrier is bounded; on a timeout the kernel records
// ERR_TIMEOUT, waits (bounded) for the loads it already issued, releases its
// tensor memory and returns.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "spg_internal.h"
#include "tc_ptx.h"

namespace spg {

namespace {

constexpr int UM = 128;      // rows of A per CTA (tcgen05 M)
constexpr int UKF = 32;      // K floats per stage: one 128-byte swizzle row
constexpr int STAGES = 3;
using tc::mbar_wait;
using tc::smem_u32;
using tc::sw128_desc;
using tc::tma_load_3d;
using tc::umma_commit;
using tc::umma_tf32;

// D tile (128 x BN) of A B^T over k-blocks [kb0, kb1) of 32, written
// transposed: out[c * ldo + r] for r < M, c < N.
template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_umma_tf32x3(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                  const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, int M, int N,
                  int nkb, int nsplit, float* out, int ldo, size_t split_stride, int* err, size_t zs) {
  out = zp(out, zs);
  err = zp(err, zs);
  constexpr uint32_t A_BYTES = UM * UKF * 4;
  constexpr uint32_t B_BYTES = BN * UKF * 4;
  constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t TM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tiles (the swizzle atom)
  const uint32_t base0 = smem_u32(smem_raw);
  const uint32_t tiles = (base0 + 1023u) & ~1023u;
  __shared__ __align__(8) unsigned long long bars[2 * STAGES + 1];
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * UM;
  const int split = blockIdx.y;
  const int kb0 = (int)((long)nkb * split / nsplit), kb1 = (int)((long)nkb * (split + 1) / nsplit);
  const int nk = kb1 - kb0;
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[STAGES]), done = smem_u32(&bars[2 * STAGES]);
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * STAGES + 1; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[s])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // loader
    int issued = 0;
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES) ok = mbar_wait(empty0 + 8 * s, ((i / STAGES) - 1) & 1, err);
      if (!ok) break;
      const uint32_t fb = full0 + 8 * s;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES) : "memory");
      const uint32_t st = tiles + s * STAGE_BYTES;
      const int kc = (kb0 + i) * UKF;
      const int z = (int)blockIdx.z;
      tma_load_3d(st, &tAh, kc, m0, z, fb);
      tma_load_3d(st + A_BYTES, &tAl, kc, m0, z, fb);
      tma_load_3d(st + 2 * A_BYTES, &tBh, kc, 0, z, fb);
      tma_load_3d(st + 2 * A_BYTES + B_BYTES, &tBl, kc, 0, z, fb);
      issued = i + 1;
    }
    // every issued load lands in this CTA's shared memory before it exits,
    // also when a wait here or in the MMA issuer gave up: wait (bounded) for
    // the last load issued into each stage (at once true when it was consumed)
    for (int s = 0; s < STAGES; ++s) {
      int last = issued - 1;
      while (last >= 0 && last % STAGES != s) --last;
      if (last >= 0) mbar_wait(full0 + 8 * s, (last / STAGES) & 1, err);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 K-steps of 8 per stage, three products each
    constexpr uint32_t idesc = tc::tf32_idesc(UM, BN);
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % STAGES;
      ok = mbar_wait(full0 + 8 * s, (i / STAGES) & 1, err);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = tiles + s * STAGE_BYTES;
      const uint64_t ah = sw128_desc(st), al = sw128_desc(st + A_BYTES);
      const uint64_t bh = sw128_desc(st + 2 * A_BYTES), bl = sw128_desc(st + 2 * A_BYTES + B_BYTES);
      for (int kk = 0; kk < UKF / 8; ++kk) {
        const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 8 floats = 32 bytes further along the row
        umma_tf32(tmem, ah + o, bh + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        umma_tf32(tmem, ah + o, bl + o, idesc, 1u);
        umma_tf32(tmem, al + o, bh + o, idesc, 1u);
      }
      umma_commit(empty0 + 8 * s);
    }
    umma_commit(done);
  }
  __syncwarp();
  // epilogue: every warp drains its 32 accumulator lanes
  const bool drained = mbar_wait(done, 0, err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (drained && nk > 0) {
    const int r = m0 + warp * 32 + lane;
    float* o = out + (size_t)split * split_stride;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < M)
        for (int q = 0; q < 16; ++q)
          if (c0 + q < N) o[(size_t)(c0 + q) * ldo + r] = __uint_as_float(v[q]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS) : "memory");
}

// The bounded wait of the kernels above on an mbarrier that nothing arrives
// on: it must give up after `limit` polls, record ERR_TIMEOUT and return
// (the failure path of every bounded wait, exercised without any copy or
// tensor memory in flight).
__global__ void k_wait_check(long limit, int* err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, err, limit);
}

using tc::split_tf32;  // rows of the split outputs are padded with zeros to kp entries

// out rows r < rows, k < kp: value X[r * ldx + k] (k < cols), else 0.
__global__ void k_split(const float* __restrict__ X, int rows, int cols, int ldx, int kp, float* __restrict__ hi,
                        float* __restrict__ lo, size_t zs) {
  X = zp(X, zs);
  hi = zp(hi, zs);
  lo = zp(lo, zs);
  const size_t tot = (size_t)rows * kp;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / kp), k = (int)(e % kp);
    float h = 0.f, l = 0.f;
    if (k < cols) split_tf32(X[(size_t)r * ldx + k], h, l);
    hi[e] = h;
    lo[e] = l;
  }
}

// Transposed: out rows r < cols_in (columns of X), k < kp: X[k * ldx + r] for
// k < rows_in, else 0; 32 x 32 tiles through shared memory.
__global__ void k_split_t(const float* __restrict__ X, int rows_in, int cols_in, int ldx, int kp,
                          float* __restrict__ hi, float* __restrict__ lo, size_t zs) {
  X = zp(X, zs);
  hi = zp(hi, zs);
  lo = zp(lo, zs);
  __shared__ float t[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;  // k: rows of X, r: columns of X
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int k = k0 + y, r = r0 + threadIdx.x;
    t[y][threadIdx.x] = (k < rows_in && r < cols_in) ? X[(size_t)k * ldx + r] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, k = k0 + threadIdx.x;
    if (r < cols_in && k < kp) {
      float h, l;
      split_tf32(t[threadIdx.x][y], h, l);
      hi[(size_t)r * kp + k] = h;
      lo[(size_t)r * kp + k] = l;
    }
  }
}

__global__ void k_sum_splits(const float* __restrict__ part, int nsplit, size_t stride, int n, int ldo, int rows,
                             float* __restrict__ out, size_t zs) {
  part = zp(part, zs);
  out = zp(out, zs);
  const size_t tot = (size_t)n * rows;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / rows), r = (int)(e % rows);
    float a = 0.f;
    for (int s = 0; s < nsplit; ++s) a += part[s * stride + (size_t)c * ldo + r];
    out[(size_t)c * ldo + r] = a;
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// K-major [rows x kp] FP32 matrix (kp a multiple of 32), box of 32 x box_rows
// with 128-byte swizzle; rows past the end read as zeros.  The outer
// dimension counts the instances of a lockstep group (zs bytes apart; one
// instance without a group).
bool make_map(CUtensorMap* map, const float* base, int rows, int kp, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const size_t mat = ((size_t)rows * kp * 4 + 15) / 16 * 16;
  const size_t z = zn() > 1 ? zs() : mat;
  if (z % 16 != 0 || z < mat) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)zn()};
  const cuuint64_t strides[2] = {(cuuint64_t)kp * 4, (cuuint64_t)z};
  const cuuint32_t box[3] = {(cuuint32_t)UKF, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_bn(const CUtensorMap* m, int M, int N, int nkb, int nsplit, float* out, int ldo, size_t sstride,
                      int* err, cudaStream_t st) {
  constexpr size_t smem = (size_t)STAGES * (2 * UM * UKF * 4 + 2 * BN * UKF * 4) + 1024;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_umma_tf32x3<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  dim3 grid((M + UM - 1) / UM, nsplit, zn());
  k_umma_tf32x3<BN><<<grid, 128, smem, st>>>(m[0], m[1], m[2], m[3], M, N, nkb, nsplit, out, ldo, sstride, err,
                                             zs());
  return cudaGetLastError();
}

}  // namespace

// A tensor map of a K-major FP32 matrix for the tcgen05 kernels of other
// translation units (the layout and instance rules of make_map).
bool make_f32_tensor_map(void* map, const float* base, int rows, int kp, int box_rows) {
  return make_map(static_cast<CUtensorMap*>(map), base, rows, kp, box_rows);
}

size_t tc_gemm_elems(int m, int n, int s) {
  const size_t mp = ((size_t)m + 31) / 32 * 32, np = ((size_t)n + 31) / 32 * 32;
  // A hi/lo of M (m x np) and of M^T (n x mp), B hi/lo (up to SMAX rows of
  // max(mp, np)), split partials (16 x SMAX x max(m, n))
  (void)s;
  return 2 * (size_t)m * np + 2 * (size_t)n * mp + 2 * (size_t)SMAX * std::max(mp, np) +
         16 * (size_t)SMAX * std::max(m, n) + 1024;
}

bool tc_gemm_eligible(int m, int n, int s) {
  return s % 16 == 0 && s >= 16 && s <= 128 && m >= 256 && n >= 256 && (double)m * n * s >= (double)(1 << 22);
}

TcGemm::TcGemm(float* work, size_t elems, const float* M, int m, int n, int* err, cudaStream_t st)
    : m_(m), n_(n), err_(err), st_(st) {
  mp_ = (m + 31) / 32 * 32;
  np_ = (n + 31) / 32 * 32;
  float* p = work;
  Mh_ = p;
  p += (size_t)m * np_;
  Ml_ = p;
  p += (size_t)m * np_;
  MTh_ = p;
  p += (size_t)n * mp_;
  MTl_ = p;
  p += (size_t)n * mp_;
  Bh_ = p;
  Bl_ = p + (size_t)SMAX * std::max(mp_, np_);
  part_ = Bl_ + (size_t)SMAX * std::max(mp_, np_);
  (void)elems;
  const size_t tot = (size_t)m * np_;
  if (!zok(work, M, err, part_ + 16 * (size_t)SMAX * std::max(m, n) - 1)) return;
  count_launches("k_split", st);
  k_split<<<dim3((int)std::min<size_t>((tot + 255) / 256, 8192), 1, zn()), 256, 0, st>>>(M, m, n, n, np_, Mh_, Ml_,
                                                                                         zs());
  count_launches("k_split_t", st);
  dim3 g((mp_ + 31) / 32, (n + 31) / 32, zn());
  k_split_t<<<g, dim3(32, 8), 0, st>>>(M, m, n, n, mp_, MTh_, MTl_, zs());
}

// out[j * ldo + i] = sum_k A[i][k] B[j][k]: the rows of out are the s
// columns of the product (Yt = (M Z)^T with trans == false, Zt = (M^T Y)^T
// with trans == true); Bt: the s x K operand (Zt or Yt, row stride K).
cudaError_t TcGemm::run(bool trans, const float* Bt, int s, float* out) {
  const int rowsA = trans ? n_ : m_;
  const int K = trans ? m_ : n_;
  const int kp = trans ? mp_ : np_;
  const float* Ah = trans ? MTh_ : Mh_;
  const float* Al = trans ? MTl_ : Ml_;
  const size_t tot = (size_t)s * kp;
  ZOK(Bt, out);
  count_launches("k_split", st_);
  k_split<<<dim3((int)std::min<size_t>((tot + 255) / 256, 8192), 1, zn()), 256, 0, st_>>>(Bt, s, K, K, kp, Bh_,
                                                                                           Bl_, zs());
  CUtensorMap maps[4];
  if (!make_map(&maps[0], Ah, rowsA, kp, UM) || !make_map(&maps[1], Al, rowsA, kp, UM) ||
      !make_map(&maps[2], Bh_, s, kp, s) || !make_map(&maps[3], Bl_, s, kp, s))
    return cudaErrorInvalidValue;
  const int nkb = kp / UKF;
  const int mt = (rowsA + UM - 1) / UM;
  int nsplit = 1;
  while (mt * nsplit < 148 && nsplit < 16 && nkb / (2 * nsplit) >= 8) nsplit *= 2;
  float* dst = nsplit > 1 ? part_ : out;
  const size_t sstride = (size_t)s * rowsA;
  const double fl = 2.0 * rowsA * s * K;
  cudaError_t e;
  count_launches("k_umma_tf32x3", st_, fl);
  switch (s) {
    case 16: e = launch_bn<16>(maps, rowsA, s, nkb, nsplit, dst, rowsA, sstride, err_, st_); break;
    case 32: e = launch_bn<32>(maps, rowsA, s, nkb, nsplit, dst, rowsA, sstride, err_, st_); break;
    case 48: e = launch_bn<48>(maps, rowsA, s, nkb, nsplit, dst, rowsA, sstride, err_, st_); break;
    case 64: e = launch_bn<64>(maps, rowsA, s, nkb, nsplit, dst, rowsA, sstride, err_, st_); break;
    case 80: e = launch_bn<80>(maps, rowsA, s, nkb, nsplit, dst, rowsA, sstride, err_, st_); break;
    case 96: e = launch_bn<96>(maps, rowsA, s, nkb, nsplit, dst, rowsA, sstride, err_, st_); break;
    case 112: e = launch_bn<112>(maps, rowsA, s, nkb, nsplit, dst, rowsA, sstride, err_, st_); break;
    case 128: e = launch_bn<128>(maps, rowsA, s, nkb, nsplit, dst, rowsA, sstride, err_, st_); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (nsplit > 1) {
    count_launches("k_sum_splits", st_);
    k_sum_splits<<<dim3((int)std::min<size_t>((sstride + 255) / 256, 4096), 1, zn()), 256, 0, st_>>>(
        part_, nsplit, sstride, s, rowsA, rowsA, out, zs());
  }
  return cudaGetLastError();
}

cudaError_t launch_wait_check(long limit, int* err, cudaStream_t st) {
  if (zn() != 1) return cudaErrorInvalidValue;
  count_launches("k_wait_check", st);
  k_wait_check<<<1, 32, 0, st>>>(limit, err);
  return cudaGetLastError();
}

}  // namespace spg
