// Learned initial-iterate proposal: patch features, targets, proposal
// scatter, and a 3-layer MLP trained with hand-written bfloat16 tensor-core
// GEMMs (tcgen05.mma, FP32 accumulation in tensor memory) and Adam.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include "../../include/tmop.h"
#include "../../include/tmop_mlp.h"
#include "tmop_kparams.h"

namespace tmop {
namespace mlp {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------- patches
struct Grid2 {
  int k, nx, ny, Nx, Ny, ldx;
  const double* x;
  double xi[6];  // Gauss-Lobatto node positions of one element on [0,1] (reference lattice)
  __device__ __forceinline__ double at(int c, int gx, int gy) const { return x[(size_t)c * ldx + gy * Nx + gx]; }
  // x-direction reflection, gy in range
  __device__ __forceinline__ double qx(int c, int gx, int gy) const {
    if (gx < 0) return 2.0 * at(c, 0, gy) - at(c, -gx, gy);
    if (gx > Nx - 1) return 2.0 * at(c, Nx - 1, gy) - at(c, 2 * (Nx - 1) - gx, gy);
    return at(c, gx, gy);
  }
  __device__ __forceinline__ double pos(int c, int gx, int gy) const {
    if (gy < 0) return 2.0 * qx(c, gx, 0) - qx(c, gx, -gy);
    if (gy > Ny - 1) return 2.0 * qx(c, gx, Ny - 1) - qx(c, gx, 2 * (Ny - 1) - gy);
    return qx(c, gx, gy);
  }
};

// one warp per patch
__global__ void k_features(Grid2 G, int first, int count, bf16* feat, int ldf) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= count) return;
  const int e = first + warp, ex = e % G.nx, ey = e / G.nx, k = G.k;
  const int side = 3 * k + 1, nfeat = 2 * side * side;
  double c[2];
#pragma unroll
  for (int d = 0; d < 2; ++d)
    c[d] = 0.25 * (G.at(d, k * ex, k * ey) + G.at(d, k * ex + k, k * ey) + G.at(d, k * ex, k * ey + k) +
                   G.at(d, k * ex + k, k * ey + k));
  const double inv_h = (double)G.nx;
  bf16* row = feat + (size_t)warp * ldf;
  for (int f = lane; f < ldf; f += 32) {
    float v = 0.0f;
    if (f < nfeat) {
      const int d = f & 1, node = f >> 1, a = node % side, b = node / side;
      // position of this patch node in a uniform patch, relative to the centre
      // element's centre, in units of h
      const int ab = d == 0 ? a : b;
      const double ref = (double)(ab / k - 1) + G.xi[ab % k] - 0.5;
      v = (float)((G.pos(d, k * (ex - 1) + a, k * (ey - 1) + b) - c[d]) * inv_h - ref);
    }
    row[f] = __float2bfloat16_rn(v);
  }
}

__global__ void k_targets(Grid2 G0, const double* x1, int first, int count, float* T, int ldt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = G0.k, per = 2 * k * k;
  if (t >= count * per) return;
  const int p = t / per, f = t % per, e = first + p;
  const int d = f & 1, o = f >> 1, i = o % k, j = o / k;
  const int ex = e % G0.nx, ey = e / G0.nx;
  const size_t node = (size_t)(k * ey + j) * G0.Nx + k * ex + i;
  T[(size_t)p * ldt + f] = (float)((x1[(size_t)d * G0.ldx + node] - G0.x[(size_t)d * G0.ldx + node]) * G0.nx);
}

__global__ void k_apply(Grid2 G0, const uint8_t* fixed, const float* Y, int ldy, double scale, double* xo) {
  const size_t nn = (size_t)G0.Nx * G0.Ny;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= 2 * nn) return;
  const int d = (int)(t / nn);
  const size_t node = t % nn;
  const int gx = (int)(node % G0.Nx), gy = (int)(node / G0.Nx), k = G0.k;
  const size_t dof = (size_t)d * G0.ldx + node;
  double v = G0.x[dof];
  const bool owned = gx < k * G0.nx && gy < k * G0.ny;
  if (owned && !(fixed && fixed[dof])) {
    const int e = (gy / k) * G0.nx + gx / k, i = gx % k, j = gy % k;
    v += scale * (double)Y[(size_t)e * ldy + 2 * (j * k + i) + d] / G0.nx;
  }
  xo[dof] = v;
}

// ---------------------------------------------------------------- GEMM (tcgen05)
// C[m][n] = sum_k A(m,k) B(n,k) with A(m,k) = AK ? A[m*lda+k] : A[k*lda+m] and
// B(n,k) = BK ? B[n*ldb+k] : B[k*ldb+n], on the fifth-generation tensor cores.
// One CTA of 4 warps per 128 x 64 tile of C. K goes in chunks of 64: the
// threads stage the A and B chunks in shared memory in the K-major,
// unswizzled operand layout of tcgen05 (8-row x 16-byte core matrices,
// transposing operands that are stored MN-major), one thread issues four
// tcgen05.mma (kind::f16: bf16 inputs, FP32 accumulator in tensor memory,
// 128 lanes x 64 columns) and tcgen05.commit, which signals an mbarrier; at
// the end each warp reads its 32 accumulator lanes with tcgen05.ld for the
// epilogue. blockIdx.z splits K for the weight gradients (a small M x N grid
// over K = batch): each split writes its FP32 partial tile to a slice of a
// workspace, and k_splitk_sum adds the slices in split order.
// Requirements (checked by gemm()): M, N multiples of 64, K of 64, leading
// dimensions multiples of 8 (16-byte rows); rows of the last 128-row tile
// beyond M read as zero and are not stored.
constexpr int TM = 128, TN = 64, TK = 64;
static_assert((TM * TK / 8) % 128 == 0 && (TN * TK / 8) % 128 == 0, "chunk staging: whole passes of 128 threads");
constexpr uint32_t kTmemCols = 64;                    // FP32 accumulator columns (power of 2, >= 32)
constexpr long kMmaSpin = 1L << 20;                   // bound on the wait for one chunk's MMAs
enum { EPI_BIAS_RELU_BF16 = 0, EPI_BIAS_F32 = 1, EPI_MASK_BF16 = 2, EPI_F32 = 3 };

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a [rows][TK] tile in the core-matrix layout:
// core matrix (r / 8, k / 8) is 128 contiguous bytes, K-adjacent core matrices
// 128 B apart (leading byte offset), row-adjacent ones TK / 8 * 128 B apart
// (stride byte offset)
__device__ __forceinline__ int cm_off(int r, int k) {
  return ((r >> 3) * (TK >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bit
// 17, M / 16 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

template <bool AK, bool BK, int EPI>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, int kper, const bf16* __restrict__ A, int lda,
                                                 const bf16* __restrict__ B, int ldb, void* __restrict__ C, int ldc,
                                                 size_t split_stride, const float* __restrict__ bias,
                                                 const bf16* __restrict__ ref, int ldr, int* err) {
  // 24 KB of operands, padded to 26 KB so that at most 8 CTAs share an SM:
  // 8 x 64 accumulator columns = the SM's 512 columns of tensor memory
  __shared__ __align__(128) unsigned char sA[TM * TK * 2 + 2048];
  __shared__ __align__(128) unsigned char sB[TN * TK * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int kb = blockIdx.z * kper, ke = min(K, kb + kper);

  if (warp == 0) {  // the accumulator: 128 lanes x 64 FP32 columns of tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  bool ok = true;
  int chunk = 0;
  for (int k0 = kb; k0 < ke; k0 += TK, ++chunk) {
    // ---- stage the chunk (zero rows beyond M)
    // (compile-time trip counts: every thread issues all its loads of the chunk
    // before the stores that wait on them)
#pragma unroll
    for (int i = 0; i < TM * TK / 8 / 128; ++i) {
      const int c = tid + 128 * i;
      if (AK) {
        const int r = c / (TK / 8), kc = (c % (TK / 8)) * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (m0 + r < M) v = *reinterpret_cast<const uint4*>(&A[(size_t)(m0 + r) * lda + k0 + kc]);
        *reinterpret_cast<uint4*>(sA + cm_off(r, kc)) = v;
      } else {
        const int kk = c / (TM / 8), mc = (c % (TM / 8)) * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (m0 + mc < M) v = *reinterpret_cast<const uint4*>(&A[(size_t)(k0 + kk) * lda + m0 + mc]);
        const unsigned short* e = reinterpret_cast<const unsigned short*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) *reinterpret_cast<unsigned short*>(sA + cm_off(mc + j, kk)) = e[j];
      }
    }
#pragma unroll
    for (int i = 0; i < TN * TK / 8 / 128; ++i) {
      const int c = tid + 128 * i;
      if (BK) {
        const int r = c / (TK / 8), kc = (c % (TK / 8)) * 8;
        *reinterpret_cast<uint4*>(sB + cm_off(r, kc)) =
            *reinterpret_cast<const uint4*>(&B[(size_t)(n0 + r) * ldb + k0 + kc]);
      } else {
        const int kk = c / (TN / 8), nc = (c % (TN / 8)) * 8;
        const uint4 v = *reinterpret_cast<const uint4*>(&B[(size_t)(k0 + kk) * ldb + n0 + nc]);
        const unsigned short* e = reinterpret_cast<const unsigned short*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) *reinterpret_cast<unsigned short*>(sB + cm_off(nc + j, kk)) = e[j];
      }
    }
    // generic-proxy stores -> visible to the tensor core's (async proxy) reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < TK / 16; ++s) {  // K = 16 per instruction: two core matrices along K
        const uint64_t ad = umma_desc(saddr(sA) + s * 256, 128, (TK / 8) * 128);
        const uint64_t bd = umma_desc(saddr(sB) + s * 256, 128, (TK / 8) * 128);
        const uint32_t acc = (chunk > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&bar))
                   : "memory");
    }
    // the chunk's MMAs have read the staged operands (and written the accumulator)
    bool done = false;
    for (long i = 0; i < kMmaSpin && !done; ++i) done = mbar_try(&bar, (uint32_t)(chunk & 1));
    if (!done) ok = false;
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
  }
  tc_fence_after();
  if (ok && chunk > 0) {
    // ---- epilogue: warp w owns accumulator lanes (rows) 32 w .. 32 w + 31
    const int m = m0 + warp * 32 + lane;
#pragma unroll
    for (int cb = 0; cb < TN / 16; ++cb) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int n = n0 + cb * 16 + j;
          float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
          if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_BIAS_F32) {
            v0 += bias[n];
            v1 += bias[n + 1];
          }
          if (EPI == EPI_BIAS_RELU_BF16) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
          }
          if (EPI == EPI_MASK_BF16) {
            const __nv_bfloat162 rr = *reinterpret_cast<const __nv_bfloat162*>(&ref[(size_t)m * ldr + n]);
            if (!(__bfloat162float(rr.x) > 0.0f)) v0 = 0.0f;
            if (!(__bfloat162float(rr.y) > 0.0f)) v1 = 0.0f;
          }
          if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_BF16) {
            *reinterpret_cast<__nv_bfloat162*>(&reinterpret_cast<bf16*>(C)[(size_t)m * ldc + n]) =
                __floats2bfloat162_rn(v0, v1);
          } else {
            float* Cf = reinterpret_cast<float*>(C) + blockIdx.z * split_stride;
            *reinterpret_cast<float2*>(&Cf[(size_t)m * ldc + n]) = make_float2(v0, v1);
          }
        }
      }
    }
  }
  if (!ok) {
    // a wait gave up (not expected): report it, give the committed MMAs a
    // second bounded wait so that none still writes the accumulator when it
    // is freed, and fill this CTA's output tile with NaN so that no consumer
    // takes it for a product
    if (tid == 0) atomicExch(err, 1);
    bool done = false;
    for (long i = 0; i < kMmaSpin && !done; ++i) done = mbar_try(&bar, (uint32_t)(chunk & 1));
    const int m = m0 + warp * 32 + lane;
    if (m < M) {
      const float qnan = __uint_as_float(0x7fc00000u);
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + j;
        if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_BF16)
          reinterpret_cast<bf16*>(C)[(size_t)m * ldc + n] = __float2bfloat16(qnan);
        else
          (reinterpret_cast<float*>(C) + blockIdx.z * split_stride)[(size_t)m * ldc + n] = qnan;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// C[i] = sum over splits z (in order) of W[z][i], i < count
__global__ void k_splitk_sum(const float* __restrict__ W, int splits, size_t stride, size_t count, float* C) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += W[z * stride + i];
    C[i] = s;
  }
}

// ---------------------------------------------------------------- GEMM, TMA-fed pipeline
// The same C tile (128 x 64, FP32 accumulator in tensor memory) for operands
// that are both stored K-major, fed by the Tensor Memory Accelerator: a ring
// of kStages shared-memory stages, each holding one 64-wide K chunk of A
// (128 rows) and B (64 rows) in the 128-byte-swizzled K-major layout that
// both cp.async.bulk.tensor (SWIZZLE_128B) and tcgen05 (layout type
// SWIZZLE_128B) use: row r of a chunk is 128 bytes, its 16-byte pieces
// XOR-permuted by r mod 8, and 8-row groups 1024 bytes apart. Thread 0
// loads: it arms a stage's "full" mbarrier with the chunk's byte count and
// issues the two tensor copies, after waiting on the stage's "empty" mbarrier
// for the MMAs of the chunk that last used it. Thread 32 multiplies: it
// waits on "full", issues the chunk's four MMAs (K = 16 each: the
// descriptors' start address advances 32 bytes within the swizzled rows),
// and commits them to "empty"; after the last chunk it commits to "done",
// on which every thread waits before the epilogue. So up to kStages chunks
// are in flight while the tensor cores work. Every wait is bounded; a wait
// that gives up raises *err, the copies and MMAs in flight are waited for
// (bounded again) and the tile is filled with NaN.
constexpr int kStages = 4;
constexpr int kStageA = TM * TK * 2, kStageB = TN * TK * 2;   // bytes per stage
constexpr size_t kTmaSmem = (size_t)kStages * (kStageA + kStageB) + 1024;   // + alignment slack

// K-major, 128-byte swizzle: leading byte offset unused (1), stride byte
// offset 1024 (8 rows of 128 bytes), version 1, layout type 2 (SWIZZLE_128B)
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          saddr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  bool done = false;
  for (long i = 0; i < kMmaSpin && !done; ++i) done = mbar_try(bar, parity);
  return done;
}

template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_tma(const __grid_constant__ CUtensorMap mapA,
                                                  const __grid_constant__ CUtensorMap mapB, int M, int kper,
                                                  void* __restrict__ C, int ldc, size_t split_stride,
                                                  const float* __restrict__ bias, const bf16* __restrict__ ref,
                                                  int ldr, bf16* __restrict__ CT, int ldct, int* err) {
  extern __shared__ unsigned char tma_smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tma_smem_raw) + 1023) &
                                                       ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int nch = kper / TK, c0 = blockIdx.z * nch;   // this split's K chunks
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapB) : "memory");
    fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  auto stageA = [&](int s) { return sm + (size_t)s * (kStageA + kStageB); };
  auto stageB = [&](int s) { return sm + (size_t)s * (kStageA + kStageB) + kStageA; };

  if (tid == 0) {              // loads
    int c = 0;
    for (; c < nch; ++c) {
      const int s = c % kStages;
      if (c >= kStages && !mbar_wait(&empty[s], (uint32_t)((c / kStages - 1) & 1))) { fail = 1; break; }
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&full[s])),
                   "r"((uint32_t)(kStageA + kStageB))
                   : "memory");
      tma_load_2d(stageA(s), &mapA, &full[s], (c0 + c) * TK, m0);
      tma_load_2d(stageB(s), &mapB, &full[s], (c0 + c) * TK, n0);
    }
    // the copies issued must have landed before the CTA may end: the last
    // phase armed on every stage (earlier ones completed before it was armed)
    for (int s = 0; s < kStages && s < c; ++s) {
      const int last = c - 1 - ((c - 1 - s) % kStages);
      if (!mbar_wait(&full[s], (uint32_t)((last / kStages) & 1))) fail = 1;
    }
  } else if (tid == 32) {      // MMAs
    int c = 0;
    for (; c < nch; ++c) {
      const int s = c % kStages;
      if (!mbar_wait(&full[s], (uint32_t)((c / kStages) & 1))) { fail = 1; break; }
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < TK / 16; ++k) {
        const uint64_t ad = umma_desc_sw128(saddr(stageA(s)) + k * 32);
        const uint64_t bd = umma_desc_sw128(saddr(stageB(s)) + k * 32);
        const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       saddr(&empty[s]))
                   : "memory");
    }
    // "done" follows every MMA issued (also after a failed wait, so that the
    // others stop waiting as soon as the issued work is complete)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&done))
                 : "memory");
  }
  const bool landed = mbar_wait(&done, 0u);
  __syncthreads();
  const bool ok = landed && !fail && nch > 0;
  tc_fence_after();
  const int m = m0 + warp * 32 + lane;
  if (ok) {
#pragma unroll
    for (int cb = 0; cb < TN / 16; ++cb) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int n = n0 + cb * 16 + j;
          float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
          if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_BIAS_F32) {
            v0 += bias[n];
            v1 += bias[n + 1];
          }
          if (EPI == EPI_BIAS_RELU_BF16) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
          }
          if (EPI == EPI_MASK_BF16) {
            const __nv_bfloat162 rr = *reinterpret_cast<const __nv_bfloat162*>(&ref[(size_t)m * ldr + n]);
            if (!(__bfloat162float(rr.x) > 0.0f)) v0 = 0.0f;
            if (!(__bfloat162float(rr.y) > 0.0f)) v1 = 0.0f;
          }
          if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_BF16) {
            const __nv_bfloat162 o = __floats2bfloat162_rn(v0, v1);
            *reinterpret_cast<__nv_bfloat162*>(&reinterpret_cast<bf16*>(C)[(size_t)m * ldc + n]) = o;
            if (CT) {  // the transpose too (lanes: consecutive m, so consecutive addresses)
              CT[(size_t)n * ldct + m] = o.x;
              CT[(size_t)(n + 1) * ldct + m] = o.y;
            }
          } else {
            float* Cf = reinterpret_cast<float*>(C) + blockIdx.z * split_stride;
            *reinterpret_cast<float2*>(&Cf[(size_t)m * ldc + n]) = make_float2(v0, v1);
          }
        }
      }
    }
  } else {
    // a wait gave up (not expected): report, let the issued MMAs finish
    // (bounded), and poison this tile
    if (tid == 0) atomicExch(err, 1);
    mbar_wait(&done, 0u);
    if (m < M) {
      const float qnan = __uint_as_float(0x7fc00000u);
      for (int j = 0; j < TN; ++j) {
        if (EPI == EPI_BIAS_RELU_BF16 || EPI == EPI_MASK_BF16) {
          reinterpret_cast<bf16*>(C)[(size_t)m * ldc + n0 + j] = __float2bfloat16(qnan);
          if (CT) CT[(size_t)(n0 + j) * ldct + m] = __float2bfloat16(qnan);
        } else {
          (reinterpret_cast<float*>(C) + blockIdx.z * split_stride)[(size_t)m * ldc + n0 + j] = qnan;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*TensorMapEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TensorMapEncodeFn tensor_map_encoder() {
  static TensorMapEncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TensorMapEncodeFn>(p);
  }
  return fn;
}

// a [rows][K] bf16 matrix (leading dimension ld elements) in boxes of
// 64 (K) x box_rows, 128-byte swizzle; rows beyond `rows` read as zero
bool make_map(CUtensorMap* map, const bf16* ptr, int rows, int K, int ld, int box_rows) {
  TensorMapEncodeFn enc = tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(ptr) & 15)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
  const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(ptr), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launch; FP32 outputs with a small tile grid and a long K are split along K
// through the workspace ws (capacity ws_cap floats).
template <bool AK, bool BK, int EPI>
int gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, void* C, int ldc, const float* bias,
         const bf16* ref, int ldr, float* ws, size_t ws_cap, int* err, cudaStream_t s, bf16* CT = nullptr,
         int ldct = 0) {
  if (M % 64 || N % TN || K % TK || lda % 8 || ldb % 8 || ldc % 2 || M <= 0 || N <= 0 || K <= 0) return TMOP_ERR_ARG;
  const int mt = (M + TM - 1) / TM, nt = N / TN;
  if constexpr (AK && BK) {  // both operands K-major: the TMA-fed pipeline
    // FP32 outputs of a small tile grid over a long K (the weight gradients)
    // split K: about one CTA per SM, at least four chunks per split
    int sp = 1;
    if (EPI == EPI_F32 && ws) {
      const int nchunks = K / TK;
      while (sp < 64 && mt * nt * sp * 2 <= 152 && nchunks % (sp * 2) == 0 && nchunks / (sp * 2) >= 4 &&
             (size_t)(sp * 2) * M * ldc <= ws_cap)
        sp *= 2;
    }
    static bool attr = false;
    if (!attr) {
      if (cudaFuncSetAttribute(k_gemm_tma<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem) !=
          cudaSuccess)
        return TMOP_ERR_CUDA;
      attr = true;
    }
    CUtensorMap ma, mb;
    if (make_map(&ma, A, M, K, lda, TM) && make_map(&mb, B, N, K, ldb, TN)) {
      const size_t stride = (size_t)M * ldc;
      dim3 g(nt, mt, sp);
      k_gemm_tma<EPI><<<g, 128, kTmaSmem, s>>>(ma, mb, M, K / sp, sp > 1 ? (void*)ws : C, ldc, sp > 1 ? stride : 0,
                                               bias, ref, ldr, CT, ldct, err);
      if (sp > 1) k_splitk_sum<<<256, 256, 0, s>>>(ws, sp, stride, stride, reinterpret_cast<float*>(C));
      return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
    }
  }
  if (CT) return TMOP_ERR_ARG;   // the transposed output exists on the TMA path only
  int splits = 1;
  if (EPI == EPI_F32 && ws) {
    while (splits < 64 && mt * nt * splits * 2 <= 512 && K % (splits * 2 * TK) == 0 &&
           (size_t)(splits * 2) * M * ldc <= ws_cap)
      splits *= 2;
  }
  const int kper = K / splits;
  dim3 grid(nt, mt, splits);
  if (splits == 1) {
    k_gemm_tc<AK, BK, EPI><<<grid, 128, 0, s>>>(M, N, K, kper, A, lda, B, ldb, C, ldc, 0, bias, ref, ldr, err);
  } else {
    const size_t stride = (size_t)M * ldc;
    k_gemm_tc<AK, BK, EPI><<<grid, 128, 0, s>>>(M, N, K, kper, A, lda, B, ldb, ws, ldc, stride, bias, ref, ldr, err);
    k_splitk_sum<<<256, 256, 0, s>>>(ws, splits, stride, stride, reinterpret_cast<float*>(C));
  }
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

// ---------------------------------------------------------------- loss, sums, Adam
// dY = 2 (Y - T) / B on the n_out real columns (0 on the padding), as FP32
// and as bf16; per-block partial sums of (Y - T)^2 / B.
__global__ void k_loss_grad(const float* Y, int ldy, const float* T, int ldt, int batch, int n_out, int npad,
                            float* dYf, bf16* dYb, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  const size_t tot = (size_t)batch * npad;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / npad), j = (int)(t % npad);
    float g = 0.0f;
    if (j < n_out) {
      const float r = Y[(size_t)b * ldy + j] - T[(size_t)b * ldt + j];
      g = 2.0f * r / (float)batch;
      s += (double)r * (double)r / (double)batch;
    }
    dYf[t] = g;
    dYb[t] = __float2bfloat16_rn(g);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// one block of 256 threads: strided partial sums, then a fixed-order tree
__global__ void k_sum_parts(const double* part, int np, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Column sums of a [rows][ld] matrix (float or bf16) into out[ncol] (the
// bias gradients), in two deterministic passes: block (x, y) sums rows
// chunk y of columns x * 64 .. x * 64 + 63 (the 4 warps of a block split the
// chunk's rows, consecutive lanes read consecutive columns), then one thread
// per column adds the chunk partials in order.
constexpr int kColChunks = 64;
template <class Tv>
__global__ void k_colsum_part(const Tv* X, int rows, int ld, int ncol, float* part) {
  __shared__ float red[4][64];
  const int lane = threadIdx.x & 63, q = threadIdx.x >> 6;   // 256 threads: 4 row quarters x 64 columns
  const int j = blockIdx.x * 64 + lane;
  const int per = (rows + kColChunks - 1) / kColChunks;
  const int r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
  float s = 0.0f;
  if (j < ncol)
    for (int r = r0 + q; r < r1; r += 4) s += (float)X[(size_t)r * ld + j];
  red[q][lane] = s;
  __syncthreads();
  if (q == 0 && j < ncol) part[(size_t)blockIdx.y * ncol + j] = ((red[0][lane] + red[1][lane]) + red[2][lane]) + red[3][lane];
}

__global__ void k_colsum_final(const float* part, int ncol, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncol) return;
  float s = 0.0f;
  for (int c = 0; c < kColChunks; ++c) s += part[(size_t)c * ncol + j];
  out[j] = s;
}

template <class Tv>
int colsum(const Tv* X, int rows, int ld, int ncol, float* part, float* out, cudaStream_t s) {
  dim3 grid((ncol + 63) / 64, kColChunks);
  k_colsum_part<Tv><<<grid, 256, 0, s>>>(X, rows, ld, ncol, part);
  k_colsum_final<<<(ncol + 127) / 128, 128, 0, s>>>(part, ncol, out);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on all six parameter blocks in one
// launch (blocks start at off[b], sz[b] entries each; the padding between
// blocks is left alone), refreshing the bf16 copies of the weights.
struct AdamSegs {
  size_t off[6], sz[6];
  bf16* wb[6];
  bf16* wbT[6];   // transposed bf16 copy [cols][rows] of a [rows][cols] weight block, or null
  int cols[6], rows[6];
};

// the step counter lives on the device (so that a captured training step
// replays correctly): t += 1, then the bias corrections 0.9^t and 0.999^t
__global__ void k_adam_step(float* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const float t = st[0] + 1.0f;
    st[0] = t;
    st[1] = powf(0.9f, t);
    st[2] = powf(0.999f, t);
  }
}

__global__ void k_adam_all(float* w, float* m, float* v, const float* g, size_t total, const AdamSegs sg, float lr,
                           const float* __restrict__ st) {
  const float b1t = st[1], b2t = st[2];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int b = 5;
    while (b > 0 && i < sg.off[b]) --b;
    const size_t j = i - sg.off[b];
    if (j >= sg.sz[b]) continue;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / (1.0f - b1t)) / (sqrtf(vi / (1.0f - b2t)) + 1e-8f);
    w[i] = wi;
    if (sg.wb[b]) sg.wb[b][j] = __float2bfloat16_rn(wi);
    if (sg.wbT[b]) sg.wbT[b][(j % sg.cols[b]) * sg.rows[b] + j / sg.cols[b]] = __float2bfloat16_rn(wi);
  }
}

// out[c][r] = in[r][c] (bf16, [rows][ld_in] -> [cols][ld_out]), in 32 x 32
// tiles through shared memory
__global__ void k_transpose_bf16(const bf16* __restrict__ in, int rows, int cols, int ld_in, bf16* __restrict__ out,
                                 int ld_out) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * ld_in + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * ld_out + r] = tile[threadIdx.x][k];
  }
}

__global__ void k_to_bf16(const float* a, bf16* b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace mlp
}  // namespace tmop

using namespace tmop::mlp;

struct tmop_mlp {
  int n_in, H, n_out, K1, N3;  // K1 = padded input, N3 = padded output (multiples of 64)
  // FP32 masters (one allocation): W1 [H][K1], b1 [H], W2 [H][H], b2 [H], W3 [N3][H], b3 [N3]
  size_t off[6], total;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr;  // bf16 copies of the weight matrices
  bf16 *W2T = nullptr, *W3T = nullptr;               // and transposed, K-major for the data gradients
  int batch_cap = 0;
  bf16 *H1 = nullptr, *H2 = nullptr, *dYb = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  // transposes [features][batch] of the activations and gradients: the
  // weight-gradient GEMMs (K = batch) read both operands K-major
  bf16 *XT = nullptr, *H1T = nullptr, *H2T = nullptr, *dYT = nullptr, *dZ2T = nullptr, *dZ1T = nullptr;
  float *Y = nullptr, *dYf = nullptr;
  double* part = nullptr;
  float* ws = nullptr;   // split-K partial tiles of the weight-gradient GEMMs
  size_t ws_cap = 0;     // in floats
  int* d_err = nullptr;  // set when a GEMM's bounded wait for its MMAs gave up
  float* d_adam = nullptr;  // Adam step count and its bias corrections (device)
};

namespace {

int ensure_batch(tmop_mlp* n, int batch) {
  if (batch <= n->batch_cap) return TMOP_OK;
  cudaFree(n->H1); cudaFree(n->H2); cudaFree(n->dYb); cudaFree(n->dZ2); cudaFree(n->dZ1);
  cudaFree(n->Y); cudaFree(n->dYf); cudaFree(n->part);
  cudaFree(n->XT); cudaFree(n->H1T); cudaFree(n->H2T); cudaFree(n->dYT); cudaFree(n->dZ2T); cudaFree(n->dZ1T);
  const size_t B = batch;
  if (cudaMalloc(&n->XT, B * n->K1 * sizeof(bf16)) || cudaMalloc(&n->H1T, B * n->H * sizeof(bf16)) ||
      cudaMalloc(&n->H2T, B * n->H * sizeof(bf16)) || cudaMalloc(&n->dYT, B * n->N3 * sizeof(bf16)) ||
      cudaMalloc(&n->dZ2T, B * n->H * sizeof(bf16)) || cudaMalloc(&n->dZ1T, B * n->H * sizeof(bf16)) ||
      cudaMalloc(&n->H1, B * n->H * sizeof(bf16)) || cudaMalloc(&n->H2, B * n->H * sizeof(bf16)) ||
      cudaMalloc(&n->dZ2, B * n->H * sizeof(bf16)) || cudaMalloc(&n->dZ1, B * n->H * sizeof(bf16)) ||
      cudaMalloc(&n->dYb, B * n->N3 * sizeof(bf16)) || cudaMalloc(&n->Y, B * n->N3 * sizeof(float)) ||
      cudaMalloc(&n->dYf, B * n->N3 * sizeof(float)) || cudaMalloc(&n->part, 1024 * sizeof(double))) {
    n->batch_cap = 0;
    return TMOP_ERR_CUDA;
  }
  n->batch_cap = batch;
  return TMOP_OK;
}

float* P(tmop_mlp* n, float* base, int i) { return base + n->off[i]; }

int refresh_bf16(tmop_mlp* n, cudaStream_t s) {
  const size_t n1 = (size_t)n->H * n->K1, n2 = (size_t)n->H * n->H, n3 = (size_t)n->N3 * n->H;
  k_to_bf16<<<256, 256, 0, s>>>(P(n, n->w, 0), n->W1, n1);
  k_to_bf16<<<256, 256, 0, s>>>(P(n, n->w, 2), n->W2, n2);
  k_to_bf16<<<64, 256, 0, s>>>(P(n, n->w, 4), n->W3, n3);
  // W2 [H][H] -> W2^T, W3 [N3][H] -> W3^T [H][N3]
  k_transpose_bf16<<<dim3((n->H + 31) / 32, (n->H + 31) / 32), dim3(32, 8), 0, s>>>(n->W2, n->H, n->H, n->H, n->W2T,
                                                                                     n->H);
  k_transpose_bf16<<<dim3((n->H + 31) / 32, (n->N3 + 31) / 32), dim3(32, 8), 0, s>>>(n->W3, n->N3, n->H, n->H,
                                                                                      n->W3T, n->N3);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

// train: also the transposed activations [H][batch] for the weight gradients
int forward_impl(tmop_mlp* n, const bf16* X, int batch, float* Y, int ldy, cudaStream_t s, bool train = false) {
  int rc = gemm<true, true, EPI_BIAS_RELU_BF16>(batch, n->H, n->K1, X, n->K1, n->W1, n->K1, n->H1, n->H,
                                                P(n, n->w, 1), nullptr, 0, n->ws, n->ws_cap, n->d_err, s,
                                                train ? n->H1T : nullptr, batch);
  if (!rc) rc = gemm<true, true, EPI_BIAS_RELU_BF16>(batch, n->H, n->H, n->H1, n->H, n->W2, n->H, n->H2, n->H,
                                                     P(n, n->w, 3), nullptr, 0, n->ws, n->ws_cap, n->d_err, s,
                                                     train ? n->H2T : nullptr, batch);
  if (!rc) rc = gemm<true, true, EPI_BIAS_F32>(batch, n->N3, n->H, n->H2, n->H, n->W3, n->H, Y, ldy,
                                               P(n, n->w, 5), nullptr, 0, n->ws, n->ws_cap, n->d_err, s);
  return rc;
}

constexpr int kMaxNLat = 8;

// ---------------------------------------------------------------- coarse stage of the proposal
// Element vertices of a 2D order-k grid, and the bilinear interpolation of a
// vertex displacement at the Gauss-Lobatto lattice nodes of every element.
struct Lattice2 {
  int k, nx, ny, Nx, Ny, ldx;
  double z[kMaxNLat];  // GLL nodes on [0,1]
};

__global__ void k_lattice_vertices(Lattice2 L, const double* __restrict__ x, double* __restrict__ xv, int ldv) {
  const int nv = (L.nx + 1) * (L.ny + 1);
  const long long tot = 2LL * nv;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / nv), v = (int)(t % nv), i = v % (L.nx + 1), j = v / (L.nx + 1);
    xv[(size_t)c * ldv + v] = x[(size_t)c * L.ldx + (size_t)(L.k * j) * L.Nx + L.k * i];
  }
}

// x_out = x_in + P (xv1 - xv0) at the free dofs, x_in at the fixed ones
__global__ void k_lattice_prolong(Lattice2 L, const double* __restrict__ xv0, const double* __restrict__ xv1,
                                  int ldv, const double* x_in, const uint8_t* __restrict__ fixed, double* x_out) {
  const long long nn = (long long)L.Nx * L.Ny, tot = 2 * nn;
  const int nvx = L.nx + 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / nn);
    const long long node = t % nn;
    const int gx = (int)(node % L.Nx), gy = (int)(node / L.Nx);
    const size_t dof = (size_t)c * L.ldx + node;
    double val = x_in[dof];
    if (!(fixed && fixed[dof])) {
      const int ex = min(gx / L.k, L.nx - 1), ey = min(gy / L.k, L.ny - 1);
      const double zx = L.z[gx - L.k * ex], zy = L.z[gy - L.k * ey];
      const double* a = xv1 + (size_t)c * ldv;
      const double* b = xv0 + (size_t)c * ldv;
      const int v00 = ey * nvx + ex;
      const double d00 = a[v00] - b[v00], d10 = a[v00 + 1] - b[v00 + 1];
      const double d01 = a[v00 + nvx] - b[v00 + nvx], d11 = a[v00 + nvx + 1] - b[v00 + nvx + 1];
      val += (1.0 - zy) * ((1.0 - zx) * d00 + zx * d10) + zy * ((1.0 - zx) * d01 + zx * d11);
    }
    x_out[dof] = val;
  }
}

}  // namespace

extern "C" {

int tmop_patch_features(int order, int nx, int ny, const double* x, int ldx, int first, int count, uint16_t* feat,
                        int ldf, void* stream) {
  if (order < 1 || order > 4 || nx < 1 || ny < 1 || !x || !feat || first < 0 || count < 0 ||
      first + (long long)count > (long long)nx * ny)
    return TMOP_ERR_ARG;
  const int side = 3 * order + 1;
  if (ldf < 2 * side * side || ldf % 8) return TMOP_ERR_ARG;
  Grid2 G{order, nx, ny, order * nx + 1, order * ny + 1, ldx, x, {0}};
  if (ldx < G.Nx * G.Ny) return TMOP_ERR_ARG;
  double w[6];
  tmop::rule_gll(order + 1, G.xi, w);
  if (count == 0) return TMOP_OK;
  const int threads = 256, blocks = (int)(((long long)count * 32 + threads - 1) / threads);
  k_features<<<blocks, threads, 0, (cudaStream_t)stream>>>(G, first, count, reinterpret_cast<bf16*>(feat), ldf);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

int tmop_patch_targets(int order, int nx, int ny, const double* x0, const double* x1, int ldx, int first, int count,
                       float* T, int ldt, void* stream) {
  if (order < 1 || order > 4 || nx < 1 || ny < 1 || !x0 || !x1 || !T || first < 0 || count < 0 ||
      first + (long long)count > (long long)nx * ny || ldt < 2 * order * order)
    return TMOP_ERR_ARG;
  Grid2 G{order, nx, ny, order * nx + 1, order * ny + 1, ldx, x0, {0}};
  if (ldx < G.Nx * G.Ny) return TMOP_ERR_ARG;
  const long long tot = (long long)count * 2 * order * order;
  if (tot == 0) return TMOP_OK;
  k_targets<<<(int)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(G, x1, first, count, T, ldt);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

int tmop_patch_apply(int order, int nx, int ny, const double* x0, const uint8_t* fixed, int ldx, const float* Y,
                     int ldy, double scale, double* x_out, void* stream) {
  if (order < 1 || order > 4 || nx < 1 || ny < 1 || !x0 || !Y || !x_out || x_out == x0 || ldy < 2 * order * order ||
      !isfinite(scale))
    return TMOP_ERR_ARG;
  Grid2 G{order, nx, ny, order * nx + 1, order * ny + 1, ldx, x0, {0}};
  if (ldx < G.Nx * G.Ny) return TMOP_ERR_ARG;
  const long long tot = 2LL * G.Nx * G.Ny;
  k_apply<<<(int)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(G, fixed, Y, ldy, scale, x_out);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

int tmop_lattice_vertices(int order, int nx, int ny, const double* x, int ldx, double* xv, int ldv, void* stream) {
  if (order < 1 || order >= kMaxNLat || nx < 1 || ny < 1 || !x || !xv) return TMOP_ERR_ARG;
  Lattice2 L{order, nx, ny, order * nx + 1, order * ny + 1, ldx, {0}};
  if (ldx < L.Nx * L.Ny || ldv < (nx + 1) * (ny + 1)) return TMOP_ERR_ARG;
  const long long tot = 2LL * (nx + 1) * (ny + 1);
  k_lattice_vertices<<<(int)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(L, x, xv, ldv);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

int tmop_lattice_prolong_add(int order, int nx, int ny, const double* xv0, const double* xv1, int ldv,
                             const double* x_in, const uint8_t* fixed, int ldx, double* x_out, void* stream) {
  if (order < 1 || order >= kMaxNLat || nx < 1 || ny < 1 || !xv0 || !xv1 || !x_in || !x_out) return TMOP_ERR_ARG;
  Lattice2 L{order, nx, ny, order * nx + 1, order * ny + 1, ldx, {0}};
  if (ldx < L.Nx * L.Ny || ldv < (nx + 1) * (ny + 1)) return TMOP_ERR_ARG;
  double zw[kMaxNLat];
  tmop::rule_gll(order + 1, L.z, zw);
  const long long tot = 2LL * L.Nx * L.Ny;
  k_lattice_prolong<<<(int)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(L, xv0, xv1, ldv, x_in, fixed, x_out);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

void tmop_mlp_destroy(tmop_mlp* n) {
  if (!n) return;
  cudaFree(n->w); cudaFree(n->g); cudaFree(n->m); cudaFree(n->v);
  cudaFree(n->W1); cudaFree(n->W2); cudaFree(n->W3);
  cudaFree(n->H1); cudaFree(n->H2); cudaFree(n->dYb); cudaFree(n->dZ2); cudaFree(n->dZ1);
  cudaFree(n->Y); cudaFree(n->dYf); cudaFree(n->part);
  cudaFree(n->XT); cudaFree(n->H1T); cudaFree(n->H2T); cudaFree(n->dYT); cudaFree(n->dZ2T); cudaFree(n->dZ1T);
  cudaFree(n->W2T); cudaFree(n->W3T);
  cudaFree(n->ws); cudaFree(n->d_err); cudaFree(n->d_adam);
  delete n;
}

int tmop_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, tmop_mlp** out) {
  if (!out) return TMOP_ERR_ARG;
  *out = nullptr;
  if (n_in < 1 || n_in > 1024 || n_hidden < 64 || n_hidden % 64 || n_hidden > 4096 || n_out < 1 || n_out > 64)
    return TMOP_ERR_ARG;
  tmop_mlp* n = new tmop_mlp();
  n->n_in = n_in; n->H = n_hidden; n->n_out = n_out;
  n->K1 = (n_in + 63) / 64 * 64;
  n->N3 = 64;
  const size_t sz[6] = {(size_t)n->H * n->K1, (size_t)n->H, (size_t)n->H * n->H, (size_t)n->H,
                        (size_t)n->N3 * n->H, (size_t)n->N3};
  size_t acc = 0;
  for (int i = 0; i < 6; ++i) { n->off[i] = acc; acc += (sz[i] + 63) / 64 * 64; }
  n->total = acc;
  std::vector<float> host(acc, 0.0f);
  std::mt19937_64 gen(seed);
  auto fill = [&](int i, int rows, int cols, int ld, float std) {
    std::normal_distribution<float> nd(0.0f, std);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) host[n->off[i] + (size_t)r * ld + c] = nd(gen);
  };
  fill(0, n->H, n_in, n->K1, sqrtf(2.0f / n_in));
  fill(2, n->H, n->H, n->H, sqrtf(2.0f / n->H));
  fill(4, n_out, n->H, n->H, 0.1f * sqrtf(2.0f / n->H));
  int rc = TMOP_OK;
  // split-K workspace: up to 64 slices of the largest weight gradient (rows padded to 128)
  n->ws_cap = (size_t)64 * ((std::max(n->H, n->N3) + 127) / 128 * 128) * std::max(n->H, n->K1);
  if (cudaMalloc(&n->ws, n->ws_cap * 4) || cudaMalloc(&n->d_err, sizeof(int)) || cudaMemset(n->d_err, 0, sizeof(int)) ||
      cudaMalloc(&n->d_adam, 4 * sizeof(float)) || cudaMemset(n->d_adam, 0, 4 * sizeof(float)))
    rc = TMOP_ERR_CUDA;
  if (rc == TMOP_OK && (cudaMalloc(&n->w, acc * 4) || cudaMalloc(&n->g, acc * 4) || cudaMalloc(&n->m, acc * 4) ||
      cudaMalloc(&n->v, acc * 4) || cudaMalloc(&n->W1, sz[0] * 2) || cudaMalloc(&n->W2, sz[2] * 2) ||
      cudaMalloc(&n->W3, sz[4] * 2) || cudaMalloc(&n->W2T, sz[2] * 2) || cudaMalloc(&n->W3T, sz[4] * 2) || cudaMemcpy(n->w, host.data(), acc * 4, cudaMemcpyHostToDevice) ||
      cudaMemset(n->g, 0, acc * 4) || cudaMemset(n->m, 0, acc * 4) || cudaMemset(n->v, 0, acc * 4)))
    rc = TMOP_ERR_CUDA;
  if (rc == TMOP_OK) rc = refresh_bf16(n, 0);
  if (rc == TMOP_OK && cudaDeviceSynchronize() != cudaSuccess) rc = TMOP_ERR_CUDA;
  if (rc != TMOP_OK) { tmop_mlp_destroy(n); return rc; }
  *out = n;
  return TMOP_OK;
}

int tmop_mlp_input_ld(const tmop_mlp* n) { return n ? n->K1 : 0; }

size_t tmop_mlp_num_params(const tmop_mlp* n) {
  if (!n) return 0;
  return (size_t)n->H * n->n_in + n->H + (size_t)n->H * n->H + n->H + (size_t)n->n_out * n->H + n->n_out;
}

// Copy between the flat unpadded host layout and the padded device layout.
static int copy_params(tmop_mlp* n, float* dev, float* host, bool to_host) {
  std::vector<float> buf(n->total);
  if (to_host) {
    if (cudaDeviceSynchronize() || cudaMemcpy(buf.data(), dev, n->total * 4, cudaMemcpyDeviceToHost))
      return TMOP_ERR_CUDA;
  } else {
    std::fill(buf.begin(), buf.end(), 0.0f);
  }
  const int rows[6] = {n->H, 1, n->H, 1, n->n_out, 1};
  const int cols[6] = {n->n_in, n->H, n->H, n->H, n->H, n->n_out};
  const int ld[6] = {n->K1, 0, n->H, 0, n->H, 0};
  size_t h = 0;
  for (int i = 0; i < 6; ++i)
    for (int r = 0; r < rows[i]; ++r)
      for (int c = 0; c < cols[i]; ++c, ++h) {
        float& d = buf[n->off[i] + (size_t)r * ld[i] + c];
        if (to_host) host[h] = d;
        else d = host[h];
      }
  if (!to_host && cudaMemcpy(dev, buf.data(), n->total * 4, cudaMemcpyHostToDevice)) return TMOP_ERR_CUDA;
  return TMOP_OK;
}

int tmop_mlp_get(tmop_mlp* n, int which, float* host, size_t cnt) {
  if (!n || !host || cnt != tmop_mlp_num_params(n) || (which != 0 && which != 1)) return TMOP_ERR_ARG;
  int rc = copy_params(n, which == 0 ? n->w : n->g, host, true);
  int e = 0;  // a GEMM whose bounded wait for its MMAs gave up since the last check
  if (rc == TMOP_OK && cudaMemcpy(&e, n->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = TMOP_ERR_CUDA;
  if (rc == TMOP_OK && e) {
    cudaMemset(n->d_err, 0, sizeof(int));
    rc = TMOP_ERR_CUDA;
  }
  return rc;
}

int tmop_mlp_set(tmop_mlp* n, const float* host, size_t cnt) {
  if (!n || !host || cnt != tmop_mlp_num_params(n)) return TMOP_ERR_ARG;
  int rc = copy_params(n, n->w, const_cast<float*>(host), false);
  if (rc == TMOP_OK) rc = refresh_bf16(n, 0);
  if (rc == TMOP_OK && cudaDeviceSynchronize() != cudaSuccess) rc = TMOP_ERR_CUDA;
  return rc;
}

int tmop_mlp_check(tmop_mlp* n, void* stream) {
  if (!n) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int e = 0;  // raised by a GEMM whose bounded wait for its MMAs gave up
  if (cudaMemcpyAsync(&e, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TMOP_ERR_CUDA;
  if (e) {
    cudaMemsetAsync(n->d_err, 0, sizeof(int), s);
    return TMOP_ERR_CUDA;
  }
  return TMOP_OK;
}

int tmop_mlp_forward(tmop_mlp* n, const uint16_t* X, int batch, float* Y, int ldy, void* stream) {
  if (!n || !X || !Y || batch <= 0 || batch % 64 || ldy < n->n_out || ldy % 2) return TMOP_ERR_ARG;
  int rc = ensure_batch(n, batch);
  if (rc) return rc;
  // the last GEMM writes all N3 padded columns
  if (ldy < n->N3) {
    rc = forward_impl(n, reinterpret_cast<const bf16*>(X), batch, n->Y, n->N3, (cudaStream_t)stream);
    if (rc) return rc;
    if (cudaMemcpy2DAsync(Y, (size_t)ldy * 4, n->Y, (size_t)n->N3 * 4, (size_t)ldy * 4, batch,
                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream))
      return TMOP_ERR_CUDA;
  } else {
    rc = forward_impl(n, reinterpret_cast<const bf16*>(X), batch, Y, ldy, (cudaStream_t)stream);
    if (rc) return rc;
  }
  // the proposal is judged on these outputs: confirm, stream-ordered, that
  // no GEMM gave up on its tensor-core work
  return tmop_mlp_check(n, stream);
}

int tmop_mlp_gradients(tmop_mlp* n, const uint16_t* Xu, const float* T, int ldt, int batch, double* loss,
                       void* stream) {
  if (!n || !Xu || !T || batch <= 0 || batch % 64 || ldt < n->n_out) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_batch(n, batch);
  if (rc) return rc;
  const bf16* X = reinterpret_cast<const bf16*>(Xu);
  // X^T [K1][batch] for the first weight gradient
  k_transpose_bf16<<<dim3((n->K1 + 31) / 32, (batch + 31) / 32), dim3(32, 8), 0, s>>>(X, batch, n->K1, n->K1, n->XT,
                                                                                       batch);
  rc = forward_impl(n, X, batch, n->Y, n->N3, s, true);
  if (rc) return rc;
  const int lblocks = 256;
  k_loss_grad<<<lblocks, 256, 0, s>>>(n->Y, n->N3, T, ldt, batch, n->n_out, n->N3, n->dYf, n->dYb, n->part);
  if (loss) k_sum_parts<<<1, 256, 0, s>>>(n->part, lblocks, loss);
  k_transpose_bf16<<<dim3((n->N3 + 31) / 32, (batch + 31) / 32), dim3(32, 8), 0, s>>>(n->dYb, batch, n->N3, n->N3,
                                                                                       n->dYT, batch);
  // Every GEMM below reads both operands K-major (the TMA-fed kernel): the
  // weight gradients (K = batch) take the transposes [features][batch], the
  // data gradients the transposed weights.
  // layer 3: dW3 = dY^T H2, db3 = colsum dY, dH2 = dY W3 masked by H2 > 0
  rc = gemm<true, true, EPI_F32>(n->N3, n->H, batch, n->dYT, batch, n->H2T, batch, P(n, n->g, 4), n->H, nullptr,
                                 nullptr, 0, n->ws, n->ws_cap, n->d_err, s);
  if (!rc) rc = colsum<float>(n->dYf, batch, n->N3, n->N3, n->ws, P(n, n->g, 5), s);
  if (!rc) rc = gemm<true, true, EPI_MASK_BF16>(batch, n->H, n->N3, n->dYb, n->N3, n->W3T, n->N3, n->dZ2, n->H,
                                                nullptr, n->H2, n->H, n->ws, n->ws_cap, n->d_err, s, n->dZ2T, batch);
  // layer 2
  if (!rc) rc = gemm<true, true, EPI_F32>(n->H, n->H, batch, n->dZ2T, batch, n->H1T, batch, P(n, n->g, 2), n->H,
                                          nullptr, nullptr, 0, n->ws, n->ws_cap, n->d_err, s);
  if (!rc) rc = colsum<bf16>(n->dZ2, batch, n->H, n->H, n->ws, P(n, n->g, 3), s);
  if (!rc) rc = gemm<true, true, EPI_MASK_BF16>(batch, n->H, n->H, n->dZ2, n->H, n->W2T, n->H, n->dZ1, n->H,
                                                nullptr, n->H1, n->H, n->ws, n->ws_cap, n->d_err, s, n->dZ1T, batch);
  // layer 1
  if (!rc) rc = gemm<true, true, EPI_F32>(n->H, n->K1, batch, n->dZ1T, batch, n->XT, batch, P(n, n->g, 0), n->K1,
                                          nullptr, nullptr, 0, n->ws, n->ws_cap, n->d_err, s);
  if (!rc) rc = colsum<bf16>(n->dZ1, batch, n->H, n->H, n->ws, P(n, n->g, 1), s);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

int tmop_mlp_adam(tmop_mlp* n, float lr, void* stream) {
  if (!n || !(lr > 0.0f)) return TMOP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  bf16* wb[6] = {n->W1, nullptr, n->W2, nullptr, n->W3, nullptr};
  bf16* wbT[6] = {nullptr, nullptr, n->W2T, nullptr, n->W3T, nullptr};
  const size_t sz[6] = {(size_t)n->H * n->K1, (size_t)n->H, (size_t)n->H * n->H, (size_t)n->H,
                        (size_t)n->N3 * n->H, (size_t)n->N3};
  const int rows[6] = {n->H, 1, n->H, 1, n->N3, 1}, cols[6] = {n->K1, n->H, n->H, n->H, n->H, n->N3};
  AdamSegs sg;
  for (int i = 0; i < 6; ++i) {
    sg.off[i] = n->off[i];
    sg.sz[i] = sz[i];
    sg.wb[i] = wb[i];
    sg.wbT[i] = wbT[i];
    sg.rows[i] = rows[i];
    sg.cols[i] = cols[i];
  }
  k_adam_step<<<1, 32, 0, s>>>(n->d_adam);
  k_adam_all<<<304, 256, 0, s>>>(n->w, n->m, n->v, n->g, n->total, sg, lr, n->d_adam);
  return cudaGetLastError() == cudaSuccess ? TMOP_OK : TMOP_ERR_CUDA;
}

}  // extern "C"
