// Tensor-core GEMM tile for sm_103a: tcgen05.mma kind::f16 (BF16 operands, FP32 accumulator
// in tensor memory), one CTA of 128 threads per 128 x N output tile.
//
//   D[128][N] = A[128][K] * B[N][K]^T      (both operands K-major, BF16)
//
// The CTA stages A and B from global memory into shared memory in the canonical no-swizzle
// K-major layout (8 x 8 core matrices of 16-byte rows; consecutive core matrices along K are
// 128 bytes apart, along M/N K*16 bytes apart) with 16-byte asynchronous copies that are all
// in flight before the first is waited for, one thread issues K/16 MMAs of shape
// 128 x N x 16, the commit arrives on an mbarrier, and each warp reads its 32 accumulator
// rows back with tcgen05.ld and hands them to the epilogue in chunks of 16 columns.
// Every wait is bounded; on time-out the CTA records an error and still frees its tensor
// memory.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace bsp {

typedef __nv_bfloat16 bf16;

struct GemmA {
  const bf16* base;
  long long ystride;   // elements added per blockIdx.y
  int lda;             // elements between rows
  int nrows;           // rows that exist (others read as zero)
  int ka;              // K columns that exist (multiple of 8; others zero)
};

struct GemmB {
  const bf16* base;    // [N][K] per (blockIdx.y, blockIdx.z)
  long long ystride;   // elements added per blockIdx.y
  long long zstride;   // elements added per blockIdx.z
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // tcgen05 descriptor version; layout type 0 = no swizzle
  return d;
}

// element (r, k) of a rows x K tile in the canonical K-major no-swizzle layout
__device__ __forceinline__ int canon_idx(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

constexpr int kUmmaWaitIters = 1 << 22;

// 16-byte global -> shared copy through the L2 (cp.async.cg); ok == false zero-fills the
// destination and reads nothing.
__device__ __forceinline__ void cp_async_16(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}

template <int N>
struct TmemCols {
  static constexpr int value = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
};

template <int N, int K>
constexpr size_t umma_smem_bytes() {
  return (size_t)2 * 128 * K + (size_t)2 * N * K + 64;
}

// --- pieces of a tile: tensor-memory set-up, MMA issue, completion, accumulator read-back ---

// Allocates NCOLS tensor-memory columns (warp 0), initialises the completion mbarrier and makes
// the staged operands visible to the tensor cores; every thread returns the accumulator address.
template <int NCOLS>
__device__ __forceinline__ uint32_t umma_setup(uint32_t* tslot, uint64_t* mbar) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)), "n"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  return *tslot;
}

// K/16 MMAs of shape 128 x N x 16 from canonical K-major tiles at shared addresses a0 (A,
// 128 x K) and b0 (B, N x K) into the accumulator; the first overwrites it unless accumulate.
// Issued by one thread.
template <int N>
__device__ __forceinline__ void umma_issue(uint32_t tmem, uint32_t a0, uint32_t b0, int K, bool accumulate) {
  // kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9 = 1, 10-12 = 1), both K-major,
  // N >> 3 at bits 17-22, M >> 4 at bits 24-28.
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
#pragma unroll 1
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = umma_desc(a0 + kk * 256, 128, K * 16);
    const uint64_t bd = umma_desc(b0 + kk * 256, 128, K * 16);
    const uint32_t acc = (kk > 0 || accumulate) ? 1u : 0u;
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(mbar)));
}

// Bounded wait for the products committed to mbar's phase of the given parity (0 for the
// first commit, 1 for the second); records an error flag on time-out.
__device__ __forceinline__ bool umma_wait(uint64_t* mbar, int* err, uint32_t parity = 0) {
  uint32_t done = 0;
  for (int it = 0; it < kUmmaWaitIters && !done; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
  }
  if (!done && (threadIdx.x & 31) == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  return done != 0;
}

// 16 accumulator columns from column c0 of the warp's 32 lanes (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void umma_ld16(uint32_t tmem, int c0, float (&v)[16]) {
  const int warp = threadIdx.x >> 5;
  uint32_t r[16];
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                 "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Each warp reads its 32 accumulator rows, 16 columns at a time, into the epilogue.
template <int N, class Epi>
__device__ __forceinline__ void umma_readback(uint32_t tmem, const Epi& epi, typename Epi::Acc& acc, int by,
                                              int bz, int row) {
  epi.begin(acc, by, bz, row);
#pragma unroll 1
  for (int c0 = 0; c0 < N; c0 += 16) {
    float v[16];
    umma_ld16(tmem, c0, v);
    epi.chunk(acc, by, bz, row, c0, v);
  }
  epi.end(acc, by, bz, row);
}

template <int NCOLS>
__device__ __forceinline__ void umma_teardown(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(NCOLS));
}

template <int N, int K, class Epi>
__global__ void __launch_bounds__(128) umma_gemm(GemmA A, GemmB B, Epi epi, int* err) {
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "N");
  static_assert(K % 16 == 0, "K");
  extern __shared__ __align__(1024) unsigned char smem[];
  bf16* sA = reinterpret_cast<bf16*>(smem);
  bf16* sB = sA + 128 * K;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + N * K);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * 128;
  const int by = blockIdx.y, bz = blockIdx.z;
  const bf16* Ab = A.base + by * A.ystride;
  const bf16* Bb = B.base + by * B.ystride + bz * B.zstride;
  // every 16-byte chunk of both operands as an asynchronous copy, all in flight at once
  // (rows of A beyond nrows and columns beyond ka are zero-filled, nothing is read there)
  constexpr int KV = K / 8;
  for (int e = tid; e < 128 * KV; e += 128) {
    const int r = e / KV, kv = e - (e / KV) * KV;
    const int grow = row0 + r;
    const bool ok = grow < A.nrows && kv * 8 < A.ka;
    cp_async_16(sA + canon_idx(r, kv * 8, K), ok ? Ab + (size_t)grow * A.lda + kv * 8 : Ab, ok);
  }
  for (int e = tid; e < N * KV; e += 128) {
    const int r = e / KV, kv = e - (e / KV) * KV;
    cp_async_16(sB + canon_idx(r, kv * 8, K), Bb + (size_t)r * K + kv * 8, true);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  constexpr int NCOLS = TmemCols<N>::value;
  const uint32_t tmem = umma_setup<NCOLS>(tslot, mbar);
  if (tid == 0) {
    umma_issue<N>(tmem, smem_u32(sA), smem_u32(sB), K, false);
    umma_commit(mbar);
  }
  // loads of the epilogue that do not depend on the product, in flight while it runs
  const int row = row0 + warp * 32 + lane;
  typename Epi::Acc acc;
  epi.prefetch(acc, by, bz, row);
  if (umma_wait(mbar, err)) umma_readback<N>(tmem, epi, acc, by, bz, row);
  umma_teardown<NCOLS>(tmem);
}

// Two products into one accumulator: D[128][N] = A1 B1^T + A2 B2^T (K1 and K2 multiples of 16),
// for stages whose output is the sum of two contractions of different operands.  Ops stages
// the four tiles of the CTA (canonical K-major layouts, by cp.async) in load(sA1, sB1, sA2, sB2).
template <int N, int K1, int K2>
constexpr size_t umma2_smem_bytes() {
  return (size_t)2 * (128 + N) * (K1 + K2) + 64;
}

template <int N, int K1, int K2, class Ops, class Epi>
__global__ void __launch_bounds__(128) umma_gemm2(Ops ops, Epi epi, int* err) {
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "N");
  static_assert(K1 % 16 == 0 && K2 % 16 == 0, "K");
  extern __shared__ __align__(1024) unsigned char smem[];
  bf16* sA1 = reinterpret_cast<bf16*>(smem);
  bf16* sB1 = sA1 + 128 * K1;
  bf16* sA2 = sB1 + N * K1;
  bf16* sB2 = sA2 + 128 * K2;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB2 + N * K2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int by = blockIdx.y, bz = blockIdx.z;
  ops.load(sA1, sB1, sA2, sB2);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  constexpr int NCOLS = TmemCols<N>::value;
  const uint32_t tmem = umma_setup<NCOLS>(tslot, mbar);
  if (tid == 0) {
    umma_issue<N>(tmem, smem_u32(sA1), smem_u32(sB1), K1, false);
    umma_issue<N>(tmem, smem_u32(sA2), smem_u32(sB2), K2, true);
    umma_commit(mbar);
  }
  const int row = blockIdx.x * 128 + warp * 32 + lane;
  typename Epi::Acc acc;
  epi.prefetch(acc, by, bz, row);
  if (umma_wait(mbar, err)) umma_readback<N>(tmem, epi, acc, by, bz, row);
  umma_teardown<NCOLS>(tmem);
}

template <int N, int K1, int K2, class Ops, class Epi>
inline cudaError_t launch_umma2(dim3 grid, const Ops& ops, const Epi& epi, int* err, cudaStream_t s) {
  constexpr size_t smem = umma2_smem_bytes<N, K1, K2>();
  auto kern = umma_gemm2<N, K1, K2, Ops, Epi>;
  static bool attr_set = false;   // per template instance (set once per process)
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  kern<<<grid, 128, smem, s>>>(ops, epi, err);
  return cudaGetLastError();
}

template <int N, int K, class Epi>
inline cudaError_t launch_umma(dim3 grid, const GemmA& A, const GemmB& B, const Epi& epi, int* err,
                               cudaStream_t s) {
  constexpr size_t smem = umma_smem_bytes<N, K>();
  auto kern = umma_gemm<N, K, Epi>;
  static bool attr_set = false;   // per template instance (set once per process)
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  kern<<<grid, 128, smem, s>>>(A, B, epi, err);
  return cudaGetLastError();
}

}  // namespace bsp
