// Block matrix-vector products of the dense solve on the 5th-generation tensor cores.
//
// The paper only states the system (Section 3.4: the N x N Nystrom matrix times the density);
// its solver, storage precision and matrix products are this library's.  The mixed-precision
// solve keeps the matrix once more in split BF16: every real component a of A (interleaved
// re, im) is stored as hi = bf16(a) and lo = bf16(a - hi), so hi + lo holds 16 significant bits
// (relative error <= 2^-16), in 8 bytes per complex entry, the size of an FP32 complex copy.
//
// Complex product as one real GEMM.  With A read as a real matrix Ar [N][2N] (row i =
// re A_i0, im A_i0, re A_i1, ...) and nr right-hand sides X [nr][N], the real matrix Bt
// [2 nr][2N] with rows
//   Bt[2j]   = ( re X_0j, -im X_0j, re X_1j, -im X_1j, ...)
//   Bt[2j+1] = ( im X_0j,  re X_0j, im X_1j,  re X_1j, ...)
// gives C = Ar Bt^T with C[i][2j] = re (A X)_ij and C[i][2j+1] = im (A X)_ij.  The split
// product is Ah Bh + Ah Bl + Al Bh (the Al Bl term is below the split's own error).
//
// Kernel: tcgen05.mma (kind::f16, BF16 in, FP32 accumulate in tensor memory), M = 128 rows,
// N = 2 nr padded to 16 or 32, K = 16 per instruction.  The operands are stored in HBM in
// exactly the shared-memory image the MMA reads (K-major, 128-byte swizzle, 1024-byte tiles of
// 8 rows x 128 bytes): one k-tile of A is 128 rows x 64 BF16 (16 KB per half), one of Bt is
// 2 nr rows x 64 BF16, so each pipeline stage is two bulk copies (cp.async.bulk) and no tensor
// map is needed.  One CTA per SM runs persistently over an equal share of all (row tile,
// k-tile) steps ("stream-K"): a warp issues the copies, one thread the MMAs, four warps read
// the accumulator (tcgen05.ld) every `chunk` k-tiles and add it into FP64 registers (short FP32
// accumulation chains), and at the end of a row tile add their rows into y with FP64 atomics.
// Every wait on a barrier is bounded; a wait that runs out sets an error flag, drains the copies
// and MMAs in flight, frees the tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "bie_internal.cuh"
#include "dw.cuh"
#include "tc_matvec.cuh"

namespace bie {

constexpr int kTcStages = 5;
constexpr int kTcThreads = 192;                 // warp 0: copies, warp 1: MMA, warps 2-5: accumulator
constexpr long long kTcTimeout = 4000000000LL;  // clock cycles (about 2 s) before a wait gives up

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false if it timed out or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kTcTimeout) {
      *abort = 1;
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// K-major operand in the 128-byte swizzle layout: 8-row groups 1024 bytes apart (SBO), the
// leading-dimension offset unused for this layout, descriptor version 1 (bits 46-48).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (encoded 1; not used with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // fixed 0b001
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}
// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t umma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ the work list of one CTA
// Steps g = mt * n_kt + kt in [g0, g1); a run of steps with the same mt is a segment, cut into
// chunks at multiples of `chunk` in kt.  All roles walk the same sequence.
struct TcWalk {
  int64_t g, g1;
  int n_kt, chunk;
  __device__ TcWalk(int64_t a, int64_t b, int nkt, int ch) : g(a), g1(b), n_kt(nkt), chunk(ch) {}
  __device__ bool done() const { return g >= g1; }
  // the chunk starting at g: [g, end); seg_end: the chunk ends its segment
  __device__ int64_t chunk_end(bool* seg_end) const {
    const int64_t mt = g / n_kt, kt = g % n_kt;
    int64_t e = mt * n_kt + ((kt / chunk) + 1) * chunk;
    const int64_t tile_end = (mt + 1) * n_kt;
    if (e > tile_end) e = tile_end;
    if (e > g1) e = g1;
    *seg_end = (e == tile_end) || (e == g1);
    return e;
  }
};

template <int BN>
struct TcSmem {
  static constexpr uint32_t kA = 128 * 128;        // one half (hi or lo) of an A k-tile
  static constexpr uint32_t kB = BN * 128;         // one half of a Bt k-tile
  static constexpr uint32_t kStage = 2 * kA + 2 * kB;
  static constexpr size_t kBytes = 1024 + (size_t)kTcStages * kStage + 256;
};

template <int BN>
__global__ void __launch_bounds__(kTcThreads, 1) tc_cgemm_kernel(const TcArgs a) {
  using L = TcSmem<BN>;
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* stages = base;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + (size_t)kTcStages * L::kStage);
  uint64_t* full = bars;                     // [kTcStages]
  uint64_t* empty = bars + kTcStages;        // [kTcStages]
  uint64_t* acc_full = bars + 2 * kTcStages; // [2]
  uint64_t* acc_empty = acc_full + 2;        // [2]
  uint64_t* drain = acc_empty + 2;           // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = (int64_t)a.n_mt * a.n_kt;
  const int64_t g0 = total * blockIdx.x / gridDim.x, g1 = total * (blockIdx.x + 1) / gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(drain, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {   // two accumulators of BN FP32 columns (64 columns: a power of two >= 32)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- copies: one thread issues the A and Bt k-tiles of every step of the range
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t g = g0; g < g1; ++g, ++issued) {
        const int s = (int)(issued % kTcStages);
        const uint32_t ph = (uint32_t)((issued / kTcStages) & 1);
        if (!mbar_wait(&empty[s], ph ^ 1u, abort)) break;
        const int64_t mt = g / a.n_kt, kt = g % a.n_kt;
        uint8_t* st = stages + (size_t)s * L::kStage;
        mbar_expect_tx(&full[s], L::kStage);
        bulk_g2s(st, a.a_img + (size_t)(mt * a.n_kt + kt) * (2 * L::kA), 2 * L::kA, &full[s]);
        bulk_g2s(st + 2 * L::kA, a.b_img + (size_t)kt * (2 * L::kB), 2 * L::kB, &full[s]);
      }
      // the last (up to kTcStages) copies issued have landed before the CTA may exit (on the
      // normal path their phases completed already and these waits return at once)
      for (int64_t i = issued > kTcStages ? issued - kTcStages : 0; i < issued; ++i) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[i % kTcStages], (uint32_t)((i / kTcStages) & 1)))
          if (clock64() - t0 > kTcTimeout) break;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA: one thread; chunk c accumulates into buffer c & 1
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(BN);
      TcWalk w(g0, g1, a.n_kt, a.chunk);
      int64_t it = 0, ci = 0;
      bool ok = true, any = false;
      while (ok && !w.done()) {
        bool seg_end;
        const int64_t e = w.chunk_end(&seg_end);
        const int buf = (int)(ci & 1);
        if (!mbar_wait(&acc_empty[buf], (uint32_t)(((ci >> 1) & 1) ^ 1), abort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * BN);
        bool first = true;
        for (; w.g < e; ++w.g, ++it) {
          const int s = (int)(it % kTcStages);
          if (!mbar_wait(&full[s], (uint32_t)((it / kTcStages) & 1), abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(stages + (size_t)s * L::kStage);
          const uint32_t sb = sa + 2 * L::kA;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {   // 4 x K = 16 BF16 across the 128-byte row
            const uint64_t ah = umma_desc(sa + ks * 32), al = umma_desc(sa + L::kA + ks * 32);
            const uint64_t bh = umma_desc(sb + ks * 32), bl = umma_desc(sb + L::kB + ks * 32);
            umma_bf16(dt, ah, bh, idesc, first ? 0u : 1u);
            first = false;
            umma_bf16(dt, ah, bl, idesc, 1u);
            umma_bf16(dt, al, bh, idesc, 1u);
          }
          any = true;
          umma_commit(&empty[s]);   // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        umma_commit(&acc_full[buf]);
        ++ci;
      }
      if (!ok && any) {
        // drain the MMAs in flight before the tensor memory is released
        umma_commit(drain);
        const long long t0 = clock64();
        while (!mbar_try_wait(drain, 0))
          if (clock64() - t0 > kTcTimeout) break;
      }
    }
    __syncwarp();
  } else {
    // ---------------- accumulator: warps 2..5 own TMEM lane quarters (warp % 4)
    const int q = warp & 3;
    const int64_t row_local = q * 32 + lane;
    double acc[BN];
#pragma unroll
    for (int c = 0; c < BN; ++c) acc[c] = 0.0;
    TcWalk w(g0, g1, a.n_kt, a.chunk);
    int64_t ci = 0;
    while (!w.done()) {
      bool seg_end;
      const int64_t e = w.chunk_end(&seg_end);
      const int64_t mt = w.g / a.n_kt;
      const int buf = (int)(ci & 1);
      // lane 0 waits, the warp follows (tcgen05.ld needs the whole warp converged)
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&acc_full[buf], (uint32_t)((ci >> 1) & 1), abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN);
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(taddr + c0, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c0 + c] += (double)v[c];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      ++ci;
      w.g = e;
      if (seg_end) {
        const int64_t row = mt * 128 + row_local;
        if (row < a.n_rows) {
#pragma unroll
          for (int j = 0; j < BN / 2; ++j) {   // unrolled: acc stays in registers
            if (j < a.nr) {
              double* yj = reinterpret_cast<double*>(a.y + (int64_t)j * a.ldy + row);
              atomicAdd(yj, acc[2 * j]);
              atomicAdd(yj + 1, acc[2 * j + 1]);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < BN; ++c) acc[c] = 0.0;
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
  }
  if (threadIdx.x == 0 && *abort) atomicExch(a.status + 1, 1);
}

// ------------------------------------------------------------------ operand images
// A (FP64 complex [n][lda], read as reals) -> split-BF16 image [n_mt][n_kt][hi, lo][128][128 B]:
// thread per 16-byte chunk (8 reals) of a tile row; rows and columns past the matrix are zero.
// The top 24 significand bits (integer split, no FP64 instruction) round to hi; the FP32
// remainder rounds to lo.
__global__ void tc_split_a_kernel(int64_t n, int64_t lda, const double* __restrict__ A, int n_mt, int n_kt,
                                  uint4* __restrict__ img) {
  const int64_t chunks = (int64_t)n_mt * n_kt * 128 * 8;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < chunks;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx & 7);
    const int r = (int)((idx >> 3) & 127);
    const int64_t tile = idx >> 10;   // mt * n_kt + kt
    const int64_t mt = tile / n_kt, kt = tile % n_kt;
    const int64_t row = mt * 128 + r;
    const int64_t col0 = kt * 64 + c * 8;   // real column
    __nv_bfloat16 hv[8], lv[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      float f = 0.f;
      if (row < n && col0 + e < 2 * n) f = dw_from(A[row * 2 * lda + col0 + e]).x;
      const __nv_bfloat16 h = __float2bfloat16_rn(f);
      hv[e] = h;
      lv[e] = __float2bfloat16_rn(f - __bfloat162float(h));
    }
    const int64_t off = tile * 2048 + r * 8 + (c ^ (r & 7));   // in 16-byte units; hi half first
    img[off] = *reinterpret_cast<const uint4*>(hv);
    img[off + 1024] = *reinterpret_cast<const uint4*>(lv);
  }
}

// X [nr][ldx] complex -> Bt image [n_kt][hi, lo][BN][128 B] (rows 2j: re, -im; rows 2j+1: im, re)
__global__ void tc_split_b_kernel(int64_t n, int nr, int BN, const double2* __restrict__ X, int64_t ldx, int n_kt,
                                  uint4* __restrict__ img) {
  const int64_t chunks = (int64_t)n_kt * BN * 8;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < chunks;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx & 7);
    const int rr = (int)((idx >> 3) % BN);
    const int64_t kt = (idx >> 3) / BN;
    const int j = rr >> 1;
    __nv_bfloat16 hv[8], lv[8];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const int64_t k = (kt * 64 + c * 8 + e) >> 1;   // complex column
      float v0 = 0.f, v1 = 0.f;
      if (j < nr && k < n) {
        const double2 x = X[(int64_t)j * ldx + k];
        const float xr = dw_from(x.x).x, xi = dw_from(x.y).x;
        if (rr & 1) { v0 = xi; v1 = xr; } else { v0 = xr; v1 = -xi; }
      }
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
      hv[e] = h0;
      hv[e + 1] = h1;
      lv[e] = __float2bfloat16_rn(v0 - __bfloat162float(h0));
      lv[e + 1] = __float2bfloat16_rn(v1 - __bfloat162float(h1));
    }
    const int64_t off = kt * (2 * BN * 8) + rr * 8 + (c ^ (rr & 7));
    img[off] = *reinterpret_cast<const uint4*>(hv);
    img[off + BN * 8] = *reinterpret_cast<const uint4*>(lv);
  }
}

// ------------------------------------------------------------------ host side
bie_status tc_image_create(bie_ctx ctx, int64_t n, const double* A, TcImage* out) {
  TcImage im;
  im.n = n;
  im.n_mt = (int)((n + 127) / 128);
  im.n_kt = (int)((2 * n + 63) / 64);
  const size_t bytes = (size_t)im.n_mt * im.n_kt * 2 * 128 * 128;
  cudaError_t e = cudaMallocAsync((void**)&im.a_img, bytes, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(split-BF16 matrix)");
  e = cudaMallocAsync((void**)&im.b_img, (size_t)im.n_kt * 2 * 32 * 128, ctx->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(im.a_img, ctx->stream);
    return cuda_fail(e, "cudaMallocAsync(split-BF16 vectors)");
  }
  tc_split_a_kernel<<<ctx->sms * 16, 256, 0, ctx->stream>>>(n, n, A, im.n_mt, im.n_kt,
                                                          reinterpret_cast<uint4*>(im.a_img));
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFreeAsync(im.a_img, ctx->stream);
    cudaFreeAsync(im.b_img, ctx->stream);
    return cuda_fail(e, "tc_split_a_kernel");
  }
  *out = im;
  return BIE_OK;
}

void tc_image_free(bie_ctx ctx, TcImage* im) {
  if (im->a_img) cudaFreeAsync(im->a_img, ctx->stream);
  if (im->b_img) cudaFreeAsync(im->b_img, ctx->stream);
  im->a_img = im->b_img = nullptr;
}

template <int BN>
static bie_status tc_launch(bie_ctx ctx, const TcImage& im, int nr, double2* y, int64_t ldy) {
  using L = TcSmem<BN>;
  static int attr_set[64] = {0};
  const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
  if (!attr_set[dev]) {
    const cudaError_t e =
        cudaFuncSetAttribute(tc_cgemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kBytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_cgemm_kernel)");
    attr_set[dev] = 1;
  }
  TcArgs a;
  a.a_img = im.a_img;
  a.b_img = im.b_img;
  a.y = y;
  a.ldy = ldy;
  a.n_rows = im.n;
  a.nr = nr;
  a.n_mt = im.n_mt;
  a.n_kt = im.n_kt;
  a.chunk = 16;
  a.status = ctx->d_status;
  const int64_t total = (int64_t)im.n_mt * im.n_kt;
  const int grid = (int)std::min<int64_t>(ctx->sms, total);
  tc_cgemm_kernel<BN><<<grid, kTcThreads, L::kBytes, ctx->stream>>>(a);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "tc_cgemm_kernel");
}

// y[j] = A x[j], j < nr <= 16: x, y [nr][ldx|ldy] complex (y overwritten)
bie_status tc_matvec(bie_ctx ctx, TcImage& im, const double2* x, int64_t ldx, int nr, double2* y, int64_t ldy) {
  if (nr < 1 || nr > 16) { set_error("tensor-core matvec: 1 <= nr <= 16"); return BIE_EINVAL; }
  const int BN = nr <= 8 ? 16 : 32;
  const int64_t chunks = (int64_t)im.n_kt * BN * 8;
  tc_split_b_kernel<<<(unsigned)std::min<int64_t>((chunks + 255) / 256, (int64_t)ctx->sms * 8), 256, 0,
                      ctx->stream>>>(im.n, nr, BN, x, ldx, im.n_kt, reinterpret_cast<uint4*>(im.b_img));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tc_split_b_kernel");
  for (int j = 0; j < nr; ++j) {
    e = cudaMemsetAsync(y + (int64_t)j * ldy, 0, sizeof(double2) * im.n, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(tensor-core matvec output)");
  }
  return BN == 16 ? tc_launch<16>(ctx, im, nr, y, ldy) : tc_launch<32>(ctx, im, nr, y, ldy);
}

}  // namespace bie
