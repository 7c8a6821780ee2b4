// Stochastic reconfiguration on the most probable samples (Sec. "ANQS-
// tailored stochastic reconfiguration", Eq. qgt_definition), min-SR form:
//   w_x = p(x) / sum_SR p,  m = sum_x w_x O_x,  Obar_x = sqrt(w_x) (O_x - m),
//   T = Obar Obar^T (N_SR x N_SR),  eps_x = sqrt(w_x) (Re E_loc(x) - E),
//   delta = Obar^T (T + lambda I)^{-1} eps   (= (S + lambda I)^{-1} g, S the QGT).
// The solve deflates T's known null vector sqrt(w) (sr_solve_kernel).
// O = d log psi / d theta of the N_SR samples, FP32 [N_SR][P] (real), P large.
//
// T is the one dense contraction of the method: M = N = N_SR <= 128, K = P.
// gram_kernel streams O once: each CTA takes a range of 64-column K tiles,
// centres and scales them on the CUDA cores, splits every value into bf16
// hi + lo (about 16 significant bits together), stores both in shared memory
// in the tensor core's canonical K-major layout and lets one thread issue
// tcgen05.mma (kind::f16, bf16 in, FP32 accumulate in TMEM, M = N = 128):
// D += hi hi^T + hi lo^T + lo hi^T (the lo lo^T term is below the split's
// error).  Two shared-memory stages; an mbarrier signalled by tcgen05.commit
// tells the loaders when a stage's MMAs are done.  The 128 x 128 FP32
// accumulator (128 TMEM columns) is read back with tcgen05.ld and written as
// the CTA's partial; the partials are summed in FP64 in a fixed order.
#include <algorithm>
#include <cfloat>
#include <cstring>

#include <cuda.h>   // CUtensorMap and its enums; the encoder is fetched through the runtime
#include <cuda_bf16.h>
#include <mutex>

#include "device_util.cuh"
#include "nqs_internal.cuh"

namespace nqs {

constexpr int kSrRows = 128;      // N_SR padded to the MMA's M = N
constexpr int kSrKTile = 64;      // K elements per stage (4 MMAs of K = 16)
constexpr int kSrThreads = 128;   // 4 warps: loaders; warp w reads TMEM lanes 32w..32w+31
constexpr int kSrStages = 2;
constexpr int kSrTileBytes = kSrRows * kSrKTile * 2;   // one bf16 tile: 16 KB
constexpr int kSrSmem = kSrStages * 2 * kSrTileBytes + 1024;
constexpr long long kSrWaitLimit = 1ll << 26;          // mbarrier polls before giving up

static inline int64_t a256r(int64_t v) { return (v + 255) & ~int64_t(255); }

// ---------------------------------------------------------------------------
// PTX helpers (tcgen05, mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return done != 0;
}

// bounded wait: false (and the caller records an error) if the phase never completes
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  for (long long it = 0; it < kSrWaitLimit; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, bf16 in, FP32 accumulate
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) completing on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// 2-D tiled tensor copy global -> shared (box of the tensor map at column x, row y)
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes (rows 16 B apart); lbo = byte distance between the two
// core matrices adjacent along K, sbo = between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture family; base offset 0, no swizzle
  return d;
}

// instruction descriptor: D FP32, A and B bf16, both K-major, N = 128, M = 128
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kSrRows >> 3) << 17) |
                                ((uint32_t)(kSrRows >> 4) << 24);

// the same with N = 256: B = the hi tile followed by the lo tile (rows 128 .. 255), so one
// MMA gives [hi hi^T | hi lo^T] (lo hi^T is the transpose of the second half)
constexpr uint32_t kIdescBf16N256 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                                    ((uint32_t)(kSrRows >> 4) << 24);

// byte offset of (row r, k) inside a 128 x 64 tile: core matrix (r / 8, k / 8)
// at (r / 8) * 1024 + (k / 8) * 128, then row r % 8 at 16 B and k % 8 at 2 B
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
constexpr uint32_t kSrLbo = 128, kSrSbo = 1024;

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// ---------------------------------------------------------------------------
// Gram kernel: partial[blockIdx.x] = sum over this CTA's K tiles of Obar Obar^T
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSrThreads) gram_kernel(int n, int64_t P, const float* __restrict__ O,
                                                          const float* __restrict__ m, const float* __restrict__ sw,
                                                          int64_t tiles_per_cta, float* __restrict__ partial,
                                                          int32_t* __restrict__ error) {
  extern __shared__ __align__(1024) unsigned char sr_smem[];
  __shared__ uint64_t bars[kSrStages];
  __shared__ uint32_t s_taddr;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)sr_smem + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t n_tiles = (P + kSrKTile - 1) / kSrKTile;
  const int64_t t0 = (int64_t)blockIdx.x * tiles_per_cta;
  const int64_t t1 = t0 + tiles_per_cta < n_tiles ? t0 + tiles_per_cta : n_tiles;
  if (tid == 0) {
    for (int s = 0; s < kSrStages; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(&s_taddr, kSrRows);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  bool ok = true;
  int64_t it = 0;
  for (int64_t t = t0; t < t1; ++t, ++it) {
    const int s = (int)(it & 1);
    unsigned char* hi = base + s * 2 * kSrTileBytes;
    unsigned char* lo = hi + kSrTileBytes;
    if (it >= kSrStages && !mbar_wait(&bars[s], (uint32_t)(((it - kSrStages) >> 1) & 1))) ok = false;
    // load, centre, scale and split 128 rows x 64 columns: thread tid takes rows r = 2 i + tid / 64,
    // columns 4 ((tid % 64) % 16) .. + 3 of quarter (tid % 64) / 16 -- i.e. float4 groups along K
    const int64_t k0 = t * kSrKTile;
#pragma unroll 4
    for (int i = 0; i < (kSrRows * kSrKTile / 4) / kSrThreads; ++i) {
      const int g = i * kSrThreads + tid;       // float4 group index within the tile
      const int r = g / (kSrKTile / 4);
      const int kq = (g % (kSrKTile / 4)) * 4;  // first k of the group
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (r < n) {
        const float s_r = __ldg(sw + r);
        const int64_t k = k0 + kq;
        if (k + 3 < P && (((uintptr_t)(O + (int64_t)r * P + k)) & 15) == 0) {
          const float4 o = __ldg(reinterpret_cast<const float4*>(O + (int64_t)r * P + k));
          const float4 mm = __ldg(reinterpret_cast<const float4*>(m + k));
          v[0] = s_r * (o.x - mm.x); v[1] = s_r * (o.y - mm.y); v[2] = s_r * (o.z - mm.z); v[3] = s_r * (o.w - mm.w);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (k + j < P) v[j] = s_r * (__ldg(O + (int64_t)r * P + k + j) - __ldg(m + k + j));
        }
      }
      float h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        h[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
        l[j] = v[j] - h[j];
      }
      const uint32_t off = tile_off(r, kq);
      *reinterpret_cast<uint2*>(hi + off) = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
      *reinterpret_cast<uint2*>(lo + off) = make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sh = smem_u32(hi), sl = smem_u32(lo);
#pragma unroll
      for (int j = 0; j < kSrKTile / 16; ++j) {
        const uint32_t adv = (uint32_t)j * 2 * kSrLbo;   // two core matrices along K per MMA
        const uint64_t dh = umma_desc(sh + adv, kSrLbo, kSrSbo);
        const uint64_t dl = umma_desc(sl + adv, kSrLbo, kSrSbo);
        mma_bf16(taddr, dh, dh, kIdescBf16, (it > 0 || j > 0) ? 1u : 0u);
        mma_bf16(taddr, dh, dl, kIdescBf16, 1u);
        mma_bf16(taddr, dl, dh, kIdescBf16, 1u);
      }
      mma_commit(&bars[s]);
    }
    __syncthreads();
  }
  // wait for the last stage's MMAs (they complete in order), then read D
  if (it > 0) {
    const int64_t last = it - 1;
    if (!mbar_wait(&bars[last & 1], (uint32_t)((last >> 1) & 1))) ok = false;
  }
  tc_fence_after();
  const int row = warp * 32 + (tid & 31);
  float* out = partial + (int64_t)blockIdx.x * kSrRows * kSrRows + (int64_t)row * kSrRows;
  if (ok && it > 0) {
#pragma unroll
    for (int c = 0; c < kSrRows; c += 32) {
      float v[32];
      tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) out[c + i] = v[i];
    }
  } else {
    for (int c = 0; c < kSrRows; ++c) out[c] = 0.f;
  }
  if (!ok && (tid & 31) == 0) atomicOr(error, kStatusLimit);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, kSrRows);
}


// ---------------------------------------------------------------------------
// Gram kernel, streamed form (P a multiple of 4, so that the rows of O are
// 16-byte strided): one CTA per SM over a contiguous range of K tiles,
// warp-specialised.  The producer warp loads each tile (all rows x 64 FP32
// columns) with two 2-D tensor copies of 128 x 32 values (rows >= n and
// columns >= P arrive as zeros), 128-byte swizzled so that the converters'
// 16-byte reads are conflict-free, plus the tile's 64 means with a bulk copy,
// into one of kBulkStages stages (completion counted in bytes on the stage's
// mbarrier); kBulkConverters warps centre, scale and split a stage into the
// bf16 hi / lo operand tiles (two operand stages) and release the FP32 stage;
// one thread of the MMA warp issues the tile's four MMAs (M = 128, N = 256: A = hi,
// B = hi followed by lo, giving [hi hi^T | hi lo^T] in 256 TMEM columns; lo hi^T is
// the transpose of the second half, added when the partials are summed) and commits them to
// the operand stage's mbarrier, which releases it to the converters.  Every
// wait is bounded; a wait that runs out stops the CTA's loop and flags the error.
// ---------------------------------------------------------------------------
constexpr int kBulkConverters = 16;
constexpr int kConvSteps = (kSrRows / 8) * (kSrKTile / 16) / kBulkConverters;   // steps a converter warp owns
constexpr int kBulkProducer = kBulkConverters;  // warp indices
constexpr int kBulkMma = kBulkConverters + 1;
constexpr int kBulkThreads = 32 * (kBulkConverters + 2);
constexpr int kBulkStages = 4;
constexpr int kBoxCols = 32;                                   // 128 bytes: the swizzle span
constexpr int kBoxBytes = kSrRows * kBoxCols * 4;              // 16 KB
constexpr int kBulkStageBytes = 2 * kBoxBytes;                 // 64 columns
constexpr int kBulkMeanOff = kBulkStages * kBulkStageBytes;
constexpr int kBulkOpOff = kBulkMeanOff + kBulkStages * kSrKTile * 4;
constexpr int kBulkSmem = kBulkOpOff + 2 * 2 * kSrTileBytes + 1024;
static_assert(kBulkOpOff % 1024 == 0 && kBulkStageBytes % 1024 == 0, "swizzled stages and operand tiles on 1 KB");

__global__ void __launch_bounds__(kBulkThreads, 1)
    gram_bulk_kernel(const __grid_constant__ CUtensorMap omap, int n, int64_t P, const float* __restrict__ m,
                     const float* __restrict__ sw, int64_t tiles_per_cta, float* __restrict__ partial,
                     int32_t* __restrict__ error) {
  extern __shared__ __align__(1024) unsigned char sr_smem[];
  __shared__ uint64_t full[kBulkStages], empty[kBulkStages], opfull[2], opempty[2];
  __shared__ uint32_t s_taddr;
  __shared__ float s_sw[kSrRows];
  __shared__ int s_fail;
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)sr_smem + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n_tiles = (P + kSrKTile - 1) / kSrKTile;
  const int64_t t0 = (int64_t)blockIdx.x * tiles_per_cta;
  const int64_t t1 = t0 + tiles_per_cta < n_tiles ? t0 + tiles_per_cta : n_tiles;
  const int64_t nt = t1 > t0 ? t1 - t0 : 0;
  if (tid == 0) {
    for (int s = 0; s < kBulkStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kBulkConverters);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&opfull[s], kBulkConverters);
      mbar_init(&opempty[s], 1);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < kSrRows) s_sw[tid] = tid < n ? sw[tid] : 0.f;
  {  // operand rows the converters never write (>= n rounded up to 8) stay zero
    uint4* op = reinterpret_cast<uint4*>(base + kBulkOpOff);
    for (int i = tid; i < 2 * 2 * kSrTileBytes / 16; i += blockDim.x) op[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (warp == 0) {
    tmem_alloc(&s_taddr, 2 * kSrRows);
    tmem_relinquish();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  bool ok = true;
  if (warp == kBulkProducer) {
    int64_t issued = 0;
    if (lane == 0) {
      for (int64_t it = 0; it < nt; ++it) {
        const int s = (int)(it % kBulkStages);
        if (it >= kBulkStages && !mbar_wait(&empty[s], (uint32_t)(((it / kBulkStages) - 1) & 1))) { ok = false; break; }
        if (*(volatile int*)&s_fail) break;
        const int64_t k0 = (t0 + it) * kSrKTile;
        const uint32_t mbytes = 4u * (uint32_t)(P - k0 < kSrKTile ? P - k0 : kSrKTile);
        unsigned char* st = base + s * kBulkStageBytes;
        mbar_expect_tx(&full[s], (uint32_t)kBulkStageBytes + mbytes);
        tma_load_2d(st, &omap, (int)k0, 0, &full[s]);
        tma_load_2d(st + kBoxBytes, &omap, (int)k0 + kBoxCols, 0, &full[s]);
        bulk_g2s(base + kBulkMeanOff + s * kSrKTile * 4, m + k0, mbytes, &full[s]);
        issued = it + 1;
      }
      // no copy may still be landing when the CTA leaves: wait for the last fill of every stage
      for (int64_t it = issued > kBulkStages ? issued - kBulkStages : 0; it < issued; ++it)
        if (!mbar_wait(&full[it % kBulkStages], (uint32_t)((it / kBulkStages) & 1))) ok = false;
    }
    __syncwarp();
  } else if (warp == kBulkMma) {
    for (int64_t it = 0; it < nt; ++it) {
      const int s2 = (int)(it & 1);
      if (!mbar_wait(&opfull[s2], (uint32_t)((it >> 1) & 1))) { ok = false; break; }
      if (*(volatile int*)&s_fail) break;
      if (lane == 0) {
        tc_fence_after();
        const uint32_t sh = smem_u32(base + kBulkOpOff + s2 * 2 * kSrTileBytes);
#pragma unroll
        for (int j = 0; j < kSrKTile / 16; ++j) {
          const uint32_t adv = (uint32_t)j * 2 * kSrLbo;
          const uint64_t dh = umma_desc(sh + adv, kSrLbo, kSrSbo);   // A: hi; B: hi then lo (256 rows)
          mma_bf16(taddr, dh, dh, kIdescBf16N256, (it > 0 || j > 0) ? 1u : 0u);
        }
        mma_commit(&opempty[s2]);
      }
      __syncwarp();
    }
  } else {
    // this warp's steps (at most kConvSteps): a step = 8 rows x two core matrices along K,
    // lane (row r % 8, half of 8 k) of core matrix 2 q + lane / 16, so that the warp's
    // 8-byte stores fill 256 contiguous bytes; the lane's offsets are fixed for all tiles
    const int n_steps = ((n + 7) / 8) * (kSrKTile / 16);
    int in_off[kConvSteps], k_of[kConvSteps];
    uint32_t op_off[kConvSteps];
    float scale[kConvSteps];
#pragma unroll
    for (int q = 0; q < kConvSteps; ++q) {
      const int step = warp + q * kBulkConverters;
      const int rg = step / (kSrKTile / 16);
      const int kc = (step % (kSrKTile / 16)) * 2 + (lane >> 4);
      const int r = step < n_steps ? rg * 8 + ((lane >> 1) & 7) : 0;
      const int k = kc * 8 + (lane & 1) * 4;
      k_of[q] = k;
      in_off[q] = (k >> 5) * kBoxBytes + r * 128 + ((((k & 31) >> 2) ^ (r & 7)) << 4);  // 128-byte swizzle
      op_off[q] = tile_off(r, k);
      scale[q] = s_sw[r];   // 0 for rows >= n
    }
    for (int64_t it = 0; it < nt; ++it) {
      const int s = (int)(it % kBulkStages), s2 = (int)(it & 1);
      if (!mbar_wait(&full[s], (uint32_t)((it / kBulkStages) & 1))) { ok = false; break; }
      if (it >= 2 && !mbar_wait(&opempty[s2], (uint32_t)(((it >> 1) - 1) & 1))) { ok = false; break; }
      if (*(volatile int*)&s_fail) break;
      const unsigned char* st = base + s * kBulkStageBytes;
      const float* mm = reinterpret_cast<const float*>(base + kBulkMeanOff + s * kSrKTile * 4);
      unsigned char* hi = base + kBulkOpOff + s2 * 2 * kSrTileBytes;
      unsigned char* lo = hi + kSrTileBytes;
      const int cols = (int)(P - (t0 + it) * kSrKTile < kSrKTile ? P - (t0 + it) * kSrKTile : kSrKTile);
      // rows >= n arrive as zeros with a zero scale; columns >= P (no mean copied) give 0
      float4 o[kConvSteps], mv[kConvSteps];
#pragma unroll
      for (int q = 0; q < kConvSteps; ++q) {
        if (warp + q * kBulkConverters < n_steps) {
          o[q] = *reinterpret_cast<const float4*>(st + in_off[q]);
          mv[q] = *reinterpret_cast<const float4*>(mm + k_of[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < kConvSteps; ++q) {
        if (warp + q * kBulkConverters >= n_steps) continue;
        const int k = k_of[q];
        const float sr = scale[q];
        const float v[4] = {k + 0 < cols ? sr * (o[q].x - mv[q].x) : 0.f, k + 1 < cols ? sr * (o[q].y - mv[q].y) : 0.f,
                            k + 2 < cols ? sr * (o[q].z - mv[q].z) : 0.f, k + 3 < cols ? sr * (o[q].w - mv[q].w) : 0.f};
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          h[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
          l[j] = v[j] - h[j];
        }
        *reinterpret_cast<uint2*>(hi + op_off[q]) = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
        *reinterpret_cast<uint2*>(lo + op_off[q]) = make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&opfull[s2]);
        mbar_arrive(&empty[s]);
      }
    }
  }
  if (!ok) atomicExch(&s_fail, 1);
  __syncthreads();
  // the last tile's MMAs complete after all earlier ones: wait for its commit, then read D
  bool done = !s_fail;
  if (done && nt > 0) done = mbar_wait(&opempty[(nt - 1) & 1], (uint32_t)(((nt - 1) >> 1) & 1));
  tc_fence_after();
  if (warp < 4) {
    const int row = warp * 32 + lane;
    float* out = partial + ((int64_t)blockIdx.x * kSrRows + row) * (2 * kSrRows);   // [hi hi^T | hi lo^T] row
    if (done && nt > 0) {
#pragma unroll 1
      for (int c = 0; c < 2 * kSrRows; c += 32) {
        float v[32];
        tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) out[c + i] = v[i];
      }
    } else {
      for (int c = 0; c < 2 * kSrRows; ++c) out[c] = 0.f;
    }
  }
  if (!done && nt > 0 && tid == 0) atomicOr(error, kStatusLimit);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, 2 * kSrRows);
}

// The tensor map of O [n rows][P columns] FP32 (row stride 4 P bytes) with 128 x 32 boxes,
// 128-byte swizzle, zeros outside; the driver's encoder is fetched once through the runtime.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

static bool make_o_map(CUtensorMap* map, const float* O, int n, int64_t P) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)P * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kBoxCols, (cuuint32_t)kSrRows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(O), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// weights, column mean, Gram sum + regularised solve, step
// ---------------------------------------------------------------------------
// w = p / sum p (p = exp(2 (a - max a))), sqrt(w) as FP32 for the Gram kernel and FP64
__global__ void sr_weights_kernel(int n, const double* __restrict__ a, double* __restrict__ w,
                                  float* __restrict__ swf, float* __restrict__ wf) {
  __shared__ double red[kSrRows / 32];
  __shared__ double s_max, s_sum;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const double at = t < n ? a[t] : -DBL_MAX;
  double v = at;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (t == 0) {
    double m = red[0];
    for (int i = 1; i < kSrRows / 32; ++i) m = fmax(m, red[i]);
    s_max = m;
  }
  __syncthreads();
  const double p = t < n ? exp(2.0 * (at - s_max)) : 0.0;
  v = p;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (t == 0) {
    double sum = 0.0;
    for (int i = 0; i < kSrRows / 32; ++i) sum += red[i];
    s_sum = sum;
  }
  __syncthreads();
  if (t < n) {
    const double wt = p / s_sum;
    w[t] = wt;
    swf[t] = (float)sqrt(wt);
    wf[t] = (float)wt;
  }
}

// m_p = sum_x w_x O_xp (FP64 accumulation over the N_SR rows), stored FP32
__global__ void sr_mean_kernel(int n, int64_t P, const float* __restrict__ O, const double* __restrict__ w,
                               float* __restrict__ m) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int x = 0; x < n; ++x) s += __ldg(w + x) * (double)__ldg(O + (int64_t)x * P + p);
    m[p] = (float)s;
  }
}

// Four columns a thread (P a multiple of 4), the rows' loads four at a time in flight: m_p =
// sum_x w_x O_xp with FP32 products summed with compensation (TwoSum), stored FP32
__global__ void sr_mean4_kernel(int n, int64_t P, const float* __restrict__ O, const float* __restrict__ wf,
                                float* __restrict__ m) {
  const int64_t P4 = P / 4;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P4; q += (int64_t)gridDim.x * blockDim.x) {
    const float4* col = reinterpret_cast<const float4*>(O) + q;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    int x = 0;
    for (; x + 4 <= n; x += 4) {
      float4 o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) o[u] = __ldg(col + (int64_t)(x + u) * P4);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float wx = __ldg(wf + x + u);
        const float t[4] = {wx * o[u].x, wx * o[u].y, wx * o[u].z, wx * o[u].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float a = s[j] + t[j], bb = a - s[j];
          c[j] += (s[j] - (a - bb)) + (t[j] - bb);
          s[j] = a;
        }
      }
    }
    for (; x < n; ++x) {
      const float4 o = __ldg(col + (int64_t)x * P4);
      const float wx = __ldg(wf + x);
      const float t[4] = {wx * o.x, wx * o.y, wx * o.z, wx * o.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float a = s[j] + t[j], bb = a - s[j];
        c[j] += (s[j] - (a - bb)) + (t[j] - bb);
        s[j] = a;
      }
    }
    reinterpret_cast<float4*>(m)[q] = make_float4(s[0] + c[0], s[1] + c[1], s[2] + c[2], s[3] + c[3]);
  }
}

// The streamed kernel's partials [hi hi^T | hi lo^T] (128 x 256 each): S = their sum in CTA
// order (FP64), one thread per element, coalesced; then G(r, c) = S(r, c) + S(r, 128 + c) +
// S(c, 128 + r)  (lo hi^T = (hi lo^T)^T)
__global__ void sr_gram_sum2_kernel(int n_part, const float* __restrict__ partial, double* __restrict__ S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kSrRows * 2 * kSrRows) return;
  double s = 0.0;
  for (int q = 0; q < n_part; ++q) s += (double)__ldg(partial + (int64_t)q * kSrRows * 2 * kSrRows + i);
  S[i] = s;
}

__global__ void sr_gram_fold_kernel(int n, const double* __restrict__ S, double* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n) return;
  const int r = i / n, c = i % n;
  G[i] = S[r * 2 * kSrRows + c] + (S[r * 2 * kSrRows + kSrRows + c] + S[c * 2 * kSrRows + kSrRows + r]);
}

// G = sum of the CTAs' partials in CTA order (FP64), one thread per entry of the n x n block
__global__ void sr_gram_sum_kernel(int n, int n_part, const float* __restrict__ partial, double* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n) return;
  const int r = i / n, c = i % n;
  double s = 0.0;
  for (int q = 0; q < n_part; ++q) s += (double)__ldg(partial + (int64_t)q * kSrRows * kSrRows + r * kSrRows + c);
  G[i] = s;
}

// T = (G + G^T) / 2; (T + lambda I + c u u^T) y = eps by an L D L^T factorisation, one block of kSolveThreads
// threads.  u = sqrt(w) is a unit null vector of the exact T (Obar^T u = sum_x w_x (O_x - m)
// = 0), so the rank-one term changes y only along u, which the step Obar^T y annihilates:
// delta is that of (T + lambda I)^{-1}.  With c = tr T / n the u direction no longer has
// eigenvalue lambda, below the Gram's rounding for small lambda, which would leave
// T + lambda I indefinite and amplify y along u by 1 / lambda.
//
// The factorisation and the substitutions run in double-float arithmetic (about 48
// significant bits, FP32 pipes; this GPU's FP64 rate is a small fraction of its FP32
// rate): the matrix is assembled in FP64, split into (hi, lo) pairs, factorised as
// L D L^T right-looking (the trailing lower triangle and the right-hand side spread
// over all threads, one barrier per column), and y is returned in FP64.  A pivot that
// is not positive flags kStatusRange.
constexpr int kSolveThreads = 512;

// a - l * m in double-float (l * m's rounding error carried)
__device__ __forceinline__ df df_sub_prod(df a, df l, df m) {
  const float p = __fmul_rn(l.hi, m.hi);
  float e = __fmaf_rn(l.hi, m.hi, -p);
  e = __fmaf_rn(l.hi, m.lo, e);
  e = __fmaf_rn(l.lo, m.hi, e);
  const df s = two_sum(a.hi, -p);
  return fast_two_sum(s.hi, __fadd_rn(__fsub_rn(a.lo, e), s.lo));
}

// sqrt and reciprocal of a positive double-float: FP32 estimate and one Newton step in df
__device__ __forceinline__ df df_sqrt(df d) {
  const float r0 = sqrtf(d.hi);
  const df sq = {__fmul_rn(r0, r0), __fmaf_rn(r0, r0, -__fmul_rn(r0, r0))};
  const float resid = __fadd_rn(__fsub_rn(d.hi, sq.hi), __fsub_rn(d.lo, sq.lo));
  return fast_two_sum(r0, __fdiv_rn(resid, __fmul_rn(2.f, r0)));
}
__device__ __forceinline__ df df_recip(df d) {
  const float r0 = __fdiv_rn(1.f, d.hi);
  const df pr = df_mul(d, df{r0, 0.f});          // d r0 = 1 - e
  const float e = __fsub_rn(__fsub_rn(1.f, pr.hi), pr.lo);
  return fast_two_sum(r0, __fmul_rn(r0, e));
}

// The system, assembled over many blocks: T = (G + G^T) / 2 (written out when asked),
// A = T + lambda I + c u u^T with c = tr T / n (each thread sums the diagonal itself), and
// eps, both split into double-float pairs for the solve
__global__ void sr_assemble_kernel(int n, const double* __restrict__ G, const double* __restrict__ w,
                                   const double* __restrict__ eloc, const double* __restrict__ evar,
                                   double lambda, double* __restrict__ T, float2* __restrict__ A,
                                   float2* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n) return;
  const int r = i / n, c = i % n;
  double tr = 0.0;
  for (int k = 0; k < n; ++k) tr += __ldg(G + k * n + k);
  const double v = 0.5 * (G[i] + G[c * n + r]);
  if (T) T[i] = v;
  const df a = df_from_double(v + (r == c ? lambda : 0.0) + (tr / n) * sqrt(w[r] * w[c]));
  A[i] = make_float2(a.hi, a.lo);
  if (c == 0) {
    const df e = df_from_double(sqrt(w[r]) * (eloc[r] - evar[0]));
    b[r] = make_float2(e.hi, e.lo);
  }
}

__global__ void __launch_bounds__(kSolveThreads) sr_solve_kernel(int n, const float2* __restrict__ Ag,
                                                                  const float2* __restrict__ bg,
                                                                  double* __restrict__ y,
                                                                  int32_t* __restrict__ error) {
  extern __shared__ df A[];   // [n][n], then b[n], the pivots' reciprocals [n], the triangle table
  df* b = A + n * n;
  df* rinv = b + n;
  uint16_t* tri_rc = reinterpret_cast<uint16_t*>(rinv + n);   // e -> (r, c), e = r (r + 1) / 2 + c
  const int t = threadIdx.x;
  for (int i = t; i < n * n; i += blockDim.x) {
    const float2 v = __ldg(Ag + i);
    A[i] = df{v.x, v.y};
  }
  if (t < n) {
    const float2 v = __ldg(bg + t);
    b[t] = df{v.x, v.y};
  }
  for (int r = t; r < n; r += blockDim.x)
    for (int c = 0; c <= r; ++c) tri_rc[r * (r + 1) / 2 + c] = (uint16_t)(r | (c << 8));
  __syncthreads();
  // A = L D L^T, right-looking: column j is kept unscaled (l_ij = A_ij / d_j is formed where it
  // is used), the trailing lower triangle and the right-hand side lose column j's
  // contribution, so that b ends as L^{-1} b; one barrier per column
  for (int j = 0; j < n; ++j) {
    df d = A[j * n + j];
    if (!(d.hi > 0.f)) {
      if (t == 0) atomicOr(error, kStatusRange);
      d = df{FLT_MIN, 0.f};
    }
    const df inv = df_recip(d);
    if (t == 0) rinv[j] = inv;
    const int m = n - j - 1;
    const int tri = m * (m + 1) / 2;
    for (int e = t; e < tri + m; e += blockDim.x) {
      if (e >= tri) {  // right-hand side entry j + 1 + (e - tri)
        const int ii = j + 1 + (e - tri);
        b[ii] = df_sub_prod(b[ii], A[ii * n + j], df_mul(b[j], inv));
        continue;
      }
      const uint32_t rc = tri_rc[e];
      const int ii = j + 1 + (int)(rc & 255u), kk = j + 1 + (int)(rc >> 8);
      A[ii * n + kk] = df_sub_prod(A[ii * n + kk], A[ii * n + j], df_mul(A[kk * n + j], inv));
    }
    __syncthreads();
  }
  // D^{-1}, then L^T y = D^{-1} L^{-1} b column by column from the last (L^T_{ij} = A_ji / d_i)
  if (t < n) b[t] = df_mul(b[t], rinv[t]);
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const df bj = b[j];
    for (int i = t; i < j; i += blockDim.x) b[i] = df_sub_prod(b[i], df_mul(A[j * n + i], rinv[i]), bj);
    __syncthreads();
  }
  if (t < n) y[t] = df_to_double(b[t]);
}

// delta_p = sum_x sqrt(w_x) (O_xp - m_p) y_x, FP32 compensated (two-sum) accumulation
__global__ void sr_step_kernel(int n, int64_t P, const float* __restrict__ O, const float* __restrict__ m,
                               const float* __restrict__ sw, const double* __restrict__ y, double* __restrict__ delta) {
  __shared__ float cy[kSrRows];
  if (threadIdx.x < n) cy[threadIdx.x] = (float)(y[threadIdx.x] * (double)sw[threadIdx.x]);
  __syncthreads();
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const float mp = __ldg(m + p);
    float s = 0.f, c = 0.f;
    for (int x = 0; x < n; ++x) {
      const float tm = cy[x] * (__ldg(O + (int64_t)x * P + p) - mp);
      const float u = s + tm;
      const float bb = u - s;
      c += (s - (u - bb)) + (tm - bb);
      s = u;
    }
    delta[p] = (double)s + (double)c;
  }
}

// the same with four columns a thread (P a multiple of 4), the rows' loads four at a time in flight
__global__ void sr_step4_kernel(int n, int64_t P, const float* __restrict__ O, const float* __restrict__ m,
                                const float* __restrict__ sw, const double* __restrict__ y, double* __restrict__ delta) {
  __shared__ float cy[kSrRows];
  if (threadIdx.x < n) cy[threadIdx.x] = (float)(y[threadIdx.x] * (double)sw[threadIdx.x]);
  __syncthreads();
  const int64_t P4 = P / 4;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P4; q += (int64_t)gridDim.x * blockDim.x) {
    const float4* col = reinterpret_cast<const float4*>(O) + q;
    const float4 mq = __ldg(reinterpret_cast<const float4*>(m) + q);
    const float mp[4] = {mq.x, mq.y, mq.z, mq.w};
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    auto add_row = [&](const float4& o, float cx) {
      const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float tm = cx * (ov[j] - mp[j]);
        const float a = s[j] + tm, bb = a - s[j];
        c[j] += (s[j] - (a - bb)) + (tm - bb);
        s[j] = a;
      }
    };
    int x = 0;
    for (; x + 4 <= n; x += 4) {
      float4 o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) o[u] = __ldg(col + (int64_t)(x + u) * P4);
#pragma unroll
      for (int u = 0; u < 4; ++u) add_row(o[u], cy[x + u]);
    }
    for (; x < n; ++x) add_row(__ldg(col + (int64_t)x * P4), cy[x]);
    double2* d = reinterpret_cast<double2*>(delta + 4 * q);
    d[0] = make_double2((double)s[0] + (double)c[0], (double)s[1] + (double)c[1]);
    d[1] = make_double2((double)s[2] + (double)c[2], (double)s[3] + (double)c[3]);
  }
}

// ---------------------------------------------------------------------------
// the n_sr samples of highest probability: stable descending order of log |psi|
// (ties by index), by a 64-bit radix sort of order-preserving keys
// ---------------------------------------------------------------------------
__global__ void sr_top_keys_kernel(int64_t n, const double* __restrict__ a, uint64_t* __restrict__ keys,
                                   int32_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = a[i];
    if (v == 0.0) v = 0.0;
    const uint64_t u = (uint64_t)__double_as_longlong(v);
    keys[i] = ~((u >> 63) ? ~u : (u | 0x8000000000000000ull));
    idx[i] = (int32_t)i;
  }
}

int64_t sr_top_scratch_bytes(int64_t n) {
  const int64_t m = std::max<int64_t>(n, 1);
  return a256r(8 * m) * 2 + a256r(4 * m) * 2 + a256r(4 * 256 * sort_blocks(m)) + a256r(4 * sort_scan_partials(m));
}

cudaError_t launch_sr_top(int64_t n, const double* a, int64_t n_sr, int32_t* out, void* scratch, cudaStream_t s) {
  char* p = (char*)scratch;
  const int64_t m = std::max<int64_t>(n, 1);
  uint64_t* k0 = (uint64_t*)p; p += a256r(8 * m);
  uint64_t* k1 = (uint64_t*)p; p += a256r(8 * m);
  int32_t* i0 = (int32_t*)p; p += a256r(4 * m);
  int32_t* i1 = (int32_t*)p; p += a256r(4 * m);
  int32_t* hist = (int32_t*)p; p += a256r(4 * 256 * sort_blocks(m));
  int32_t* part = (int32_t*)p;
  sr_top_keys_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * num_sms())), 256, 0, s>>>(
      n, a, k0, i0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  uint64_t* kbuf[2] = {k1, k0};
  int32_t* ibuf[2] = {i1, i0};
  int out_buf = -1;
  if ((e = launch_sort_words(k0, i0, n, 1, 8, kbuf, ibuf, hist, part, &out_buf, s)) != cudaSuccess) return e;
  const int32_t* order = out_buf >= 0 ? ibuf[out_buf] : i0;
  return cudaMemcpyAsync(out, order, 4 * std::min(n, n_sr), cudaMemcpyDeviceToDevice, s);
}

struct SrScratch {
  double* w;
  float* sw;
  float* wf;
  float* m;
  float* partial;
  double* G;
  double* S;        // [128][256] sums of the streamed kernel's partials
  float2* Adf;      // [n][n] the assembled system, double-float
  float2* bdf;      // [n]
  double* y;
  int32_t* error;
  int64_t n_part;
  int64_t bytes;
};

static SrScratch sr_scratch_view(char* base, int64_t P, int n_part) {
  SrScratch v;
  std::memset(&v, 0, sizeof(v));
  int64_t off = 0;
  auto take = [&](int64_t bytes) { char* p = base ? base + off : nullptr; off = a256r(off + bytes); return p; };
  v.error = (int32_t*)take(256);
  v.w = (double*)take(8 * kSrRows);
  v.sw = (float*)take(4 * kSrRows);
  v.wf = (float*)take(4 * kSrRows);
  v.y = (double*)take(8 * kSrRows);
  v.G = (double*)take(8 * kSrRows * kSrRows);
  v.S = (double*)take(8 * kSrRows * 2 * kSrRows);
  v.Adf = (float2*)take(8 * kSrRows * kSrRows);
  v.bdf = (float2*)take(8 * kSrRows);
  v.m = (float*)take(4 * std::max<int64_t>(P, 1) + 16);
  v.partial = (float*)take(4 * (int64_t)n_part * kSrRows * kSrRows);
  v.n_part = n_part;
  v.bytes = off;
  return v;
}

static int sr_parts() { return 2 * num_sms(); }

int64_t sr_scratch_bytes(int64_t P) { return sr_scratch_view(nullptr, P, sr_parts()).bytes; }

cudaError_t launch_sr_step(int n, int64_t P, const float* O, const double* a, const double* eloc,
                           const double* evar, double lambda, void* scratch, double* delta, double* T,
                           int32_t* status_out, cudaStream_t s) {
  const SrScratch sc = sr_scratch_view((char*)scratch, P, sr_parts());
  cudaError_t e = cudaMemsetAsync(sc.error, 0, 4, s);
  if (e != cudaSuccess) return e;
  sr_weights_kernel<<<1, kSrRows, 0, s>>>(n, a, sc.w, sc.sw, sc.wf);
  const int sms = num_sms();
  const int64_t n_tiles = (P + kSrKTile - 1) / kSrKTile;
  // rows of O on 16-byte boundaries: the streamed kernels (float4 columns, bulk copies)
  const bool streamed = (P % 4) == 0 && (((uintptr_t)O) & 15) == 0 && (((uintptr_t)delta) & 15) == 0;
  CUtensorMap omap;
  const bool tiled = streamed && P < (int64_t(1) << 31) && make_o_map(&omap, O, n, P);
  const int stream_grid = (int)std::max<int64_t>(1, std::min<int64_t>((P / 4 + 255) / 256, 4 * sms));
  if (streamed)
    sr_mean4_kernel<<<stream_grid, 256, 0, s>>>(n, P, O, sc.wf, sc.m);
  else
    sr_mean_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, 8 * sms)), 256, 0, s>>>(n, P, O,
                                                                                                          sc.w, sc.m);
  int n_part;
  if (tiled) {
    n_part = (int)std::min<int64_t>(sms, n_tiles);
    const int64_t per = (n_tiles + n_part - 1) / n_part;
    if ((e = cudaFuncSetAttribute(gram_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBulkSmem)) !=
        cudaSuccess)
      return e;
    gram_bulk_kernel<<<n_part, kBulkThreads, kBulkSmem, s>>>(omap, n, P, sc.m, sc.sw, per, sc.partial, sc.error);
  } else {
    n_part = (int)sc.n_part;
    const int64_t per = (n_tiles + n_part - 1) / n_part;
    if ((e = cudaFuncSetAttribute(gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSrSmem)) != cudaSuccess)
      return e;
    gram_kernel<<<n_part, kSrThreads, kSrSmem, s>>>(n, P, O, sc.m, sc.sw, per, sc.partial, sc.error);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t solve_smem = sizeof(df) * (size_t)(n * n + 2 * n) + sizeof(uint16_t) * (size_t)(n * (n + 1) / 2);
  if ((e = cudaFuncSetAttribute(sr_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_smem)) !=
      cudaSuccess)
    return e;
  if (tiled) {
    sr_gram_sum2_kernel<<<kSrRows * 2 * kSrRows / 256, 256, 0, s>>>(n_part, sc.partial, sc.S);
    sr_gram_fold_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(n, sc.S, sc.G);
  } else
    sr_gram_sum_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(n, n_part, sc.partial, sc.G);
  sr_assemble_kernel<<<(n * n + 255) / 256, 256, 0, s>>>(n, sc.G, sc.w, eloc, evar, lambda, T, sc.Adf, sc.bdf);
  sr_solve_kernel<<<1, kSolveThreads, solve_smem, s>>>(n, sc.Adf, sc.bdf, sc.y, sc.error);
  if (streamed)
    sr_step4_kernel<<<stream_grid, 256, 0, s>>>(n, P, O, sc.m, sc.sw, sc.y, delta);
  else
    sr_step_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, 8 * sms)), 256, 0, s>>>(
        n, P, O, sc.m, sc.sw, sc.y, delta);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int32_t err = 0;
  if ((e = cudaMemcpyAsync(&err, sc.error, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *status_out = err;
  return cudaSuccess;
}

}  // namespace nqs
