// Sample staging and FindCoupledPairs, LoopOverTerms schedule (Alg. 2A).
//
// Membership test "x' in U" (Alg. 2A): a GF(2)-linear 32-bit hash
// h(v) = XOR_{b in v} R[b] makes the hash of a candidate x' = x XOR XY one XOR
// of two precomputed values, h(x) ^ h(XY).  A blocked Bloom filter of U
// (one 32-bit word per key, two bits set) lives in shared memory and rejects
// most candidates; survivors are verified in an open-addressing table of U
// (linear probing, load <= 1/2) that stays resident in L2.
#include "device_util.cuh"
#include "nqs_internal.cuh"

namespace nqs {

// --------------------------------------------------------------------------
// staging: hash of each sample, hash table and Bloom filter of U
// --------------------------------------------------------------------------
template <int W>
__global__ void stage_kernel(const uint64_t* __restrict__ U, int64_t n, int n_qubits,
                             const uint32_t* __restrict__ basis, int64_t cap, uint32_t wmask,
                             uint32_t* __restrict__ hx_out, int32_t* __restrict__ table,
                             uint32_t* __restrict__ bloom, int32_t* __restrict__ status) {
  __shared__ uint32_t R[64 * W];
  for (int i = threadIdx.x; i < 64 * W; i += blockDim.x) R[i] = basis[i];
  __syncthreads();
  const int tail = n_qubits - 64 * (W - 1);
  const uint64_t tail_mask = tail == 64 ? ~0ull : ((1ull << tail) - 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v[W];
    load_words<W>(U + i * W, v);
    if (v[W - 1] & ~tail_mask) atomicOr(status, kStatusBadBits);
    uint32_t h = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint64_t m = v[w];
      while (m) {
        int b = __ffsll((long long)m) - 1;
        h ^= R[64 * w + b];
        m &= m - 1;
      }
    }
    hx_out[i] = h;
    int64_t slot = h & (cap - 1);
    bool placed = false;
    for (int64_t it = 0; it < cap; ++it) {
      int prev = atomicCAS(&table[slot], -1, (int)i);
      if (prev == -1) { placed = true; break; }
      bool eq = true;
#pragma unroll
      for (int w = 0; w < W; ++w) eq = eq && (__ldg(U + (int64_t)prev * W + w) == v[w]);
      if (eq) { atomicOr(status, kStatusDuplicate); placed = true; break; }
      slot = (slot + 1) & (cap - 1);
    }
    if (!placed) atomicOr(status, kStatusLimit);
    atomicOr(&bloom[h & wmask], bloom_bits(h));
  }
}

cudaError_t launch_stage(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                         const StageHeader& L, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4 * num_sms());
  auto* hx = (uint32_t*)(stage + L.off_hx);
  auto* table = (int32_t*)(stage + L.off_table);
  auto* bloom = (uint32_t*)(stage + L.off_bloom);
  auto* status = (int32_t*)(stage + offsetof(StageHeader, status));
  uint32_t wmask = (uint32_t)(L.nwords - 1);
  switch (ham->W) {
    case 1: stage_kernel<1><<<blocks, 256, 0, s>>>(U, n, ham->n_qubits, ham->hash_basis, L.cap, wmask, hx, table, bloom, status); break;
    case 2: stage_kernel<2><<<blocks, 256, 0, s>>>(U, n, ham->n_qubits, ham->hash_basis, L.cap, wmask, hx, table, bloom, status); break;
    case 3: stage_kernel<3><<<blocks, 256, 0, s>>>(U, n, ham->n_qubits, ham->hash_basis, L.cap, wmask, hx, table, bloom, status); break;
    default: stage_kernel<4><<<blocks, 256, 0, s>>>(U, n, ham->n_qubits, ham->hash_basis, L.cap, wmask, hx, table, bloom, status); break;
  }
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// LoopOverTerms search.  One warp scans kRowsPerWarp rows against the whole
// search table; lanes take 32 consecutive slots, whose hash low bits are
// distinct, so each shared-memory Bloom probe is conflict-free.  Filter hits
// go to a per-warp queue; a full queue is verified lane-parallel against the
// hash table.  COUNT writes per-row pair counts; FILL writes (j, k) at the
// offsets of a previous COUNT, in the same deterministic order.
// --------------------------------------------------------------------------
constexpr int kSearchThreads = 1024;
constexpr int kSearchWarps = kSearchThreads / 32;

template <int W, bool FILL>
__device__ __forceinline__ void flush_queue(const uint32_t* q, int qn, int64_t r0,
                                            const uint64_t* __restrict__ U,
                                            const uint32_t* __restrict__ hx,
                                            const int32_t* __restrict__ table, int64_t capmask,
                                            const uint32_t* __restrict__ srch_hash,
                                            const uint32_t* __restrict__ srch_id,
                                            const uint64_t* __restrict__ xy,
                                            int64_t (&acc)[kRowsPerWarp],
                                            uint32_t* __restrict__ pair_j,
                                            uint32_t* __restrict__ pair_k, int32_t* status) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  for (int e0 = 0; e0 < qn; e0 += 32) {
    const int e = e0 + lane;
    bool found = false;
    uint32_t j = 0, id = 0, r = 0;
    if (e < qn) {
      const uint32_t v = q[e];
      r = v >> 28;
      const uint32_t pos = v & 0x0FFFFFFFu;
      id = __ldg(srch_id + pos);
      if (id != kDummy) {
        const int64_t row = r0 + r;
        uint64_t key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = __ldg(U + row * W + w) ^ __ldg(xy + (int64_t)id * W + w);
        int64_t slot = (__ldg(hx + row) ^ __ldg(srch_hash + pos)) & capmask;
        int64_t it = 0;
        for (; it <= capmask; ++it) {
          const int t = __ldg(table + slot);
          if (t < 0) break;
          bool eq = true;
#pragma unroll
          for (int w = 0; w < W; ++w) eq = eq && (__ldg(U + (int64_t)t * W + w) == key[w]);
          if (eq) { found = true; j = (uint32_t)t; break; }
          slot = (slot + 1) & capmask;
        }
        if (it > capmask) atomicOr(status, kStatusLimit);
      }
    }
#pragma unroll
    for (int rr = 0; rr < kRowsPerWarp; ++rr) {
      const uint32_t m = __ballot_sync(kFull, found && r == (uint32_t)rr);
      if (FILL) {
        if (found && r == (uint32_t)rr) {
          const int64_t p = acc[rr] + __popc(m & lt);
          pair_j[p] = j;
          pair_k[p] = id;
        }
      }
      acc[rr] += __popc(m);
    }
  }
}

template <int W, bool FILL>
__global__ void __launch_bounds__(kSearchThreads, 1)
pairs_terms_kernel(const uint64_t* __restrict__ U, const uint32_t* __restrict__ hx,
                   const int32_t* __restrict__ table, int64_t capmask,
                   const uint32_t* __restrict__ bloom_g, uint32_t wmask, int nwords,
                   const uint32_t* __restrict__ srch_hash, const uint32_t* __restrict__ srch_id,
                   int64_t n_groups, const uint64_t* __restrict__ xy, int has_diag,
                   int64_t row_begin, int64_t row_end, int64_t* __restrict__ rp,
                   uint32_t* __restrict__ pair_j, uint32_t* __restrict__ pair_k,
                   int32_t* __restrict__ status) {
  extern __shared__ uint32_t smem[];
  uint32_t* bloom = smem;
  uint32_t* queue = smem + nwords;
  {
    const uint4* src = reinterpret_cast<const uint4*>(bloom_g);
    uint4* dst = reinterpret_cast<uint4*>(bloom);
    for (int i = threadIdx.x; i < nwords / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  uint32_t* q = queue + warp * kQueueCap;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t n_rows = row_end - row_begin;
  const int64_t n_batches = (n_rows + kRowsPerWarp - 1) / kRowsPerWarp;
  const int64_t tw = (int64_t)gridDim.x * kSearchWarps;
  const int64_t pbase = FILL ? rp[0] : 0;
  for (int64_t bt = (int64_t)blockIdx.x * kSearchWarps + warp; bt < n_batches; bt += tw) {
    const int64_t r0 = row_begin + bt * kRowsPerWarp;
    uint32_t hr[kRowsPerWarp];
    bool val[kRowsPerWarp];
    int64_t acc[kRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r) {
      const int64_t row = r0 + r;
      val[r] = row < row_end;
      hr[r] = val[r] ? __ldg(hx + row) : 0u;
      acc[r] = (FILL && val[r]) ? rp[row - row_begin] - pbase : 0;
      if (has_diag && val[r]) {  // the diagonal pair (x, x) comes first
        if (FILL && lane == 0) {
          pair_j[acc[r]] = (uint32_t)row;
          pair_k[acc[r]] = 0u;
        }
        acc[r] += 1;
      }
    }
    int qn = 0;
    for (int64_t g = 0; g < n_groups; ++g) {
      const uint32_t pos = (uint32_t)(g * 32 + lane);
      const uint32_t hk = __ldg(srch_hash + pos);
#pragma unroll
      for (int r = 0; r < kRowsPerWarp; ++r) {
        const uint32_t s = hr[r] ^ hk;
        const uint32_t w = bloom[s & wmask];
        const bool hit = val[r] && bloom_hit(w, s);
        const uint32_t bal = __ballot_sync(kFull, hit);
        if (bal) {
          if (hit) q[qn + __popc(bal & lt)] = ((uint32_t)r << 28) | pos;
          qn += __popc(bal);
        }
      }
      if (qn > kQueueCap - 32 * kRowsPerWarp) {
        __syncwarp();
        flush_queue<W, FILL>(q, qn, r0, U, hx, table, capmask, srch_hash, srch_id, xy, acc, pair_j,
                             pair_k, status);
        __syncwarp();
        qn = 0;
      }
    }
    __syncwarp();
    flush_queue<W, FILL>(q, qn, r0, U, hx, table, capmask, srch_hash, srch_id, xy, acc, pair_j,
                         pair_k, status);
    __syncwarp();
    if (!FILL && lane == 0) {
#pragma unroll
      for (int r = 0; r < kRowsPerWarp; ++r)
        if (val[r]) rp[r0 + r - row_begin] = acc[r];
    }
  }
}

template <int W, bool FILL>
static cudaError_t launch_terms_w(const nqs_ham* ham, const uint64_t* U, const char* stage,
                                  const StageHeader& L, int64_t rb, int64_t re, int64_t* rp,
                                  uint32_t* pj, uint32_t* pk, cudaStream_t s) {
  const size_t smem = 4 * (size_t)L.nwords + (size_t)kSearchWarps * kQueueCap * 4;
  auto kern = pairs_terms_kernel<W, FILL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kSearchThreads, smem);
  if (occ < 1) occ = 1;
  const int64_t batches = (re - rb + kRowsPerWarp - 1) / kRowsPerWarp;
  const int64_t need = (batches + kSearchWarps - 1) / kSearchWarps;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * occ));
  kern<<<blocks, kSearchThreads, smem, s>>>(
      U, (const uint32_t*)(stage + L.off_hx), (const int32_t*)(stage + L.off_table), L.cap - 1,
      (const uint32_t*)(stage + L.off_bloom), (uint32_t)(L.nwords - 1), (int)L.nwords,
      ham->srch_hash, ham->srch_id, ham->n_srch / 32, ham->xy, ham->has_diag, rb, re, rp, pj, pk,
      (int32_t*)(stage + offsetof(StageHeader, status)));
  return cudaGetLastError();
}

cudaError_t launch_pairs_terms(const nqs_ham* ham, const uint64_t* U, const char* stage,
                               const StageHeader& L, int64_t rb, int64_t re, int64_t* rp,
                               uint32_t* pj, uint32_t* pk, bool fill, cudaStream_t s) {
  if (ham->n_srch >= (int64_t(1) << 28)) return cudaErrorInvalidValue;
  switch (ham->W) {
    case 1: return fill ? launch_terms_w<1, true>(ham, U, stage, L, rb, re, rp, pj, pk, s)
                        : launch_terms_w<1, false>(ham, U, stage, L, rb, re, rp, pj, pk, s);
    case 2: return fill ? launch_terms_w<2, true>(ham, U, stage, L, rb, re, rp, pj, pk, s)
                        : launch_terms_w<2, false>(ham, U, stage, L, rb, re, rp, pj, pk, s);
    case 3: return fill ? launch_terms_w<3, true>(ham, U, stage, L, rb, re, rp, pj, pk, s)
                        : launch_terms_w<3, false>(ham, U, stage, L, rb, re, rp, pj, pk, s);
    default: return fill ? launch_terms_w<4, true>(ham, U, stage, L, rb, re, rp, pj, pk, s)
                         : launch_terms_w<4, false>(ham, U, stage, L, rb, re, rp, pj, pk, s);
  }
}

cudaError_t launch_pairs_batch(const nqs_ham*, const uint64_t*, const char*, const StageHeader&,
                               int64_t, int64_t, int64_t*, uint32_t*, uint32_t*, bool, cudaStream_t) {
  return cudaErrorNotSupported;
}

// --------------------------------------------------------------------------
// inclusive scan of int64 counts in place (three phases, deterministic)
// --------------------------------------------------------------------------
constexpr int kScanTile = 1024;

__global__ void scan_tiles(int64_t* __restrict__ d, int64_t n, int64_t* __restrict__ partial) {
  __shared__ int64_t sh[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int t = threadIdx.x;
  sh[t] = (base + t < n) ? d[base + t] : 0;
  __syncthreads();
  for (int o = 1; o < kScanTile; o <<= 1) {
    int64_t v = (t >= o) ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  if (base + t < n) d[base + t] = sh[t];
  if (t == kScanTile - 1) partial[blockIdx.x] = sh[t];
}

__global__ void scan_partials(int64_t* __restrict__ partial, int64_t m) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t run = 0;
    for (int64_t i = 0; i < m; ++i) {
      int64_t v = partial[i];
      partial[i] = run;
      run += v;
    }
  }
}

__global__ void scan_add(int64_t* __restrict__ d, int64_t n, const int64_t* __restrict__ partial) {
  const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  if (i < n) d[i] += partial[blockIdx.x];
}

cudaError_t launch_scan(int64_t* data, int64_t n, char* stage, const StageHeader& L, cudaStream_t s) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int64_t* partial = (int64_t*)(stage + L.off_scan);
  if (tiles > L.scan_blocks) return cudaErrorInvalidValue;
  scan_tiles<<<(unsigned)tiles, kScanTile, 0, s>>>(data, n, partial);
  scan_partials<<<1, 32, 0, s>>>(partial, tiles);
  scan_add<<<(unsigned)tiles, kScanTile, 0, s>>>(data, n, partial);
  return cudaGetLastError();
}

}  // namespace nqs
