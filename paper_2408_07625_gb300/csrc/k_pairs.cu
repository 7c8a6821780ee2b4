// Sample staging and FindCoupledPairs: LoopOverTerms (Alg. 2A) and
// LoopOverBatch (Alg. 2B).
//
// Membership test "x' in U" (Algs. 2A, 2B): a GF(2)-linear 32-bit hash
// h(v) = XOR_{b in v} R[b] makes the hash of a candidate x' = x XOR XY one XOR
// of two precomputed values, h(x) ^ h(XY).  A blocked Bloom filter of U (one
// 32-bit word per key, three bits set) lives in shared memory and rejects most
// candidates; survivors are verified in a bucketed table of U resident in L2:
// 32-byte buckets of four (hash tag, index) slots, at most one key per bucket
// on average, so a miss reads one sector; only a tag match reads the sample.
//
// Oriented LoopOverTerms.  x XOR x' = XY is symmetric, so a coupled pair
// {x, x'} with x != x' needs to be found once: exactly one of the two has
// XY's highest set qubit t, so it is found either from the one with bit t set
// or from the one with bit t clear, whichever side of t holds fewer samples.
// The search table is grouped by t and staging lists, per qubit t, the
// samples on that side; a work item probes 8 samples of one list against the
// patterns of the matching group.  For peaked molecular batches most qubits
// are nearly always empty or nearly always occupied, which cuts the probes by
// an order of magnitude against probing every (sample, pattern).  Each pair found is written to both of its rows,
// and each row is then sorted by column, so the list of a row (the diagonal
// pair first, then ascending column index) depends on the row alone.
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "device_util.cuh"
#include "nqs_internal.cuh"

namespace nqs {

// --------------------------------------------------------------------------
// staging: hash of each sample, bucketed table and Bloom filter of U, and the
// number of samples with each qubit set
// --------------------------------------------------------------------------

// lane b of the warp adds, for each 32-qubit slice c, the number of the warp's
// samples with qubit 32 c + b set (one ballot per qubit)
template <int W>
__device__ __forceinline__ void count_qubits(const uint64_t (&v)[W], uint32_t (&mine)[2 * W]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 0; w < W; ++w)
#pragma unroll
    for (int b = 0; b < 64; ++b) {
      const uint32_t c = __popc(__ballot_sync(kFull, (uint32_t)(v[w] >> b) & 1u));
      mine[2 * w + (b >> 5)] += (lane == (b & 31)) ? c : 0u;
    }
}

template <int W>
__global__ void stage_kernel(const uint64_t* __restrict__ U, int64_t n, int n_qubits,
                             const uint32_t* __restrict__ basis, int64_t cap, uint32_t wmask,
                             uint32_t* __restrict__ hx_out, unsigned long long* __restrict__ table,
                             uint32_t* __restrict__ bloom, uint32_t* __restrict__ qcnt,
                             int32_t* __restrict__ status) {
  __shared__ uint32_t R[64 * W];
  __shared__ uint32_t qc[64 * W];
  for (int i = threadIdx.x; i < 64 * W; i += blockDim.x) {
    R[i] = basis[i];
    qc[i] = 0u;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int tail = n_qubits - 64 * (W - 1);
  const uint64_t tail_mask = tail == 64 ? ~0ull : ((1ull << tail) - 1);
  uint32_t mine[2 * W];
#pragma unroll
  for (int c = 0; c < 2 * W; ++c) mine[c] = 0u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    const bool valid = i < n;
    uint64_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = valid ? __ldg(U + i * W + w) : 0ull;
    if (v[W - 1] & ~tail_mask) atomicOr(status, kStatusBadBits);
    v[W - 1] &= tail_mask;  // bits >= N are an error (reported); the lists never hold them
    count_qubits<W>(v, mine);
    if (!valid) continue;
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
    const unsigned long long key = (unsigned long long)h | ((unsigned long long)i << 32);
    int64_t b = h & (cap - 1);
    bool placed = false;
    for (int64_t it = 0; it < cap && !placed; ++it) {
      unsigned long long* bk = table + b * 4;
      for (int k = 0; k < 4; ++k) {
        const unsigned long long prev = atomicCAS(bk + k, ~0ull, key);
        if (prev == ~0ull) { placed = true; break; }
        if ((uint32_t)prev == h) {  // same tag: compare the samples themselves
          const int64_t o = (int64_t)(prev >> 32);
          bool eq = true;
#pragma unroll
          for (int w = 0; w < W; ++w) eq = eq && (__ldg(U + o * W + w) == v[w]);
          if (eq) { atomicOr(status, kStatusDuplicate); placed = true; break; }
        }
      }
      b = (b + 1) & (cap - 1);
    }
    if (!placed) atomicOr(status, kStatusLimit);
    atomicOr(&bloom[h & wmask], bloom_bits(h));
  }
#pragma unroll
  for (int c = 0; c < 2 * W; ++c)
    if (mine[c]) atomicAdd(&qc[32 * c + lane], mine[c]);
  __syncthreads();
  for (int q = threadIdx.x; q < 64 * W; q += blockDim.x)
    if (qc[q]) atomicAdd(&qcnt[q], qc[q]);
}

// Exclusive scan of n <= 256 values in shared memory by one warp (each lane
// takes a contiguous run of ceil(n / 32) values); the total goes to *total.
__device__ __forceinline__ void warp_exclusive_scan(int64_t* v, int n, int64_t* total) {
  const int lane = threadIdx.x & 31;
  const int per = (n + 31) / 32;
  const int lo = lane * per < n ? lane * per : n;
  const int hi = lo + per < n ? lo + per : n;
  int64_t sum = 0;
  for (int i = lo; i < hi; ++i) sum += v[i];
  int64_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  int64_t run = incl - sum;
  for (int i = lo; i < hi; ++i) {
    const int64_t x = v[i];
    v[i] = run;
    run += x;
  }
  if (lane == 31 && total) *total = incl;
}

// Side of qubit q whose list the search uses: the samples with bit q set if
// they are at most half of the batch, else the samples with bit q clear.
__device__ __forceinline__ bool list_side(uint32_t qcnt_q, int64_t n) { return 2 * (int64_t)qcnt_q <= n; }
__device__ __forceinline__ int64_t list_len(uint32_t qcnt_q, int64_t n) {
  return list_side(qcnt_q, n) ? (int64_t)qcnt_q : n - (int64_t)qcnt_q;
}

// Per-qubit lists: for every qubit q, the samples on the rarer side of q (bit
// set, or bit clear).  Each block takes a contiguous slice of U, counts its
// samples per qubit, reserves that many places in each list (one atomic per
// qubit and block), then writes the samples (warp-aggregated positions; the
// order inside a list is irrelevant).
template <int W>
__global__ void qubit_rows_kernel(const uint64_t* __restrict__ U, int64_t n, int n_qubits, int64_t per_block,
                                  const uint32_t* __restrict__ qcnt, uint32_t* __restrict__ qcur,
                                  uint32_t* __restrict__ qrows) {
  __shared__ int64_t base[64 * W];
  __shared__ uint32_t cnt[64 * W];
  __shared__ uint64_t side[W];  // bit q: the list of qubit q holds the samples with bit q set
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t s0 = (int64_t)blockIdx.x * per_block;
  const int64_t s1 = s0 + per_block < n ? s0 + per_block : n;
  const int tail = n_qubits - 64 * (W - 1);
  const uint64_t tail_mask = tail == 64 ? ~0ull : ((1ull << tail) - 1);
  for (int q = threadIdx.x; q < 64 * W; q += blockDim.x) cnt[q] = 0u;
  if (threadIdx.x < W) side[threadIdx.x] = 0ull;
  __syncthreads();
  for (int q = threadIdx.x; q < 64 * W; q += blockDim.x)
    if (list_side(qcnt[q], n)) atomicOr((unsigned long long*)&side[q >> 6], 1ull << (q & 63));
  uint32_t mine[2 * W];
#pragma unroll
  for (int c = 0; c < 2 * W; ++c) mine[c] = 0u;
  for (int64_t i0 = s0 + (threadIdx.x & ~31); i0 < s1; i0 += blockDim.x) {
    const int64_t i = i0 + lane;
    uint64_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = i < s1 ? __ldg(U + i * W + w) : 0ull;
    v[W - 1] &= tail_mask;
    count_qubits<W>(v, mine);
  }
#pragma unroll
  for (int c = 0; c < 2 * W; ++c)
    if (mine[c]) atomicAdd(&cnt[32 * c + lane], mine[c]);
  __syncthreads();
  for (int q = threadIdx.x; q < 64 * W; q += blockDim.x) {
    base[q] = list_len(qcnt[q], n);
    if (!((side[q >> 6] >> (q & 63)) & 1ull)) cnt[q] = (uint32_t)(s1 > s0 ? s1 - s0 : 0) - cnt[q];
  }
  __syncthreads();
  if (threadIdx.x < 32) warp_exclusive_scan(base, 64 * W, nullptr);
  __syncthreads();
  for (int q = threadIdx.x; q < 64 * W; q += blockDim.x) {
    if (cnt[q]) base[q] += atomicAdd(&qcur[q], cnt[q]);
    cnt[q] = 0u;
  }
  __syncthreads();
  for (int64_t i0 = s0 + (threadIdx.x & ~31); i0 < s1; i0 += blockDim.x) {
    const int64_t i = i0 + lane;
    uint64_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = i < s1 ? __ldg(U + i * W + w) : 0ull;
    v[W - 1] &= tail_mask;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint64_t sd = side[w];
#pragma unroll 4
      for (int b = 0; b < 64; ++b) {
        const bool set = i < s1 && (((v[w] ^ ~sd) >> b) & 1ull);  // on the listed side of qubit 64 w + b
        const uint32_t m = __ballot_sync(kFull, set);
        if (m == 0u) continue;
        uint32_t at = 0u;
        if (lane == __ffs(m) - 1) at = atomicAdd(&cnt[64 * w + b], (uint32_t)__popc(m));
        at = __shfl_sync(kFull, at, __ffs(m) - 1);
        if (set) qrows[base[64 * w + b] + at + __popc(m & lt)] = (uint32_t)i;
      }
    }
  }
}

cudaError_t launch_stage(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                         const StageHeader& L, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(stage + L.off_table, 0xFF, 32 * L.cap, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(stage + L.off_bloom, 0, 4 * L.nwords, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(stage + L.off_q, 0, 2 * 4 * 64 * kMaxWords, s)) != cudaSuccess) return e;
  if (n == 0) return cudaSuccess;
  auto* hx = (uint32_t*)(stage + L.off_hx);
  auto* table = (unsigned long long*)(stage + L.off_table);
  auto* bloom = (uint32_t*)(stage + L.off_bloom);
  auto* status = (int32_t*)(stage + offsetof(StageHeader, status));
  auto* qcnt = (uint32_t*)(stage + L.off_q);
  auto* qcur = qcnt + 64 * kMaxWords;
  auto* qrows = (uint32_t*)(stage + L.off_qrows);
  const uint32_t wmask = (uint32_t)(L.nwords - 1);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4 * num_sms());
  const int qblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * num_sms()));
  const int64_t per_block = (((n + qblocks - 1) / qblocks) + 31) & ~int64_t(31);
#define NQS_STAGE(WW)                                                                                    \
  case WW:                                                                                               \
    stage_kernel<WW><<<blocks, 256, 0, s>>>(U, n, ham->n_qubits, ham->hash_basis, L.cap, wmask, hx,      \
                                            table, bloom, qcnt, status);                                 \
    if ((e = cudaGetLastError()) != cudaSuccess) return e;                                               \
    qubit_rows_kernel<WW><<<qblocks, 256, 0, s>>>(U, n, ham->n_qubits, per_block, qcnt, qcur, qrows);                   \
    break;
  switch (ham->W) {
    NQS_STAGE(1)
    NQS_STAGE(2)
    NQS_STAGE(3)
    default:
    NQS_STAGE(4)
  }
#undef NQS_STAGE
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// one-pass scratch: three uint32 arrays of found pairs (i, j, k), handed out
// to the search warps in chunks of kRecChunk records; the unused tail of a
// warp's last chunk is marked with i = kNoRecord
// --------------------------------------------------------------------------
static inline int64_t a256(int64_t v) { return (v + 255) & ~int64_t(255); }
constexpr int kSearchThreads = 1024;
constexpr int kSearchWarps = kSearchThreads / 32;
constexpr int kRecChunk = 128;
constexpr uint32_t kNoRecord = 0xFFFFFFFFu;

static inline int64_t rec_slack() { return (int64_t)num_sms() * kSearchWarps * kRecChunk; }

// records for up to max_pairs + slack pairs (a record serves at most two rows
// and at least one of the range), then one 64-bit sort key per pair
int64_t pair_scratch_bytes(int64_t rows, int64_t max_pairs) {
  (void)rows;
  const int64_t m = std::max<int64_t>(max_pairs, 1);
  return 256 + 3 * a256(4 * (m + rec_slack())) + a256(8 * m);
}

PairScratch pair_scratch_view(void* base, int64_t rows, int64_t bytes) {
  (void)rows;
  PairScratch sc;
  char* p = (char*)base;
  sc.cursor = (int64_t*)p;
  // 12 bytes of records per pair (plus the slack) and 8 of sort key, each array 256-byte aligned
  int64_t m = std::max<int64_t>((bytes - 256 - 12 * rec_slack()) / 20, 0);  // at most ~50 too large
  while (m > 0 && pair_scratch_bytes(rows, m) > bytes) --m;
  sc.max_pairs = m;
  sc.max_rec = m > 0 ? m + rec_slack() : 0;
  const int64_t stride = a256(4 * std::max<int64_t>(sc.max_rec, 1));
  sc.rec_i = (uint32_t*)(p + 256);
  sc.rec_j = (uint32_t*)(p + 256 + stride);
  sc.rec_k = (uint32_t*)(p + 256 + 2 * stride);
  sc.keys = (uint64_t*)(p + 256 + 3 * stride);
  return sc;
}

// --------------------------------------------------------------------------
// Oriented LoopOverTerms search.  A warp takes work items from a global
// counter; item = (segment s of the search table, 8 consecutive entries of
// the list of samples on the rarer side of qubit t_s, a run of groups of the
// segment).  Lane t scans slot 32 g + t of each group g; the 32 slots of a
// group have at most two patterns per hash residue mod 32, so the 32
// filter-word loads of one row touch each shared-memory bank at most twice.
// Per slot a lane keeps a bit mask of the rows whose filter test passed; each
// pass goes to the warp's queue as (candidate hash, slot, row), and the queue
// is verified against the hash table of U, lane-parallel, when the next group
// might not fit.  1024 threads per block (one block per SM: the filter takes
// up to 128 KB of shared memory), at most 64 registers a thread.
// --------------------------------------------------------------------------
constexpr int R = kRowsPerWarp;
constexpr int kMaxSegs = 64 * kMaxWords;
// work items a warp takes per atomic, and search-table groups per work item
// (bounds an item's length): launch parameters (SearchTune), 4 and 16 by default
constexpr int kQueueCap = 32 * R;   // per-warp queue of filter passes: one group adds at most 32 R
constexpr int kGens = 2;            // row caches per warp; a queue entry names the one it refers to
// queue entry: x = candidate hash h(x) ^ h(XY) (after phase 1 of the
// verification: the first tag match, bit 31 set for the slow path);
// y = slot | row << 28 | cache << 31 (slots < 2^28)
constexpr uint32_t kSlotMask = (1u << 28) - 1u;

struct TermsArgs {
  const uint64_t* U;
  const uint32_t* hx;
  const unsigned long long* table;
  int64_t capmask;
  const uint32_t* bloom_g;
  uint32_t wmask;
  int nwords;
  const uint32_t* srch_hash;
  const uint64_t* srch_rec;
  int rec_words;
  const int4* segs;
  int n_segs;
  int nq;
  int64_t n_unq;
  const uint32_t* qcnt;
  const uint32_t* qrows;
  int64_t row_begin, row_end;
  int64_t* counts;        // COUNT / EMIT: per-row counts of the range
  const int64_t* rp;      // FILL: CSR offsets of the range
  unsigned long long* cursor;  // FILL: per-row write cursors (relative to the row's start)
  uint32_t* pair_j;
  uint32_t* pair_k;
  PairScratch sc;         // EMIT
  int32_t* status;
  unsigned long long* item_counter;
  int items_per_grab;
  int part, n_parts;      // slice `part` of `n_parts` equal slices of the work items
  int groups_per_item;
};

template <int W>
struct RowCache {   // per-warp copies of the rows of the item (two generations)
  int32_t row[kGens][R];
  uint32_t hx[kGens][R];
  uint32_t cnt[kGens][R];   // COUNT / EMIT: pairs found for the row since the cache was filled
  uint64_t x[kGens][R][W];
};

// Place one pair in row r (relative to the range) at the row's next free
// position; a row that is already full (counts that do not match this
// search, e.g. a changed batch) flags the status instead of writing past it.
__device__ __forceinline__ void place_pair(const int64_t* rp, int64_t r, unsigned long long* cursor, uint32_t* pj,
                                           uint32_t* pk, uint32_t col, uint32_t k, int32_t* status) {
  const int64_t a = rp[r] - rp[0];
  const int64_t len = rp[r + 1] - rp[r];
  const int64_t c = (int64_t)atomicAdd(cursor + r, 1ull);
  if (c < len) {
    pj[a + c] = col;
    pk[a + c] = k;
  } else {
    atomicOr(status, kStatusLimit);
  }
}

struct RecState {  // warp-uniform: current record chunk (base < 0: none) and its fill
  int64_t base;
  int fill;
};

// One round of verified candidates (lane order).  The pair (i, j) is listed
// in row i and in row j.
template <int MODE>
__device__ __forceinline__ void emit_found(bool found, int64_t i, uint32_t j, uint32_t id, RecState& rs,
                                           const TermsArgs& a, uint32_t* icount = nullptr) {
  const int lane = threadIdx.x & 31;
  const bool in_i = found && i >= a.row_begin && i < a.row_end;
  const bool in_j = found && (int64_t)j >= a.row_begin && (int64_t)j < a.row_end;
  if (MODE == kFill) {
    if (in_i) place_pair(a.rp, i - a.row_begin, a.cursor, a.pair_j, a.pair_k, j, id, a.status);
    if (in_j) place_pair(a.rp, (int64_t)j - a.row_begin, a.cursor, a.pair_j, a.pair_k, (uint32_t)i, id, a.status);
    return;
  }
  if (MODE != kEmitHalf) {
    if (in_i) {
      if (icount) atomicAdd(icount, 1u);  // row i's shared counter, added to counts when the cache is reused
      else atomicAdd((unsigned long long*)(a.counts + (i - a.row_begin)), 1ull);
    }
    if (in_j) atomicAdd((unsigned long long*)(a.counts + ((int64_t)j - a.row_begin)), 1ull);
  }
  if (MODE == kEmit || MODE == kEmitHalf) {
    const bool keep = in_i || in_j;
    const uint32_t m = __ballot_sync(kFull, keep);
    const int n = __popc(m);
    if (n == 0) return;
    const int off = __popc(m & ((1u << lane) - 1u));
    const int room = rs.base >= 0 ? kRecChunk - rs.fill : 0;
    int64_t q = -1;
    if (off < room) q = rs.base + rs.fill + off;
    if (n > room) {  // the rest goes to a fresh chunk
      long long fresh = -1;
      if (lane == 0) {
        const unsigned long long c = atomicAdd((unsigned long long*)a.sc.cursor, (unsigned long long)kRecChunk);
        if ((int64_t)c + kRecChunk <= a.sc.max_rec) fresh = (long long)c;
        else a.sc.cursor[1] = 1;  // scratch too small: counting goes on, the list is completed by a fill pass
      }
      fresh = __shfl_sync(kFull, fresh, 0);
      if (off >= room && fresh >= 0) q = fresh + (off - room);
      rs.base = fresh;
      rs.fill = fresh >= 0 ? n - room : kRecChunk;
    } else {
      rs.fill += n;
    }
    if (keep && q >= 0) {
      a.sc.rec_i[q] = (uint32_t)i;
      a.sc.rec_j[q] = j;
      a.sc.rec_k[q] = id;
    }
  }
}

// Exact membership of x' = x XOR XY(pos) in the bucket chain starting at
// bucket sh (slow path: full buckets, several equal tags).
template <int W>
__device__ __noinline__ bool verify_slow(const uint64_t* x, uint32_t pos, uint32_t sh, const TermsArgs& a,
                                         uint32_t& j) {
  const uint64_t* rec = a.srch_rec + (int64_t)pos * a.rec_words;
  uint64_t key[W];
#pragma unroll
  for (int w = 0; w < W; ++w) key[w] = x[w] ^ __ldg(rec + 1 + w);
  int64_t b = sh & a.capmask;
  for (int64_t it = 0; it <= a.capmask; ++it) {
    const uint2* bk = reinterpret_cast<const uint2*>(a.table + b * 4);
    for (int k = 0; k < 4; ++k) {
      const uint2 sl = __ldg(bk + k);
      if (sl.y == ~0u) return false;  // an empty slot ends the chain
      if (sl.x == sh) {
        bool eq = true;
#pragma unroll
        for (int w = 0; w < W; ++w) eq = eq && (__ldg(a.U + (int64_t)sl.y * W + w) == key[w]);
        if (eq) { j = sl.y; return true; }
      }
    }
    b = (b + 1) & a.capmask;
  }
  atomicOr(a.status, kStatusLimit);
  return false;
}

// Verification of queued filter passes, in two converged phases.  Phase 1
// (kWays1 entries per lane in flight): the candidate's hash picks a bucket of
// the table of U; entries with a tag match, or a full bucket, are compacted
// in place (the first tag match beside them; bit 31 when several tags match
// or the bucket is full).  Phase 2: the first tag match is confirmed exactly
// against x XOR XY (x from the row cache); otherwise, with bit 31, the slow
// path walks the chain; found pairs are emitted.
constexpr uint32_t kNoMatch = 0x7FFFFFFFu;  // no sample has this index (n_unq < 2^31)
constexpr int kWays1 = 2;
template <int W>
struct Ways2 {
  static constexpr int v = 1;
};

template <int W, int MODE>
__device__ __forceinline__ void verify_queue(uint2* q, int qn, RowCache<W>* rc, RecState& rs,
                                             const TermsArgs& a) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  int ns = 0;
  for (int e0 = 0; e0 < qn; e0 += 32 * kWays1) {
    uint2 ent[kWays1];
    uint4 b0[kWays1], b1[kWays1];
#pragma unroll
    for (int u = 0; u < kWays1; ++u) {
      const int e = e0 + u * 32 + lane;
      ent[u] = q[e < qn ? e : 0];
    }
#pragma unroll
    for (int u = 0; u < kWays1; ++u) {
      const uint4* bk = reinterpret_cast<const uint4*>(a.table + (int64_t)(ent[u].x & a.capmask) * 4);
      b0[u] = __ldg(bk);
      b1[u] = __ldg(bk + 1);
    }
#pragma unroll
    for (int u = 0; u < kWays1; ++u) {
      // tag matches among occupied slots; slots fill in order, so slot 3 occupied = full
      const uint32_t s = ent[u].x;
      const uint32_t mm = (uint32_t)(b0[u].x == s && b0[u].y != ~0u) | ((uint32_t)(b0[u].z == s && b0[u].w != ~0u) << 1) |
                          ((uint32_t)(b1[u].x == s && b1[u].y != ~0u) << 2) | ((uint32_t)(b1[u].z == s && b1[u].w != ~0u) << 3);
      const uint32_t jc = mm == 0u ? kNoMatch : (mm & 1u) ? b0[u].y : (mm & 2u) ? b0[u].w : (mm & 4u) ? b1[u].y : b1[u].w;
      const bool full = b1[u].w != ~0u;
      const bool keep = e0 + u * 32 + lane < qn && (mm != 0u || full);
      const uint32_t m = __ballot_sync(kFull, keep);
      __syncwarp();  // every lane holds this round's entries before any is overwritten
      if (keep) q[ns + __popc(m & lt)] = make_uint2(jc | (((mm & (mm - 1u)) != 0u || full) ? 0x80000000u : 0u), ent[u].y);
      ns += __popc(m);
    }
  }
  __syncwarp();
  constexpr int K2 = Ways2<W>::v;
  for (int e0 = 0; e0 < ns; e0 += 32 * K2) {
    uint2 ent[K2];
    uint64_t rec0[K2], xy[K2][W], uj[K2][W];
#pragma unroll
    for (int u = 0; u < K2; ++u) {
      const int e = e0 + u * 32 + lane;
      ent[u] = q[e < ns ? e : 0];
      const uint32_t jc = ent[u].x & kNoMatch;
      const uint64_t* rec = a.srch_rec + (int64_t)(ent[u].y & kSlotMask) * a.rec_words;
      rec0[u] = __ldg(rec);
#pragma unroll
      for (int w = 0; w < W; ++w) {
        xy[u][w] = __ldg(rec + 1 + w);
        uj[u][w] = jc != kNoMatch ? __ldg(a.U + (int64_t)jc * W + w) : ~0ull;
      }
    }
#pragma unroll
    for (int u = 0; u < K2; ++u) {
      const bool live = e0 + u * 32 + lane < ns;
      const int r = (int)((ent[u].y >> 28) & 7u), gen = (int)(ent[u].y >> 31);
      const uint32_t id = (uint32_t)(rec0[u] >> 32);
      uint32_t j = ent[u].x & kNoMatch;
      uint64_t x[W];
      bool eq = j != kNoMatch;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        x[w] = rc->x[gen][r][w];
        eq = eq && ((x[w] ^ xy[u][w]) == uj[u][w]);
      }
      bool found = live && eq;
      if (live && !eq && (ent[u].x >> 31))
        found = verify_slow<W>(x, ent[u].y & kSlotMask, rc->hx[gen][r] ^ (uint32_t)rec0[u], a, j);
      found = found && id != kDummy;  // padding slots carry XY = 0 and never count
      if (e0 + u * 32 < ns)
        emit_found<MODE>(found, (int64_t)rc->row[gen][r], j, id, rs, a, const_cast<uint32_t*>(&rc->cnt[gen][r]));
    }
  }
  __syncwarp();
}

// Oriented LoopOverTerms search kernel.  The filter test of sample hash hr
// against pattern hash hk: v = hr ^ hk is the candidate's hash; word
// v mod nwords of the filter; the three bit positions f are the 5-bit fields
// of v at bits 15, 20 and 25, and bit f - 1 (mod 32) is tested as bit 31 of
// the word rotated right by f, which shifts straight into the row mask.
template <int W, int MODE>
__global__ void __launch_bounds__(kSearchThreads, 1) pairs_terms_kernel(const TermsArgs a) {
  if (MODE == kFill && (*(volatile int32_t*)a.status & kStatusCapacity)) return;  // buffers too small
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int64_t s_qoff[kMaxSegs];
  __shared__ int64_t s_cum[kMaxSegs + 1];
  uint32_t* bloom = smem;
  RowCache<W>* caches = reinterpret_cast<RowCache<W>*>(smem + a.nwords);
  uint2* queues = reinterpret_cast<uint2*>(caches + kSearchWarps);
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.bloom_g);
    uint4* dst = reinterpret_cast<uint4*>(bloom);
    for (int i = threadIdx.x; i < a.nwords / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  // list offsets per qubit; work items per segment (exclusive prefix, total last)
  for (int qq = threadIdx.x; qq < a.nq; qq += blockDim.x) s_qoff[qq] = list_len(a.qcnt[qq], a.n_unq);
  for (int sg = threadIdx.x; sg < a.n_segs; sg += blockDim.x) {
    const int4 g = __ldg(&a.segs[sg]);
    s_cum[sg] = (list_len(a.qcnt[g.x], a.n_unq) + R - 1) / R * ((g.z - g.y + a.groups_per_item - 1) / a.groups_per_item);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    warp_exclusive_scan(s_qoff, a.nq, nullptr);
    warp_exclusive_scan(s_cum, a.n_segs, s_cum + a.n_segs);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  uint2* q = queues + warp * kQueueCap;
  const uint32_t lt = (1u << lane) - 1u;
  RowCache<W>* rc = caches + warp;
  if (lane < kGens * R) {
    rc->row[lane / R][lane % R] = -1;
    rc->cnt[lane / R][lane % R] = 0u;
  }
  __syncwarp();
  // this launch's slice of the work items
  const int64_t i_begin = s_cum[a.n_segs] * a.part / a.n_parts;
  const int64_t i_end = s_cum[a.n_segs] * (a.part + 1) / a.n_parts;
  const uint32_t wmask4 = a.wmask << 2;
  const char* bloom_bytes = reinterpret_cast<const char*>(bloom);
  RecState rs{-1, kRecChunk};
  int qn = 0;
  int cur_seg = -1;
  int64_t cur_batch = -1;
  int gen = 1;
  uint32_t qgens = 0;  // bit c: the queue holds entries of row cache c
  uint32_t hr4[R];
  uint32_t vmask = 0;
  // the rows' hashes are re-read from the row cache after every verification,
  // so that they are not held in registers across it
  auto load_rows = [&]() {
    vmask = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      hr4[r] = *reinterpret_cast<volatile const uint32_t*>(&rc->hx[gen][r]) << 2;
      if (*reinterpret_cast<volatile const int32_t*>(&rc->row[gen][r]) >= 0) vmask |= 1u << (R - 1 - r);
    }
  };
  // add the shared counters of row cache c to the rows' counts (its queue entries are verified)
  auto add_counts = [&](int c) {
    if (MODE == kCount || MODE == kEmit) {
      __syncwarp();
      if (lane < R) {
        const int32_t row = rc->row[c][lane];
        const uint32_t k = rc->cnt[c][lane];
        if (k != 0u)  // only rows of the range count
          atomicAdd((unsigned long long*)(a.counts + ((int64_t)row - a.row_begin)), (unsigned long long)k);
        rc->cnt[c][lane] = 0u;
      }
      __syncwarp();
    }
  };
  auto flush = [&]() {
    __syncwarp();
    verify_queue<W, MODE>(q, qn, rc, rs, a);
    __syncwarp();
    qn = 0;
    qgens = 0;
  };
  while (true) {
    unsigned long long itu = 0;
    if (lane == 0) itu = atomicAdd(a.item_counter, (unsigned long long)a.items_per_grab);
    const int64_t it0 = i_begin + (int64_t)__shfl_sync(kFull, itu, 0);
    if (it0 >= i_end) break;
    const int64_t it1 = it0 + a.items_per_grab < i_end ? it0 + a.items_per_grab : i_end;
    for (int64_t it = it0; it < it1; ++it) {
      int lo = 0, hi = a.n_segs;  // s_cum[lo] <= it < s_cum[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_cum[mid] <= it) lo = mid; else hi = mid;
      }
      // item = (segment, batch of R list entries, chunk of groups_per_item groups)
      const int4 sg = __ldg(&a.segs[lo]);
      const int n_chunks = (sg.z - sg.y + a.groups_per_item - 1) / a.groups_per_item;
      const int64_t local = it - s_cum[lo];
      const int64_t batch = local < 0x7FFFFFFF ? (int64_t)((uint32_t)local / (uint32_t)n_chunks) : local / n_chunks;
      const int g0 = sg.y + (int)(local - batch * n_chunks) * a.groups_per_item;
      const int g1 = g0 + a.groups_per_item < sg.z ? g0 + a.groups_per_item : sg.z;
      if (lo != cur_seg || batch != cur_batch) {  // new rows (consecutive chunks share them) in the other cache
        cur_seg = lo;
        cur_batch = batch;
        if (qgens & (1u << (gen ^ 1))) flush();  // the queue still refers to that cache
        gen ^= 1;
        add_counts(gen);
        const int64_t b0 = batch * R;
        const int64_t count_t = list_len(a.qcnt[sg.x], a.n_unq);
        __syncwarp();
        if (lane < R) {
          const bool valid = b0 + lane < count_t;
          const int32_t row = valid ? (int32_t)__ldg(a.qrows + s_qoff[sg.x] + b0 + lane) : -1;
          rc->hx[gen][lane] = valid ? __ldg(a.hx + row) : 0u;
          rc->row[gen][lane] = row;
          rc->cnt[gen][lane] = 0u;
#pragma unroll
          for (int w = 0; w < W; ++w) rc->x[gen][lane][w] = valid ? __ldg(a.U + (int64_t)row * W + w) : 0ull;
        }
        __syncwarp();
      }
      load_rows();
      const uint32_t cache_bits = (uint32_t)gen << 31;
      uint32_t hk_next = __ldg(a.srch_hash + (uint32_t)(g0 * 32 + lane));
      for (int g = g0; g < g1; ++g) {
        const uint32_t pos = (uint32_t)(g * 32 + lane);
        const uint32_t hk = hk_next;
        if (g + 1 < g1) hk_next = __ldg(a.srch_hash + pos + 32);  // next group's hashes in flight
        const uint32_t hk4 = hk << 2;
        uint32_t hm = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t v4 = hr4[r] ^ hk4;
          const uint32_t w = *reinterpret_cast<const uint32_t*>(bloom_bytes + (v4 & wmask4));
          const uint32_t t = __funnelshift_r(w, w, v4 >> 17) & __funnelshift_r(w, w, v4 >> 22) &
                             __funnelshift_r(w, w, v4 >> 27);
          hm = __funnelshift_l(t, hm, 1);  // hm << 1 | bit 31 of t
        }
        hm &= vmask;
        if (__ballot_sync(kFull, hm != 0u)) {
          // exclusive prefix of the lanes' pass counts (at most R = 8) from their bit planes
          const uint32_t c = __popc(hm);
          int excl = 0, total = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const uint32_t m = __ballot_sync(kFull, (c >> b) & 1u);
            excl += __popc(m & lt) << b;
            total += __popc(m) << b;
          }
          if (qn + total > kQueueCap) {  // verify the queue first (total <= kQueueCap fits then)
            flush();
            load_rows();
          }
          int at = qn + excl;
          while (hm) {  // one entry per passing row
            const int b = 31 - __clz(hm);
            hm &= ~(1u << b);
            const int r = R - 1 - b;
            q[at++] = make_uint2(rc->hx[gen][r] ^ hk, pos | ((uint32_t)r << 28) | cache_bits);
          }
          qn += total;
          qgens |= 1u << gen;
        }
      }
    }  // items of this grab
  }
  flush();
  add_counts(0);
  add_counts(1);
  if ((MODE == kEmit || MODE == kEmitHalf) && rs.base >= 0)  // mark the unused tail of the last chunk
    for (int f = rs.fill + lane; f < kRecChunk; f += 32) a.sc.rec_i[rs.base + f] = kNoRecord;
}

template <int W>
static size_t search_smem(int64_t nwords) {
  return 4 * (size_t)nwords + kSearchWarps * sizeof(RowCache<W>) + (size_t)kSearchWarps * kQueueCap * sizeof(uint2);
}
constexpr int64_t kMaxBloomWords = 32768;   // stage_layout caps the filter at 128 KB

// Optional timing of the search kernel for benchmarks: while enabled, each
// launch is bracketed by two CUDA events on its stream; nqs_search_time sums
// the recorded intervals (waiting for them) and forgets them.
static std::mutex g_timing_mu;
static bool g_timing_on = false;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_timing_events;

template <int W, int MODE>
static cudaError_t launch_terms_w(const TermsArgs& args, const StageHeader& L, cudaStream_t s) {
  auto kern = pairs_terms_kernel<W, MODE>;
  const size_t smem = search_smem<W>(L.nwords);
  // the attribute is set to the largest size any batch needs, not this launch's: launches of
  // several batches captured into one graph then all stay within it whatever their order
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)search_smem<W>(kMaxBloomWords));
  if (e != cudaSuccess) return e;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  {
    std::lock_guard<std::mutex> lock(g_timing_mu);
    if (g_timing_on && cudaEventCreate(&ev.first) == cudaSuccess && cudaEventCreate(&ev.second) == cudaSuccess) {
      cudaEventRecord(ev.first, s);
    } else if (ev.first) {
      cudaEventDestroy(ev.first);
      ev.first = nullptr;
    }
  }
  kern<<<num_sms(), kSearchThreads, smem, s>>>(args);
  e = cudaGetLastError();
  if (ev.first) {
    cudaEventRecord(ev.second, s);
    std::lock_guard<std::mutex> lock(g_timing_mu);
    g_timing_events.push_back(ev);
  }
  return e;
}

void search_timing(bool on) {
  std::lock_guard<std::mutex> lock(g_timing_mu);
  g_timing_on = on;
}

cudaError_t search_time(double* total_ms, int64_t* launches) {
  std::lock_guard<std::mutex> lock(g_timing_mu);
  double t = 0.0;
  cudaError_t err = cudaSuccess;
  for (auto& ev : g_timing_events) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(ev.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.first, ev.second);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    t += ms;
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  *launches = (int64_t)g_timing_events.size();
  g_timing_events.clear();
  *total_ms = t;
  return err;
}

// --------------------------------------------------------------------------
// CSR assembly: row initialisation (diagonal pair, cursors), scatter of the
// one-pass records, and the per-row sort by column.
// --------------------------------------------------------------------------

// COUNT/EMIT: counts[r] = has_diag.  FILL: the diagonal pair at the row's
// start (it leads the row and is not sorted) and cursor[r] = has_diag, or,
// with `absolute`, the row's first free position in the list (with `keys`
// the diagonal pair goes to the sort keys instead of pj/pk).  In FILL mode,
// if the pairs outgrow `capacity` or the scratch overflowed, flag the status
// and write nothing.
__global__ void pairs_init_kernel(int mode, int64_t rows, int64_t rb, int has_diag, int64_t* __restrict__ counts,
                                  const int64_t* __restrict__ rp, unsigned long long* __restrict__ cursor,
                                  int absolute, uint32_t* __restrict__ pj, uint32_t* __restrict__ pk,
                                  int64_t capacity, const int64_t* __restrict__ overflow,
                                  int32_t* __restrict__ status, uint64_t* __restrict__ keys) {
  if (mode == kFill) {
    const bool too_small = (capacity >= 0 && rp[rows] - rp[0] > capacity) || (overflow && *overflow != 0);
    if (too_small) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusCapacity);
      return;
    }
    if (*(volatile int32_t*)status & kStatusCapacity) return;
  }
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    if (mode != kFill) {
      counts[r] = has_diag;
    } else {
      const int64_t p = rp[r] - rp[0];
      cursor[r] = (unsigned long long)((absolute ? p : 0) + has_diag);
      if (has_diag) {
        if (keys) {
          keys[p] = (uint64_t)(rb + r) << 32;
        } else {
          pj[p] = (uint32_t)(rb + r);
          pk[p] = 0u;
        }
      }
    }
  }
}

// records -> sort keys grouped by row (each pair in both of its rows); the
// cursors hold each row's next free position, and no write passes the end
// of the list.  A warp's records come from few search rows, so the lanes
// sharing their first row take their places with one atomic.
__global__ void pairs_scatter_kernel(PairScratch sc, int64_t rb, int64_t re, const int64_t* __restrict__ rp,
                                     unsigned long long* __restrict__ cursor, int32_t* __restrict__ status) {
  if (*(volatile const int32_t*)status & kStatusCapacity) return;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t n_rec = *sc.cursor < sc.max_rec ? *sc.cursor : sc.max_rec;
  const uint64_t total = (uint64_t)(rp[re - rb] - rp[0]);
  const int64_t rows = re - rb;
  // warp-uniform trip count: q0 is the warp's first record
  for (int64_t q0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; q0 < n_rec;
       q0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = q0 + lane;
    const uint32_t ri = q < n_rec ? sc.rec_i[q] : kNoRecord;
    const bool live = ri != kNoRecord;
    const int64_t i = ri;
    const int64_t j = live ? (int64_t)sc.rec_j[q] : 0;
    const uint64_t k = live ? (uint64_t)sc.rec_k[q] : 0;
    // first row: one atomic per distinct row of the warp
    const int64_t r0 = i - rb;
    const bool in0 = live && r0 >= 0 && r0 < rows;
    const uint32_t peers = __match_any_sync(kFull, in0 ? ri : kNoRecord);
    const int leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (in0 && lane == leader) base = atomicAdd(cursor + r0, (unsigned long long)__popc(peers));
    base = __shfl_sync(kFull, base, leader);
    if (in0) {
      const unsigned long long pos = base + __popc(peers & lt);
      if (pos < total) sc.keys[pos] = ((uint64_t)j << 32) | k;
      else atomicOr(status, kStatusLimit);
    }
    // second row
    const int64_t r1 = j - rb;
    if (live && r1 >= 0 && r1 < rows) {
      const unsigned long long pos = atomicAdd(cursor + r1, 1ull);
      if (pos < total) sc.keys[pos] = ((uint64_t)i << 32) | k;
      else atomicOr(status, kStatusLimit);
    }
  }
}

// A pair's sort key: column above, pattern index below (the column is unique
// within a row).
__device__ __forceinline__ uint64_t pair_key(const uint64_t* keys, const uint32_t* pj, const uint32_t* pk,
                                             int64_t e) {
  return keys ? keys[e] : (((uint64_t)pj[e] << 32) | pk[e]);
}
__device__ __forceinline__ void put_pair(uint32_t* pj, uint32_t* pk, int64_t e, uint64_t key) {
  pj[e] = (uint32_t)(key >> 32);
  pk[e] = (uint32_t)key;
}

__device__ __forceinline__ void warp_exclusive_scan_u32(uint32_t* v, int n) {
  const int lane = threadIdx.x & 31;
  const int per = (n + 31) / 32;
  const int lo = lane * per < n ? lane * per : n;
  const int hi = lo + per < n ? lo + per : n;
  uint32_t sum = 0;
  for (int i = lo; i < hi; ++i) sum += v[i];
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  uint32_t run = incl - sum;
  for (int i = lo; i < hi; ++i) {
    const uint32_t x = v[i];
    v[i] = run;
    run += x;
  }
}

// One row of n <= kSortWarpMax pairs, sorted by a warp.  The keys are
// spread over B >= n / 4 buckets (B a power of two) by linear interpolation of
// the column between the row's smallest and largest; a pass counts the
// buckets, a scan turns the counts into starts, a second pass places each
// key at its bucket's next slot (shared atomics), and each lane then
// insertion-sorts its buckets.  The row's keys are read once, each lane
// holding 16 of them in registers (all loads in flight together).  Returns
// false, writing nothing, when the largest bucket holds more than kBucketMax
// keys (clustered columns): the row then goes to the block sort.
constexpr int kBucketMax = 16;
constexpr int kSortWarpBuckets = kSortWarpMax / 4;  // buckets of the warp sort: B >= n / 2, B >= 32

// Bucket of column c among B buckets spread over [cmin, cmin + span):
// ((c - cmin) * m) >> 32 with m = floor(B * 2^32 / span), one division per
// row instead of one per key.  Non-decreasing in c (so concatenated sorted
// buckets are a sorted row) and below B, since c - cmin < span; the product
// stays below B * 2^32.
__device__ __forceinline__ uint64_t bucket_scale(int B, uint64_t span) { return ((uint64_t)B << 32) / span; }
__device__ __forceinline__ uint32_t bucket_of(uint32_t c, uint32_t cmin, uint64_t m) {
  return (uint32_t)(((uint64_t)(c - cmin) * m) >> 32);
}

__device__ __forceinline__ uint32_t pair_col(const uint64_t* keys, const uint32_t* pj, int64_t e) {
  return keys ? (uint32_t)(__ldg(keys + e) >> 32) : pj[e];
}

__device__ __forceinline__ bool warp_sort_row(int64_t a, int n, const uint64_t* keys, uint32_t* pj, uint32_t* pk,
                                              uint32_t* cnt, uint64_t* buf, int32_t* status) {
  const int lane = threadIdx.x & 31;
  // the row's keys, read once: lane holds positions lane, lane + 32, ... (16 loads in flight)
  constexpr int kPer = kSortWarpMax / 32;
  uint64_t kv[kPer];
  uint32_t cmin = 0xFFFFFFFFu, cmax = 0u;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = lane + 32 * q;
    kv[q] = e < n ? pair_key(keys, pj, pk, a + e) : 0ull;
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    if (lane + 32 * q < n) {
      const uint32_t c = (uint32_t)(kv[q] >> 32);
      cmin = min(cmin, c);
      cmax = max(cmax, c);
    }
  }
  cmin = __reduce_min_sync(kFull, cmin);
  cmax = __reduce_max_sync(kFull, cmax);
  int B = 32;
  while (4 * B < n) B <<= 1;  // about four keys per bucket: B <= kSortWarpBuckets
  const uint64_t m = bucket_scale(B, (uint64_t)(cmax - cmin) + 1);
  for (int b = lane; b < B; b += 32) cnt[b] = 0u;
  __syncwarp();
  // bucket indices below B and places below n hold by construction; a
  // violation is flagged and skipped
  bool bad = false;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    if (lane + 32 * q < n) {
      const uint32_t bk = bucket_of((uint32_t)(kv[q] >> 32), cmin, m);
      if (bk < (uint32_t)B) atomicAdd(&cnt[bk], 1u);
      else bad = true;
    }
  }
  __syncwarp();
  uint32_t big = 0u;
  for (int b = lane; b < B; b += 32) big = max(big, cnt[b]);
  if (__reduce_max_sync(kFull, big) > kBucketMax) return false;
  warp_exclusive_scan_u32(cnt, B);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    if (lane + 32 * q < n) {
      const uint32_t bk = bucket_of((uint32_t)(kv[q] >> 32), cmin, m);
      const uint32_t o = bk < (uint32_t)B ? atomicAdd(&cnt[bk], 1u) : (uint32_t)n;
      if (o < (uint32_t)n) buf[o] = kv[q];
      else bad = true;
    }
  }
  if (bad) atomicOr(status, kStatusLimit);
  __syncwarp();
  for (int b = lane; b < B; b += 32) {  // bucket b now spans [cnt[b-1], cnt[b])
    const int lo = b ? (int)cnt[b - 1] : 0;
    const int hi = (int)cnt[b];
    for (int x = lo + 1; x < hi; ++x) {
      const uint64_t key = buf[x];
      int y = x - 1;
      while (y >= lo && buf[y] > key) {
        buf[y + 1] = buf[y];
        --y;
      }
      buf[y + 1] = key;
    }
  }
  __syncwarp();
  for (int e = lane; e < n; e += 32) put_pair(pj, pk, a + e, buf[e]);
  __syncwarp();
  return true;
}

constexpr int kSortWarpThreads = 256;
constexpr int kSortWarpWarps = kSortWarpThreads / 32;

// Rows of up to kSortWarpMax pairs, one warp each; longer rows, and rows
// with clustered columns, are queued for the block kernel.  The diagonal
// pair leads its row and is not sorted.  With `keys` the rows are read from
// the scatter's sort keys; without, pj/pk are sorted in place.
__global__ void __launch_bounds__(kSortWarpThreads, 3)
sort_rows_warp_kernel(const int64_t* __restrict__ rp, int64_t rows, const uint64_t* __restrict__ keys,
                      uint32_t* __restrict__ pj, uint32_t* __restrict__ pk, int has_diag, int32_t* __restrict__ big,
                      unsigned long long* __restrict__ big_count, int32_t* __restrict__ status) {
  __shared__ uint32_t s_cnt[kSortWarpWarps][kSortWarpBuckets];
  __shared__ uint64_t s_buf[kSortWarpWarps][kSortWarpMax];
  if (*(volatile const int32_t*)status & kStatusCapacity) return;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * kSortWarpWarps;
  const int64_t p0 = rp[0];
  for (int64_t r = blockIdx.x * (int64_t)kSortWarpWarps + warp; r < rows; r += nw) {
    const int64_t a = rp[r] - p0 + has_diag;
    const int64_t n = rp[r + 1] - p0 - a;
    if (n <= 0 || (n == 1 && !keys)) continue;
    const bool done = n <= kSortWarpMax && warp_sort_row(a, (int)n, keys, pj, pk, s_cnt[warp], s_buf[warp], status);
    if (!done && lane == 0) big[atomicAdd(big_count, 1ull)] = (int32_t)r;
  }
}

// Rows longer than kSortWarpMax (or with clustered columns): one block per
// row.  Rows of up to kBlockBucketKeys pairs take the warp sort's bucket
// method with the whole block; the rest (and rows whose columns cluster)
// take a bitonic network whose comparators all put the minimum at the lower
// index: for block sizes k = 2, 4, .., N, first compare i with i XOR (k - 1)
// (each position of the lower half with its mirror image), then i with
// i XOR d for d = k/4, .., 1.  In shared memory when the row fits
// (kSortBlockKeys keys, padded with +infinity), else in place in global
// memory (the sort keys when given, else pj/pk with the pattern indices moved
// along); there keys beyond the row's length act as +infinity and, sitting at
// the higher index of every comparator they take part in, never move, so no
// padding needs to be stored.
constexpr int kSortBlockThreads = 1024;
constexpr int kBlockBucketKeys = kSortBlockKeys / 2;

__device__ __forceinline__ uint32_t block_reduce_u32(uint32_t v, bool take_max, uint32_t* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = take_max ? __reduce_max_sync(kFull, v) : __reduce_min_sync(kFull, v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? sh[lane] : (take_max ? 0u : 0xFFFFFFFFu);
    t = take_max ? __reduce_max_sync(kFull, t) : __reduce_min_sync(kFull, t);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// exclusive scan of n values in shared memory by the block (each thread a
// contiguous run of ceil(n / blockDim.x) values)
__device__ __forceinline__ void block_exclusive_scan_u32(uint32_t* v, int n, uint32_t* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
  const int lo = min((int)threadIdx.x * per, n), hi = min(lo + per, n);
  uint32_t sum = 0;
  for (int i = lo; i < hi; ++i) sum += v[i];
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t wt = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
    uint32_t wi = wt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += t;
    }
    sh[lane] = wi - wt;
  }
  __syncthreads();
  uint32_t run = sh[warp] + (incl - sum);
  for (int i = lo; i < hi; ++i) {
    const uint32_t x = v[i];
    v[i] = run;
    run += x;
  }
  __syncthreads();
}

// the warp sort's bucket method with a whole block (n <= kBlockBucketKeys);
// false (nothing written) when a bucket holds more than kBucketMax keys
__device__ bool block_sort_row(int64_t a, int n, const uint64_t* keys, uint32_t* pj, uint32_t* pk, uint64_t* out,
                               uint32_t* cnt, uint32_t* sh, int32_t* status) {
  uint32_t cmin = 0xFFFFFFFFu, cmax = 0u;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const uint32_t c = pair_col(keys, pj, a + e);
    cmin = min(cmin, c);
    cmax = max(cmax, c);
  }
  cmin = block_reduce_u32(cmin, false, sh);
  cmax = block_reduce_u32(cmax, true, sh);
  int B = 32;
  while (B < n) B <<= 1;
  const uint64_t m = bucket_scale(B, (uint64_t)(cmax - cmin) + 1);
  for (int b = threadIdx.x; b < B; b += blockDim.x) cnt[b] = 0u;
  __syncthreads();
  bool bad = false;  // as in the warp sort: flagged and skipped
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const uint32_t bk = bucket_of(pair_col(keys, pj, a + e), cmin, m);
    if (bk < (uint32_t)B) atomicAdd(&cnt[bk], 1u);
    else bad = true;
  }
  __syncthreads();
  uint32_t big = 0u;
  for (int b = threadIdx.x; b < B; b += blockDim.x) big = max(big, cnt[b]);
  if (block_reduce_u32(big, true, sh) > kBucketMax) return false;
  block_exclusive_scan_u32(cnt, B, sh);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const uint64_t key = pair_key(keys, pj, pk, a + e);
    const uint32_t bk = bucket_of((uint32_t)(key >> 32), cmin, m);
    const uint32_t o = bk < (uint32_t)B ? atomicAdd(&cnt[bk], 1u) : (uint32_t)n;
    if (o < (uint32_t)n) out[o] = key;
    else bad = true;
  }
  if (bad) atomicOr(status, kStatusLimit);
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {  // bucket b now spans [cnt[b-1], cnt[b])
    const int lo = b ? (int)cnt[b - 1] : 0;
    const int hi = (int)cnt[b];
    for (int x = lo + 1; x < hi; ++x) {
      const uint64_t key = out[x];
      int y = x - 1;
      while (y >= lo && out[y] > key) {
        out[y + 1] = out[y];
        --y;
      }
      out[y + 1] = key;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) put_pair(pj, pk, a + e, out[e]);
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(kSortBlockThreads)
sort_rows_block_kernel(const int64_t* __restrict__ rp, uint64_t* __restrict__ keys, uint32_t* __restrict__ pj,
                       uint32_t* __restrict__ pk, int has_diag, const int32_t* __restrict__ big,
                       const unsigned long long* __restrict__ big_count, unsigned long long* __restrict__ big_next,
                       int32_t* __restrict__ status) {
  if (*(volatile const int32_t*)status & kStatusCapacity) return;
  extern __shared__ __align__(16) uint64_t sk[];  // [kSortBlockKeys] keys, then [kBlockBucketKeys] bucket counts
  uint32_t* scnt = reinterpret_cast<uint32_t*>(sk + kSortBlockKeys);
  __shared__ uint32_t sh[33];
  __shared__ int64_t s_row;
  const int64_t p0 = rp[0];
  const int64_t n_big = (int64_t)*big_count;
  while (true) {
    if (threadIdx.x == 0) {
      const unsigned long long t = atomicAdd(big_next, 1ull);
      s_row = (int64_t)t < n_big ? (int64_t)big[t] : -1;
    }
    __syncthreads();
    const int64_t r = s_row;
    __syncthreads();
    if (r < 0) break;
    const int64_t a = rp[r] - p0 + has_diag;
    const int64_t n = rp[r + 1] - p0 - a;
    if (n <= kBlockBucketKeys && block_sort_row(a, (int)n, keys, pj, pk, sk, scnt, sh, status)) continue;
    int64_t N = 1;
    while (N < n) N <<= 1;
    if (N <= kSortBlockKeys) {
      const int n32 = (int)n, N32 = (int)N;
      for (int e = threadIdx.x; e < N32; e += blockDim.x) sk[e] = e < n32 ? pair_key(keys, pj, pk, a + e) : ~0ull;
      __syncthreads();
      for (int k = 2; k <= N32; k <<= 1) {
        for (int m = k - 1, d = k; d > 1; d >>= 1, m = d >> 1) {
          // comparator (e, e ^ m) with e the lower index: e has bit hb = highest bit of m clear
          const int hb = (m == k - 1) ? (k >> 1) : m;
          for (int c = threadIdx.x; c < N32 / 2; c += blockDim.x) {
            const int e = ((c & ~(hb - 1)) << 1) | (c & (hb - 1));  // insert a 0 at bit hb
            const int f = e ^ m;
            const uint64_t x = sk[e], y = sk[f];
            if (y < x) { sk[e] = y; sk[f] = x; }
          }
          __syncthreads();
        }
      }
      for (int e = threadIdx.x; e < n32; e += blockDim.x) put_pair(pj, pk, a + e, sk[e]);
      __syncthreads();
    } else if (keys) {  // in place in the sort keys
      uint64_t* v = keys + a;
      for (int64_t k = 2; k <= N; k <<= 1) {
        for (int64_t m = k - 1, d = k; d > 1; d >>= 1, m = d >> 1) {
          const int64_t hb = (m == k - 1) ? (k >> 1) : m;
          for (int64_t c = threadIdx.x; c < N / 2; c += blockDim.x) {
            const int64_t e = ((c & ~(hb - 1)) << 1) | (c & (hb - 1));
            const int64_t f = e ^ m;
            if (f >= n) continue;  // +infinity partner at the higher index: nothing moves
            const uint64_t x = v[e], y = v[f];
            if (y < x) { v[e] = y; v[f] = x; }
          }
          __syncthreads();
        }
      }
      for (int64_t e = threadIdx.x; e < n; e += blockDim.x) put_pair(pj, pk, a + e, v[e]);
      __syncthreads();
    } else {  // in place in pj/pk, sorting columns and moving pattern indices along
      uint32_t* rj = pj + a;
      uint32_t* rk = pk + a;
      for (int64_t k = 2; k <= N; k <<= 1) {
        for (int64_t m = k - 1, d = k; d > 1; d >>= 1, m = d >> 1) {
          const int64_t hb = (m == k - 1) ? (k >> 1) : m;
          for (int64_t c = threadIdx.x; c < N / 2; c += blockDim.x) {
            const int64_t e = ((c & ~(hb - 1)) << 1) | (c & (hb - 1));
            const int64_t f = e ^ m;
            if (f >= n) continue;
            const uint32_t je = rj[e], jf = rj[f];
            if (jf < je) {
              const uint32_t ke = rk[e];
              rj[e] = jf; rj[f] = je;
              rk[e] = rk[f]; rk[f] = ke;
            }
          }
          __syncthreads();
        }
      }
    }
  }
}

static cudaError_t launch_sort_rows(const int64_t* rp, int64_t rows, uint64_t* keys, uint32_t* pj, uint32_t* pk,
                                    int has_diag, char* stage, const StageHeader& L, cudaStream_t s) {
  auto* ctr = (unsigned long long*)(stage + L.off_counters);
  auto* status = (int32_t*)(stage + offsetof(StageHeader, status));
  auto* big = (int32_t*)(stage + L.off_big);
  cudaError_t e = cudaMemsetAsync(ctr + kCtrBigCount, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + kSortWarpWarps - 1) / kSortWarpWarps,
                                                                  8 * num_sms()));
  sort_rows_warp_kernel<<<blocks, kSortWarpThreads, 0, s>>>(rp, rows, keys, pj, pk, has_diag, big,
                                                            ctr + kCtrBigCount, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = sizeof(uint64_t) * kSortBlockKeys + sizeof(uint32_t) * kBlockBucketKeys;
  e = cudaFuncSetAttribute(sort_rows_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  sort_rows_block_kernel<<<num_sms(), kSortBlockThreads, smem, s>>>(rp, keys, pj, pk, has_diag, big,
                                                                   ctr + kCtrBigCount, ctr + kCtrBigNext, status);
  return cudaGetLastError();
}

static cudaError_t launch_init(int mode, int64_t rows, int64_t rb, int has_diag, int64_t* counts, const int64_t* rp,
                               unsigned long long* cursor, int absolute, uint32_t* pj, uint32_t* pk,
                               int64_t capacity, const int64_t* overflow, int32_t* status, cudaStream_t s,
                               uint64_t* keys = nullptr) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, 4 * num_sms()));
  pairs_init_kernel<<<blocks, 256, 0, s>>>(mode, rows, rb, has_diag, counts, rp, cursor, absolute, pj, pk, capacity,
                                           overflow, status, keys);
  return cudaGetLastError();
}

// keys (column << 32 | pattern) -> pj, pk in list order: a coalesced pass that
// replaces the row sort when the rows stay in search order
__global__ void split_keys_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ rp, int64_t rows,
                                  uint32_t* __restrict__ pj, uint32_t* __restrict__ pk,
                                  const int32_t* __restrict__ status) {
  if (*(volatile const int32_t*)status & kStatusCapacity) return;
  const int64_t total = rp[rows] - rp[0];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t v = keys[q];
    pj[q] = (uint32_t)(v >> 32);
    pk[q] = (uint32_t)v;
  }
}

cudaError_t launch_pairs_terms(const nqs_ham* ham, const uint64_t* U, char* stage, const StageHeader& L,
                               int64_t rb, int64_t re, int64_t* rp, uint32_t* pj, uint32_t* pk, int mode,
                               const PairScratch* sc, cudaStream_t s, const SearchTune& tune) {
  if (ham->n_srch >= (int64_t(1) << 24) || ham->n_xy >= (int64_t(1) << 29)) return cudaErrorInvalidValue;
  if ((mode == kEmit || mode == kEmitHalf) && !sc) return cudaErrorInvalidValue;
  const int64_t rows = re - rb;
  auto* ctr = (unsigned long long*)(stage + L.off_counters);
  auto* status = (int32_t*)(stage + offsetof(StageHeader, status));
  auto* cursor = (unsigned long long*)(stage + L.off_rowcur);
  TermsArgs a;
  std::memset(&a, 0, sizeof(a));
  a.U = U;
  a.hx = (const uint32_t*)(stage + L.off_hx);
  a.table = (const unsigned long long*)(stage + L.off_table);
  a.capmask = L.cap - 1;
  a.bloom_g = (const uint32_t*)(stage + L.off_bloom);
  a.wmask = (uint32_t)(L.nwords - 1);
  a.nwords = (int)L.nwords;
  a.srch_hash = ham->srch_hash;
  a.srch_rec = ham->srch_rec;
  a.rec_words = ham->rec_words;
  a.segs = ham->segs;
  a.n_segs = ham->n_segs;
  a.nq = 64 * ham->W;
  a.n_unq = L.n_unq;
  a.qcnt = (const uint32_t*)(stage + L.off_q);
  a.qrows = (const uint32_t*)(stage + L.off_qrows);
  a.row_begin = rb;
  a.row_end = re;
  a.counts = mode == kFill ? nullptr : rp;
  a.rp = mode == kFill ? rp : nullptr;
  a.cursor = cursor;
  a.pair_j = pj;
  a.pair_k = pk;
  if (sc) a.sc = *sc;
  a.status = status;
  a.item_counter = ctr + kCtrItems;
  a.items_per_grab = std::max(1, tune.terms_grab);
  a.part = tune.part;
  a.n_parts = std::max(1, tune.n_parts);
  a.groups_per_item = std::max(1, tune.terms_groups);
  cudaError_t e;
  if (mode != kEmitHalf &&
      (e = launch_init(mode, rows, rb, ham->has_diag, rp, rp, cursor, 0, pj, pk, -1, nullptr, status, s)) !=
          cudaSuccess)
    return e;
  if ((mode == kEmit || mode == kEmitHalf) && (e = cudaMemsetAsync(sc->cursor, 0, 2 * sizeof(int64_t), s)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(ctr + kCtrItems, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if (ham->n_segs > 0) {
#define NQS_TERMS(WW)                                                            \
  case WW:                                                                       \
    if (mode == kCount) e = launch_terms_w<WW, kCount>(a, L, s);                 \
    else if (mode == kFill) e = launch_terms_w<WW, kFill>(a, L, s);              \
    else if (mode == kEmit) e = launch_terms_w<WW, kEmit>(a, L, s);              \
    else e = launch_terms_w<WW, kEmitHalf>(a, L, s);                             \
    break;
    switch (ham->W) {
      NQS_TERMS(1)
      NQS_TERMS(2)
      NQS_TERMS(3)
      default:
      NQS_TERMS(4)
    }
#undef NQS_TERMS
    if (e != cudaSuccess) return e;
  }
  if (mode == kFill && tune.sort_rows) return launch_sort_rows(rp, rows, nullptr, pj, pk, ham->has_diag, stage, L, s);
  return cudaSuccess;
}

// Half-stored pairs: one EMIT_HALF search over the whole batch writes every
// unordered coupled pair {x, x'} (x != x') once, as (i, j, k) with i the
// sample that found it, into the caller's arrays in per-warp chunks; unused
// slots carry i = kNoRecordSlot.  The slot cursor and overflow flag live in
// the workspace's counters.
cudaError_t launch_find_half(const nqs_ham* ham, const uint64_t* U, char* stage, const StageHeader& L,
                             uint32_t* rec_i, uint32_t* rec_j, uint32_t* rec_k, int64_t capacity,
                             cudaStream_t s, int part, int n_parts) {
  PairScratch sc;
  std::memset(&sc, 0, sizeof(sc));
  sc.cursor = (int64_t*)(stage + L.off_counters) + kCtrHalf;
  sc.max_rec = capacity;
  sc.rec_i = rec_i;
  sc.rec_j = rec_j;
  sc.rec_k = rec_k;
  SearchTune tune;
  tune.part = part;
  tune.n_parts = n_parts;
  return launch_pairs_terms(ham, U, stage, L, 0, L.n_unq, nullptr, nullptr, nullptr, kEmitHalf, &sc, s, tune);
}

// --------------------------------------------------------------------------
// Sharded search: records to the parts owning their rows, and records -> row
// counts.  A part owns the rows [bounds[p], bounds[p + 1]).
// --------------------------------------------------------------------------
__device__ __forceinline__ int owner_part(const int64_t* b, int n_parts, int64_t row) {
  int lo = 0, hi = n_parts;  // b[lo] <= row < b[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (b[mid] <= row) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr int kMaxParts = 1024;

__global__ void route_count_kernel(const uint32_t* __restrict__ ri, const uint32_t* __restrict__ rj, int64_t n,
                                   const int64_t* __restrict__ bounds, int n_parts,
                                   unsigned long long* __restrict__ counts) {
  __shared__ int64_t b[kMaxParts + 1];
  __shared__ unsigned int c[kMaxParts];
  for (int p = threadIdx.x; p <= n_parts; p += blockDim.x) b[p] = bounds[p];
  for (int p = threadIdx.x; p < n_parts; p += blockDim.x) c[p] = 0u;
  __syncthreads();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = ri[q];
    if (i == kNoRecord) continue;
    const int pa = owner_part(b, n_parts, i), pb = owner_part(b, n_parts, rj[q]);
    atomicAdd(&c[pa], 1u);
    if (pb != pa) atomicAdd(&c[pb], 1u);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n_parts; p += blockDim.x)
    if (c[p]) atomicAdd(counts + p, (unsigned long long)c[p]);
}

__global__ void route_scatter_kernel(const uint32_t* __restrict__ ri, const uint32_t* __restrict__ rj,
                                     const uint32_t* __restrict__ rk, int64_t n, const int64_t* __restrict__ bounds,
                                     int n_parts, unsigned long long* __restrict__ cursors, uint32_t* __restrict__ oi,
                                     uint32_t* __restrict__ oj, uint32_t* __restrict__ ok) {
  __shared__ int64_t b[kMaxParts + 1];
  for (int p = threadIdx.x; p <= n_parts; p += blockDim.x) b[p] = bounds[p];
  __syncthreads();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = ri[q];
    if (i == kNoRecord) continue;
    const uint32_t j = rj[q], k = rk[q];
    const int pa = owner_part(b, n_parts, i), pb = owner_part(b, n_parts, j);
    unsigned long long at = atomicAdd(cursors + pa, 1ull);
    oi[at] = i; oj[at] = j; ok[at] = k;
    if (pb != pa) {
      at = atomicAdd(cursors + pb, 1ull);
      oi[at] = i; oj[at] = j; ok[at] = k;
    }
  }
}

__global__ void records_count_kernel(const uint32_t* __restrict__ ri, const uint32_t* __restrict__ rj, int64_t n,
                                     int64_t rb, int64_t rows, unsigned long long* __restrict__ counts) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = ri[q];
    if (i == kNoRecord) continue;
    const int64_t a = (int64_t)i - rb, c = (int64_t)rj[q] - rb;
    if (a >= 0 && a < rows) atomicAdd(counts + a, 1ull);
    if (c >= 0 && c < rows) atomicAdd(counts + c, 1ull);
  }
}

static int stream_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * num_sms())); }

cudaError_t launch_route_count(const uint32_t* rec_i, const uint32_t* rec_j, int64_t n_slots, const int64_t* bounds,
                               int n_parts, unsigned long long* counts, cudaStream_t s) {
  if (n_parts < 1 || n_parts > kMaxParts) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * n_parts, s);
  if (e != cudaSuccess || n_slots <= 0) return e;
  route_count_kernel<<<stream_grid(n_slots), 256, 0, s>>>(rec_i, rec_j, n_slots, bounds, n_parts, counts);
  return cudaGetLastError();
}

cudaError_t launch_route_scatter(const uint32_t* rec_i, const uint32_t* rec_j, const uint32_t* rec_k, int64_t n_slots,
                                 const int64_t* bounds, int n_parts, unsigned long long* cursors, uint32_t* out_i,
                                 uint32_t* out_j, uint32_t* out_k, cudaStream_t s) {
  if (n_parts < 1 || n_parts > kMaxParts) return cudaErrorInvalidValue;
  if (n_slots <= 0) return cudaSuccess;
  route_scatter_kernel<<<stream_grid(n_slots), 256, 0, s>>>(rec_i, rec_j, rec_k, n_slots, bounds, n_parts, cursors,
                                                            out_i, out_j, out_k);
  return cudaGetLastError();
}

cudaError_t launch_records_count(const uint32_t* rec_i, const uint32_t* rec_j, int64_t n_rec, int64_t rb,
                                 int64_t rows, int has_diag, int64_t* counts, int32_t* status, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  cudaError_t e = launch_init(kCount, rows, rb, has_diag, counts, nullptr, nullptr, 0, nullptr, nullptr, -1, nullptr,
                              status, s);
  if (e != cudaSuccess || n_rec <= 0) return e;
  records_count_kernel<<<stream_grid(n_rec), 256, 0, s>>>(rec_i, rec_j, n_rec, rb, rows,
                                                          (unsigned long long*)counts);
  return cudaGetLastError();
}

__global__ void write_header_kernel(StageHeader h, StageHeader* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = h;
}

cudaError_t launch_write_header(const StageHeader& L, char* stage, cudaStream_t s) {
  write_header_kernel<<<1, 32, 0, s>>>(L, reinterpret_cast<StageHeader*>(stage));
  return cudaGetLastError();
}

__global__ void clear_capacity_kernel(int32_t* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAnd(status, ~kStatusCapacity);
}

// flag the capacity bit when the rows' total exceeds `capacity` (stream-ordered)
__global__ void capacity_flag_kernel(const int64_t* rp, int64_t rows, int64_t capacity, int32_t* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && rp[rows] - rp[0] > capacity) atomicOr(status, kStatusCapacity);
}

cudaError_t launch_capacity_check(const int64_t* rp, int64_t rows, int64_t capacity, char* stage, cudaStream_t s) {
  capacity_flag_kernel<<<1, 32, 0, s>>>(rp, rows, capacity, (int32_t*)(stage + offsetof(StageHeader, status)));
  return cudaGetLastError();
}

cudaError_t launch_clear_capacity(char* stage, cudaStream_t s) {
  clear_capacity_kernel<<<1, 32, 0, s>>>((int32_t*)(stage + offsetof(StageHeader, status)));
  return cudaGetLastError();
}

cudaError_t launch_pairs_compact(const nqs_ham* ham, const PairScratch& sc, char* stage, const StageHeader& L,
                                 int64_t rb, int64_t rows, const int64_t* row_ptr, uint32_t* pair_j,
                                 uint32_t* pair_k, int64_t capacity, cudaStream_t s, bool sort_rows) {
  auto* status = (int32_t*)(stage + offsetof(StageHeader, status));
  auto* cursor = (unsigned long long*)(stage + L.off_rowcur);
  const int64_t cap = std::min<int64_t>(capacity, sc.max_pairs);
  // rows left in search order: the diagonal pairs go to the keys too, and one
  // coalesced pass splits every key into pair_j/pair_k; with pair_k == NULL
  // (packed list, rows unsorted) the keys are written straight into pair_j
  PairScratch out = sc;
  const bool packed = !sort_rows && !pair_k;
  if (packed) out.keys = reinterpret_cast<uint64_t*>(pair_j);
  cudaError_t e = launch_init(kFill, rows, rb, ham->has_diag, nullptr, row_ptr, cursor, 1, pair_j, pair_k, cap,
                              sc.cursor + 1, status, s, sort_rows ? nullptr : out.keys);
  if (e != cudaSuccess) return e;
  pairs_scatter_kernel<<<8 * num_sms(), 256, 0, s>>>(out, rb, rb + rows, row_ptr, cursor, status);
  if ((e = cudaGetLastError()) != cudaSuccess || packed) return e;
  if (!sort_rows) {
    split_keys_kernel<<<8 * num_sms(), 256, 0, s>>>(sc.keys, row_ptr, rows, pair_j, pair_k, status);
    return cudaGetLastError();
  }
  return launch_sort_rows(row_ptr, rows, sc.keys, pair_j, pair_k, ham->has_diag, stage, L, s);
}

// --------------------------------------------------------------------------
// LoopOverBatch schedule (Alg. 2B).  A warp owns 8 rows and streams the
// columns j of U (lane t takes column 32c + t): d = x_r XOR U_j passes the
// cheap test "popcount(d) is the weight of some XY pattern"; survivors are
// verified in the XY hash set (same linear hash: h(d) = h(x_r) ^ h(U_j)).
// Items keep column order per row; the diagonal pair leads its row.
// --------------------------------------------------------------------------
struct BatchArgs {
  const uint64_t* U;
  int64_t n;
  const uint32_t* hx;
  const unsigned long long* xy_table;
  int64_t xy_capmask;
  const unsigned long long* wmask;
  int has_diag;
  int64_t row_begin, row_end;
  int64_t* rp;
  uint32_t* pair_j;
  uint32_t* pair_k;
  int32_t* status;
  unsigned long long* batch_counter;
};

constexpr int kBatchThreads = 512;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kXbufCap = 384;  // expanded candidates verified per round

template <int W>
struct BatchRows {   // per-warp copy of the batch's rows (shared memory)
  uint64_t u[R][W];
  uint32_t hx[R];
  uint32_t cnt[R];
};

// COUNT counts per row (shared atomics); FILL places pairs at per-row ranks in lane order
template <int MODE, int W>
__device__ __forceinline__ void batch_emit(bool found, int r, uint32_t j, uint32_t id, int64_t (&acc)[R],
                                           BatchRows<W>* rc, const BatchArgs& a) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  if (MODE == kFill) {
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const uint32_t m = __ballot_sync(kFull, found && r == rr);
      if (found && r == rr) {
        const int64_t p = acc[rr] + __popc(m & lt);
        a.pair_j[p] = j;
        a.pair_k[p] = id;
      }
      acc[rr] += __popc(m);
    }
    return;
  }
  if (found) atomicAdd(&rc->cnt[r], 1u);
}

template <int W, int MODE>
__device__ __forceinline__ void batch_verify(const uint32_t* items, int n_items, int64_t (&acc)[R],
                                             BatchRows<W>* rc, const BatchArgs& a) {
  const int lane = threadIdx.x & 31;
  for (int e0 = 0; e0 < n_items; e0 += 32) {
    const int e = e0 + lane;
    bool found = false;
    int r = 0;
    uint32_t j = 0, id = 0;
    if (e < n_items) {
      const uint32_t it = items[e];
      r = (int)(it >> 24);
      j = it & 0x00FFFFFFu;
      uint64_t d[W];
#pragma unroll
      for (int w = 0; w < W; ++w) d[w] = rc->u[r][w] ^ __ldg(a.U + (int64_t)j * W + w);
      int64_t slot = (rc->hx[r] ^ __ldg(a.hx + j)) & a.xy_capmask;
      int64_t k = 0;
      for (; k <= a.xy_capmask; ++k) {
        const unsigned long long* sl = a.xy_table + slot * (W + 1);
        const unsigned long long tag = __ldg(sl + W);
        if (tag == ~0ull) break;
        bool eq = true;
#pragma unroll
        for (int w = 0; w < W; ++w) eq = eq && (__ldg(sl + w) == d[w]);
        if (eq) { found = true; id = (uint32_t)tag; break; }
        slot = (slot + 1) & a.xy_capmask;
      }
      if (k > a.xy_capmask) atomicOr(a.status, kStatusLimit);
    }
    batch_emit<MODE, W>(found, r, j, id, acc, rc, a);
  }
}

// expand queue entries (row mask << 24 | column) into (row << 24 | column)
// items, rows of an entry in increasing order, entries in queue order; verify
template <int W, int MODE>
__device__ __forceinline__ void batch_flush(const uint32_t* q, int qn, uint32_t* xbuf, int64_t (&acc)[R],
                                            BatchRows<W>* rc, const BatchArgs& a) {
  const int lane = threadIdx.x & 31;
  int xn = 0;
  for (int s0 = 0; s0 < qn; s0 += 32) {
    if (xn + 32 * R > kXbufCap) {
      __syncwarp();
      batch_verify<W, MODE>(xbuf, xn, acc, rc, a);
      __syncwarp();
      xn = 0;
    }
    const int e = s0 + lane;
    const uint32_t ent = e < qn ? q[e] : 0u;
    uint32_t bits = ent >> 24;
    const uint32_t col = ent & 0x00FFFFFFu;
    const int c = __popc(bits);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    int at = xn + incl - c;
    while (bits) {
      const int b = 31 - __clz(bits);
      bits &= ~(1u << b);
      xbuf[at++] = ((uint32_t)(R - 1 - b) << 24) | col;
    }
    xn += __shfl_sync(kFull, incl, 31);
  }
  __syncwarp();
  batch_verify<W, MODE>(xbuf, xn, acc, rc, a);
  __syncwarp();
}

template <int W, int MODE>
__global__ void __launch_bounds__(kBatchThreads) pairs_batch_kernel(const BatchArgs a) {
  if (MODE == kFill && (*(volatile int32_t*)a.status & kStatusCapacity)) return;  // buffers too small
  __shared__ BatchRows<W> caches[kBatchWarps];
  __shared__ uint32_t queue[kBatchWarps][kQueueCap];
  __shared__ uint32_t xbufs[kBatchWarps][kXbufCap];
  __shared__ unsigned long long wm[5];
  if (threadIdx.x < 5) wm[threadIdx.x] = __ldg(a.wmask + threadIdx.x);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t* q = queue[warp];
  uint32_t* xbuf = xbufs[warp];
  BatchRows<W>* rc = caches + warp;
  const int64_t n_rows = a.row_end - a.row_begin;
  const int64_t n_batches = (n_rows + R - 1) / R;
  const int64_t pbase = (MODE == kFill) ? a.rp[0] : 0;
  while (true) {
    unsigned long long btu = 0;
    if (lane == 0) btu = atomicAdd(a.batch_counter, 1ull);
    const int64_t bt = (int64_t)__shfl_sync(kFull, btu, 0);
    if (bt >= n_batches) break;
    const int64_t r0 = a.row_begin + bt * R;
    __syncwarp();
    if (lane < R) {
      const int64_t row = r0 + lane;
      const bool valid = row < a.row_end;
#pragma unroll
      for (int w = 0; w < W; ++w) rc->u[lane][w] = valid ? __ldg(a.U + row * W + w) : 0ull;
      rc->hx[lane] = valid ? __ldg(a.hx + row) : 0u;
      rc->cnt[lane] = 0u;
    }
    __syncwarp();
    uint64_t xr[R][W];
    uint32_t vmask = 0;
    int64_t acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = r0 + r;
      const bool valid = row < a.row_end;
#pragma unroll
      for (int w = 0; w < W; ++w) xr[r][w] = rc->u[r][w];
      if (valid) vmask |= 1u << (R - 1 - r);
      acc[r] = (MODE == kFill && valid) ? a.rp[row - a.row_begin] - pbase : 0;
    }
    if (a.has_diag) {
      const bool d = lane < R && r0 + lane < a.row_end;
      batch_emit<MODE, W>(d, lane, (uint32_t)(r0 + lane), 0u, acc, rc, a);
    }
    int qn = 0;
    for (int64_t c0 = 0; c0 < a.n; c0 += 32) {
      const int64_t j = c0 + lane;
      const bool vj = j < a.n;
      uint64_t uj[W];
#pragma unroll
      for (int w = 0; w < W; ++w) uj[w] = vj ? __ldg(a.U + j * W + w) : 0ull;
      uint32_t hm = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int wt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) wt += __popcll(xr[r][w] ^ uj[w]);
        const uint32_t t = (uint32_t)(wm[wt >> 6] >> (wt & 63)) & (wt != 0 ? 1u : 0u);
        hm = (hm << 1) | t;
      }
      hm &= vj ? vmask : 0u;
      const uint32_t bal = __ballot_sync(kFull, hm != 0u);
      if (bal) {
        if (hm) q[qn + __popc(bal & lt)] = (hm << 24) | (uint32_t)j;
        qn += __popc(bal);
        if (qn > kQueueCap - 32) {
          __syncwarp();
          batch_flush<W, MODE>(q, qn, xbuf, acc, rc, a);
          __syncwarp();
          qn = 0;
        }
      }
    }
    __syncwarp();
    batch_flush<W, MODE>(q, qn, xbuf, acc, rc, a);
    __syncwarp();
    if (MODE != kFill && lane < R && r0 + lane < a.row_end)
      a.rp[r0 + lane - a.row_begin] = (int64_t)rc->cnt[lane];
  }
}

template <int W, int MODE>
static cudaError_t launch_batch_w(const BatchArgs& args, int64_t rows, cudaStream_t s) {
  auto kern = pairs_batch_kernel<W, MODE>;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBatchThreads, 0);
  if (occ < 1) occ = 1;
  const int64_t batches = (rows + R - 1) / R;
  const int64_t need = (batches + kBatchWarps - 1) / kBatchWarps;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * occ));
  kern<<<blocks, kBatchThreads, 0, s>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_pairs_batch(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, char* stage,
                               const StageHeader& L, int64_t rb, int64_t re, int64_t* rp, uint32_t* pj,
                               uint32_t* pk, int mode, cudaStream_t s) {
  if (n_unq >= (int64_t(1) << 24) || mode == kEmit) return cudaErrorInvalidValue;
  BatchArgs a;
  a.U = U;
  a.n = n_unq;
  a.hx = (const uint32_t*)(stage + L.off_hx);
  a.xy_table = ham->xy_table;
  a.xy_capmask = ham->xy_cap - 1;
  a.wmask = ham->wmask;
  a.has_diag = ham->has_diag;
  a.row_begin = rb;
  a.row_end = re;
  a.rp = rp;
  a.pair_j = pj;
  a.pair_k = pk;
  a.status = (int32_t*)(stage + offsetof(StageHeader, status));
  a.batch_counter = (unsigned long long*)(stage + L.off_counters) + kCtrBatch;
  cudaError_t e = cudaMemsetAsync(a.batch_counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int64_t rows = re - rb;
#define NQS_BATCH(WW)                                                          \
  case WW:                                                                     \
    if (mode == kCount) return launch_batch_w<WW, kCount>(a, rows, s);         \
    return launch_batch_w<WW, kFill>(a, rows, s);
  switch (ham->W) {
    NQS_BATCH(1)
    NQS_BATCH(2)
    NQS_BATCH(3)
    default:
    NQS_BATCH(4)
  }
#undef NQS_BATCH
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
