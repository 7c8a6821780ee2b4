// Sample staging and FindCoupledPairs, LoopOverTerms schedule (Alg. 2A).
//
// Membership test "x' in U" (Alg. 2A): a GF(2)-linear 32-bit hash
// h(v) = XOR_{b in v} R[b] makes the hash of a candidate x' = x XOR XY one XOR
// of two precomputed values, h(x) ^ h(XY).  A blocked Bloom filter of U
// (one 32-bit word per key, two bits set) lives in shared memory and rejects
// most candidates; survivors are verified in a bucketed table of U resident
// in L2: 32-byte buckets of four (hash tag, index) slots, at most one key per
// bucket on average, so a miss reads one sector; only a tag match reads the
// sample itself for the exact comparison.
#include <cstring>

#include "device_util.cuh"
#include "nqs_internal.cuh"

namespace nqs {

// --------------------------------------------------------------------------
// staging: hash of each sample, keyed hash table and Bloom filter of U
// table slot = W key words followed by the sample index (all ones: empty)
// --------------------------------------------------------------------------
template <int W>
__global__ void stage_kernel(const uint64_t* __restrict__ U, int64_t n, int n_qubits,
                             const uint32_t* __restrict__ basis, int64_t cap, uint32_t wmask,
                             uint32_t* __restrict__ hx_out, unsigned long long* __restrict__ table,
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
    const unsigned long long mine = (unsigned long long)h | ((unsigned long long)i << 32);
    int64_t b = h & (cap - 1);
    bool placed = false;
    for (int64_t it = 0; it < cap && !placed; ++it) {
      unsigned long long* bk = table + b * 4;
      for (int k = 0; k < 4; ++k) {
        const unsigned long long prev = atomicCAS(bk + k, ~0ull, mine);
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
    atomicOr(&bloom[(int64_t)(h >> 31) * (wmask + 1) + (h & wmask)], bloom_bits(h));
  }
}

cudaError_t launch_stage(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                         const StageHeader& L, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4 * num_sms());
  auto* hx = (uint32_t*)(stage + L.off_hx);
  auto* table = (unsigned long long*)(stage + L.off_table);
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
// one-pass scratch: linked chunks of pair records per row batch
// --------------------------------------------------------------------------
static inline int64_t a256(int64_t v) { return (v + 255) & ~int64_t(255); }

static inline int64_t nb_max(int64_t rows) { return (rows + kRowsPerWarp - 1) / kRowsPerWarp + 2; }

int64_t pair_scratch_bytes(int64_t rows, int64_t max_pairs) {
  const int64_t nb = nb_max(rows);
  const int64_t chunks = (max_pairs + kChunk - 1) / kChunk + 2 * nb;
  return 256 + a256(16 * nb) + a256(4 * chunks) + 8 * kChunk * chunks;
}

PairScratch pair_scratch_view(void* base, int64_t rows, int64_t bytes) {
  PairScratch sc;
  const int64_t nb = nb_max(rows);
  char* p = (char*)base;
  sc.cursor = (int64_t*)p;
  sc.heads = (int32_t*)(p + 256);
  int64_t rest = bytes - 256 - a256(16 * nb);
  int64_t chunks = rest / (4 + 8 * kChunk);
  while (chunks > 0 && a256(4 * chunks) + 8 * kChunk * chunks > rest) --chunks;
  sc.max_chunks = std::max<int64_t>(chunks, 0);
  sc.next = (int32_t*)(p + 256 + a256(16 * nb));
  sc.records = (uint64_t*)((char*)sc.next + a256(4 * std::max<int64_t>(sc.max_chunks, 1)));
  return sc;
}

// --------------------------------------------------------------------------
// LoopOverTerms search.  A warp owns a batch of kRowsPerWarp rows (taken from
// a global counter) and streams the search table: lane t takes slot 32g + t.
// The 32 slots of a group have distinct low hash bits, so the 32 Bloom-word
// loads of one row hit 32 distinct shared-memory banks.  Per slot a lane keeps
// a bit mask of the rows whose filter test passed; groups with a hit append
// one (row, slot) entry per passed test to a per-warp queue (warp prefix sum),
// so a row's candidates stay in slot order whatever the other rows of its
// batch do.  A full queue is verified lane-parallel against the hash table.
// --------------------------------------------------------------------------
constexpr int kSearchThreads = 1024;
constexpr int kSearchWarps = kSearchThreads / 32;
constexpr int R = kRowsPerWarp;

struct SearchArgs {
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
  int64_t n_groups;
  int has_diag;
  int64_t row_begin, row_end;
  int64_t* rp;
  uint32_t* pair_j;
  uint32_t* pair_k;
  int32_t* status;
  unsigned long long* batch_counter;
  PairScratch sc;
  // two-pass filtering: rows of each class (top hash bit) in perm, pass index
  int pass;
  const int32_t* perm;
  int64_t perm_stride;
  const unsigned long long* cls_cnt;
  int64_t g_begin[2], g_end[2];
  int64_t* rowcur;
  int64_t nbm;
};

struct EmitState {  // warp-uniform chunk state of the one-pass mode
  int32_t chunk, fill, first, total;
};

template <int W>
struct RowCache {   // per-warp copy of the batch's rows (shared memory)
  uint64_t u[R][W];
  uint32_t hx[R];
  uint32_t cnt[R];
  int64_t row[R];
};

// Emit one round of verified candidates (lane order).  COUNT/EMIT count per
// row with shared-memory atomics; FILL places pairs at per-row ranks; EMIT
// appends records to the warp's current scratch chunk.
template <int MODE, int W>
__device__ __forceinline__ void emit_round(bool found, int r, uint32_t j, uint32_t id,
                                           int64_t (&acc)[R], EmitState& es, RowCache<W>* rc,
                                           const SearchArgs& a) {
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
  if (MODE == kEmit) {
    const uint32_t m = __ballot_sync(kFull, found);
    const int n = __popc(m);
    if (n == 0 || es.chunk == -2) return;
    es.total += n;
    const int off = __popc(m & lt);
    const uint64_t rec = (uint64_t)j | ((uint64_t)id << 32) | ((uint64_t)r << 61);
    const int room = es.chunk >= 0 ? kChunk - es.fill : 0;
    if (n <= room) {
      if (found) a.sc.records[(int64_t)es.chunk * kChunk + es.fill + off] = rec;
      es.fill += n;
      return;
    }
    int32_t fresh = -2;
    if (lane == 0) {
      const unsigned long long c = atomicAdd((unsigned long long*)a.sc.cursor, 1ull);
      if ((int64_t)c < a.sc.max_chunks) {
        fresh = (int32_t)c;
        if (es.chunk >= 0) a.sc.next[es.chunk] = fresh;
      } else {
        atomicOr((unsigned long long*)(a.sc.cursor + 1), 1ull);
      }
    }
    fresh = __shfl_sync(kFull, fresh, 0);
    if (found) {
      if (off < room) a.sc.records[(int64_t)es.chunk * kChunk + es.fill + off] = rec;
      else if (fresh >= 0) a.sc.records[(int64_t)fresh * kChunk + (off - room)] = rec;
    }
    if (fresh >= 0 && es.first < 0) es.first = fresh;
    es.chunk = fresh;
    es.fill = n - room;
  }
}

// Verification of queued candidates: each lane takes several entries at a
// time so their loads overlap (search record, then hash-table slot).
template <int W>
struct FlushWays { static constexpr int value = W == 1 ? 2 : 1; };

template <int W>
__device__ __forceinline__ void load_slot(const unsigned long long* sl, unsigned long long (&v)[W + 1]) {
  if (W == 1) {
    const ulonglong2 t = __ldg(reinterpret_cast<const ulonglong2*>(sl));
    v[0] = t.x;
    v[W] = t.y;
  } else {
#pragma unroll
    for (int w = 0; w <= W; ++w) v[w] = __ldg(sl + w);
  }
}

// Exact membership of x' = x_r XOR XY(pos) in the bucket chain starting at
// bucket b (slow path: full buckets, several equal tags).
template <int W>
__device__ __noinline__ bool verify_slow(int r, uint32_t pos, uint32_t sh, const RowCache<W>* rc,
                                         const SearchArgs& a, uint32_t& j) {
  const uint64_t* rec = a.srch_rec + (int64_t)pos * a.rec_words;
  uint64_t key[W];
#pragma unroll
  for (int w = 0; w < W; ++w) key[w] = rc->u[r][w] ^ __ldg(rec + 1 + w);
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

template <int W, int MODE>
__device__ __forceinline__ void verify_items(const uint32_t* q, int qn, int64_t (&acc)[R],
                                             EmitState& es, RowCache<W>* rc, const SearchArgs& a) {
  constexpr int kFlushWays = FlushWays<W>::value;
  const int lane = threadIdx.x & 31;
  for (int e0 = 0; e0 < qn; e0 += 32 * kFlushWays) {
    int r[kFlushWays];
    uint32_t pos[kFlushWays], s[kFlushWays];
    uint4 b0[kFlushWays], b1[kFlushWays];
    bool live[kFlushWays];
#pragma unroll
    for (int u = 0; u < kFlushWays; ++u) {  // candidate hash, then its bucket
      const int e = e0 + u * 32 + lane;
      live[u] = e < qn;
      const uint32_t ent = q[live[u] ? e : e0];
      r[u] = (int)(ent >> 24);
      pos[u] = ent & 0x00FFFFFFu;
      s[u] = rc->hx[r[u]] ^ __ldg(a.srch_hash + pos[u]);
      const uint4* bk = reinterpret_cast<const uint4*>(a.table + (int64_t)(s[u] & a.capmask) * 4);
      b0[u] = __ldg(bk);
      b1[u] = __ldg(bk + 1);
    }
#pragma unroll
    for (int u = 0; u < kFlushWays; ++u) {
      // tag matches among occupied slots; slots fill in order, so slot 3 occupied = full
      const uint32_t sh = s[u];
      const uint32_t mm = (uint32_t)(b0[u].x == sh && b0[u].y != ~0u) | ((uint32_t)(b0[u].z == sh && b0[u].w != ~0u) << 1) |
                          ((uint32_t)(b1[u].x == sh && b1[u].y != ~0u) << 2) | ((uint32_t)(b1[u].z == sh && b1[u].w != ~0u) << 3);
      const uint32_t jc = (mm & 1u) ? b0[u].y : (mm & 2u) ? b0[u].w : (mm & 4u) ? b1[u].y : b1[u].w;
      const bool full = b1[u].w != ~0u;
      bool found = false;
      uint32_t j = 0, id = kDummy;
      bool slow = false;
      if (live[u] && mm) {  // confirm the first match exactly (almost always the only one)
        const uint64_t* rec = a.srch_rec + (int64_t)pos[u] * a.rec_words;
        id = (uint32_t)(__ldg(rec) >> 32);
        bool eq = true;
#pragma unroll
        for (int w = 0; w < W; ++w)
          eq = eq && ((rc->u[r[u]][w] ^ __ldg(rec + 1 + w)) == __ldg(a.U + (int64_t)jc * W + w));
        found = eq;
        j = jc;
        slow = !eq && ((mm & (mm - 1u)) != 0u || full);
      } else if (live[u] && full) {
        slow = true;
      }
      if (slow) {
        id = (uint32_t)(__ldg(a.srch_rec + (int64_t)pos[u] * a.rec_words) >> 32);
        found = verify_slow<W>(r[u], pos[u], sh, rc, a, j);
      }
      found = found && id != kDummy;  // padding slots carry XY = 0 and never count
      if (e0 + u * 32 < qn) emit_round<MODE, W>(found, r[u], j, id, acc, es, rc, a);
    }
  }
}

// Queue entries are (row mask << 24 | slot).  Each 32-entry slice is expanded
// into one (row << 24 | slot) item per set bit, rows of an entry in increasing
// order and entries in queue order, so a row's items keep their slot order.
// Items accumulate in xbuf and are verified in full chunks.
constexpr int kXbufCap = 384;

template <int W, int MODE>
__device__ __forceinline__ void flush_queue(const uint32_t* q, int qn, uint32_t* xbuf, int64_t (&acc)[R],
                                            EmitState& es, RowCache<W>* rc, const SearchArgs& a) {
  const int lane = threadIdx.x & 31;
  int xn = 0;
  for (int c0 = 0; c0 < qn; c0 += 32) {
    if (xn + 32 * R > kXbufCap) {
      __syncwarp();
      verify_items<W, MODE>(xbuf, xn, acc, es, rc, a);
      __syncwarp();
      xn = 0;
    }
    const int e = c0 + lane;
    const uint32_t ent = e < qn ? q[e] : 0u;
    uint32_t bits = ent >> 24;
    const uint32_t pos = ent & 0x00FFFFFFu;
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
      xbuf[at++] = ((uint32_t)(R - 1 - b) << 24) | pos;
    }
    xn += __shfl_sync(kFull, incl, 31);
  }
  __syncwarp();
  verify_items<W, MODE>(xbuf, xn, acc, es, rc, a);
  __syncwarp();
}

template <int W, int MODE>
__global__ void __launch_bounds__(kSearchThreads, 1) pairs_terms_kernel(const SearchArgs a) {
  if (MODE == kFill && (*(volatile int32_t*)a.status & kStatusCapacity)) return;  // buffers too small
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* bloom = smem;
  RowCache<W>* caches = reinterpret_cast<RowCache<W>*>(smem + a.nwords);
  uint32_t* queue = reinterpret_cast<uint32_t*>(caches + kSearchWarps);
  uint32_t* xbufs = queue + kSearchWarps * kQueueCap;
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.bloom_g);
    uint4* dst = reinterpret_cast<uint4*>(bloom);
    for (int i = threadIdx.x; i < a.nwords / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  uint32_t* q = queue + warp * kQueueCap;
  uint32_t* xbuf = xbufs + warp * kXbufCap;
  const uint32_t lt = (1u << lane) - 1u;
  RowCache<W>* rc = caches + warp;
  const int64_t cnt0 = (int64_t)a.cls_cnt[0], cnt1 = (int64_t)a.cls_cnt[1];
  const int64_t nb0 = (cnt0 + R - 1) / R;
  const int64_t n_batches = nb0 + (cnt1 + R - 1) / R;
  const uint32_t wmask4 = a.wmask << 2;
  const char* bloom_bytes = reinterpret_cast<const char*>(bloom);
  const int64_t pbase = (MODE == kFill && a.pass == 0) ? a.rp[0] : 0;
  while (true) {
    unsigned long long btu = 0;
    if (lane == 0) btu = atomicAdd(a.batch_counter, 1ull);
    const int64_t bt = (int64_t)__shfl_sync(kFull, btu, 0);
    if (bt >= n_batches) break;
    const int cls = bt < nb0 ? 0 : 1;
    const int64_t b0 = (cls ? bt - nb0 : bt) * R;
    const int64_t ccount = cls ? cnt1 : cnt0;
    const int half = cls ^ a.pass;  // patterns whose top hash bit sends x' to this pass's samples
    __syncwarp();
    if (lane < R) {
      const bool valid = b0 + lane < ccount;
      const int64_t row = valid ? (int64_t)a.perm[cls * a.perm_stride + b0 + lane] : -1;
#pragma unroll
      for (int w = 0; w < W; ++w) rc->u[lane][w] = valid ? __ldg(a.U + row * W + w) : 0ull;
      rc->hx[lane] = valid ? __ldg(a.hx + row) : 0u;
      rc->cnt[lane] = 0u;
      rc->row[lane] = row;
    }
    __syncwarp();
    uint32_t hr4[R], hr17[R], hr22[R];
    uint32_t vmask = 0;
    int64_t acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t row = rc->row[r];
      const bool valid = row >= 0;
      const uint32_t h = rc->hx[r];
      hr4[r] = h << 2;
      hr17[r] = h >> 17;
      hr22[r] = h >> 22;
      if (valid) vmask |= 1u << (R - 1 - r);
      acc[r] = 0;
      if (MODE == kFill && valid)
        acc[r] = a.pass == 0 ? a.rp[row - a.row_begin] - pbase : a.rowcur[row - a.row_begin];
    }
    EmitState es{-1, 0, -1, 0};
    if (a.has_diag && a.pass == 0) {  // the diagonal pair (x, x) comes first in its row
      const int64_t myrow = rc->row[lane < R ? lane : 0];
      const bool d = lane < R && myrow >= 0;
      emit_round<MODE, W>(d, lane, (uint32_t)(d ? myrow : 0), 0u, acc, es, rc, a);
    }
    int qn = 0;
    for (int64_t g = a.g_begin[half]; g < a.g_end[half]; ++g) {
      const uint32_t pos = (uint32_t)(g * 32 + lane);
      const uint32_t hk = __ldg(a.srch_hash + pos);
      const uint32_t hk4 = hk << 2, hk17 = hk >> 17, hk22 = hk >> 22;
      uint32_t hm = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(bloom_bytes + ((hr4[r] ^ hk4) & wmask4));
        const uint32_t t = __funnelshift_r(w, w, hr17[r] ^ hk17) & __funnelshift_r(w, w, hr22[r] ^ hk22);
        hm = (hm << 1) | (t & 1u);
      }
      hm &= vmask;
      const uint32_t bal = __ballot_sync(kFull, hm != 0u);
      if (bal) {
        if (hm) q[qn + __popc(bal & lt)] = (hm << 24) | pos;
        qn += __popc(bal);
        if (qn > kQueueCap - 32) {
          __syncwarp();
          flush_queue<W, MODE>(q, qn, xbuf, acc, es, rc, a);
          __syncwarp();
          qn = 0;
        }
      }
    }
    __syncwarp();
    flush_queue<W, MODE>(q, qn, xbuf, acc, es, rc, a);
    __syncwarp();
    if (MODE != kFill && lane < R && rc->row[lane] >= 0) {
      const int64_t rl = rc->row[lane] - a.row_begin;
      if (a.pass == 0) a.rp[rl] = (int64_t)rc->cnt[lane];
      else a.rp[rl] += (int64_t)rc->cnt[lane];
    }
    if (MODE == kFill && a.pass == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lane == r && rc->row[r] >= 0) a.rowcur[rc->row[r] - a.row_begin] = acc[r];
    }
    if (MODE == kEmit && lane == 0) {
      a.sc.heads[a.pass * a.nbm + bt] = es.first;
      a.sc.heads[(2 + a.pass) * a.nbm + bt] = es.total;
      if (es.chunk >= 0) a.sc.next[es.chunk] = -1;
    }
  }
}

// Split the rows of [row_begin, row_end) by the top bit of their hash.  The
// order inside a class does not matter: a row's pairs come out in the same
// order whatever rows share its batch.
__global__ void partition_rows_kernel(const uint32_t* __restrict__ hx, int64_t rb, int64_t re,
                                      int32_t* __restrict__ perm, int64_t stride,
                                      unsigned long long* __restrict__ cnt) {
  for (int64_t row = rb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < re;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(__ldg(hx + row) >> 31);
    const unsigned long long p = atomicAdd(cnt + c, 1ull);
    perm[c * stride + (int64_t)p] = (int32_t)row;
  }
}

template <int W, int MODE>
static cudaError_t launch_terms_w(const SearchArgs& args, int64_t rows, size_t smem, cudaStream_t s) {
  auto kern = pairs_terms_kernel<W, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kSearchThreads, smem);
  if (occ < 1) occ = 1;
  const int64_t batches = nb_max(rows);
  const int64_t need = (batches + kSearchWarps - 1) / kSearchWarps;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * occ));
  kern<<<blocks, kSearchThreads, smem, s>>>(args);
  return cudaGetLastError();
}

template <int W>
static size_t search_smem(const StageHeader& L) {
  return 4 * (size_t)L.nwords + kSearchWarps * sizeof(RowCache<W>) +
         (size_t)kSearchWarps * (kQueueCap + kXbufCap) * 4;
}

cudaError_t launch_pairs_terms(const nqs_ham* ham, const uint64_t* U, const char* stage,
                               const StageHeader& L, int64_t rb, int64_t re, int64_t* rp,
                               uint32_t* pj, uint32_t* pk, int mode, const PairScratch* sc,
                               cudaStream_t s) {
  if (ham->n_srch >= (int64_t(1) << 24) || ham->n_xy >= (int64_t(1) << 29)) return cudaErrorInvalidValue;
  const int64_t rows = re - rb;
  unsigned long long* counters = (unsigned long long*)(stage + L.off_counters);
  SearchArgs a;
  a.U = U;
  a.hx = (const uint32_t*)(stage + L.off_hx);
  a.table = (const unsigned long long*)(stage + L.off_table);
  a.capmask = L.cap - 1;
  a.wmask = (uint32_t)(L.nwords - 1);
  a.nwords = (int)L.nwords;
  a.srch_hash = ham->srch_hash;
  a.srch_rec = ham->srch_rec;
  a.rec_words = ham->rec_words;
  a.n_groups = ham->n_srch / 32;
  a.has_diag = ham->has_diag;
  a.row_begin = rb;
  a.row_end = re;
  a.rp = rp;
  a.pair_j = pj;
  a.pair_k = pk;
  a.status = (int32_t*)(stage + offsetof(StageHeader, status));
  if (sc) a.sc = *sc; else a.sc = PairScratch{0, nullptr, nullptr, nullptr, nullptr};
  a.perm = (const int32_t*)(stage + L.off_perm);
  a.perm_stride = rows;
  a.cls_cnt = counters + 2;
  for (int t = 0; t < 2; ++t) { a.g_begin[t] = ham->half_begin[t]; a.g_end[t] = ham->half_end[t]; }
  a.rowcur = (int64_t*)(stage + L.off_rowcur);
  a.nbm = nb_max(rows);
  cudaError_t e = cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, 4 * num_sms()));
    partition_rows_kernel<<<blocks, 256, 0, s>>>(a.hx, rb, re, (int32_t*)a.perm, rows, counters + 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (mode == kEmit) {
    e = cudaMemsetAsync(sc->cursor, 0, 2 * sizeof(int64_t), s);
    if (e != cudaSuccess) return e;
  }
  for (int pass = 0; pass < 2; ++pass) {
    a.pass = pass;
    a.bloom_g = (const uint32_t*)(stage + L.off_bloom) + (int64_t)pass * L.nwords;
    a.batch_counter = counters + pass;
#define NQS_TERMS(WW)                                                                    \
  case WW: {                                                                             \
    const size_t smem = search_smem<WW>(L);                                              \
    if (mode == kCount) e = launch_terms_w<WW, kCount>(a, rows, smem, s);                \
    else if (mode == kFill) e = launch_terms_w<WW, kFill>(a, rows, smem, s);             \
    else e = launch_terms_w<WW, kEmit>(a, rows, smem, s);                                \
    break;                                                                               \
  }
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
  return cudaSuccess;
}

// --------------------------------------------------------------------------
// compaction of the one-pass records into CSR order (one warp per row batch)
// --------------------------------------------------------------------------
__global__ void pairs_compact_kernel(PairScratch sc, int64_t rows, const int64_t* __restrict__ rp,
                                     const int32_t* __restrict__ perm, const unsigned long long* __restrict__ cls_cnt,
                                     int64_t rb, int64_t nbm, uint32_t* __restrict__ pair_j,
                                     uint32_t* __restrict__ pair_k, int64_t capacity, int32_t* status) {
  // buffers sized ahead of time (graph replay) may be too small: report, write nothing
  if (rp[rows] - rp[0] > capacity || sc.cursor[1] != 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusCapacity);
    return;
  }
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t cnt0 = (int64_t)cls_cnt[0], cnt1 = (int64_t)cls_cnt[1];
  const int64_t nb0 = (cnt0 + R - 1) / R;
  const int64_t n_batches = nb0 + (cnt1 + R - 1) / R;
  const int64_t tw = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t p0 = rp[0];
  for (int64_t bt = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); bt < n_batches; bt += tw) {
    const int cls = bt < nb0 ? 0 : 1;
    const int64_t b0 = (cls ? bt - nb0 : bt) * R;
    const int64_t ccount = cls ? cnt1 : cnt0;
    int64_t base[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const bool valid = b0 + r < ccount;
      base[r] = valid ? rp[perm[cls * rows + b0 + r] - rb] - p0 : 0;
    }
    for (int pass = 0; pass < 2; ++pass) {  // a row's pass-0 pairs precede its pass-1 pairs
      const int64_t total = sc.heads[(2 + pass) * nbm + bt];
      int64_t consumed = 0;
      int32_t c = sc.heads[pass * nbm + bt];
      while (consumed < total && c >= 0) {
        const int n_here = (int)((total - consumed < kChunk) ? total - consumed : kChunk);
        for (int e0 = 0; e0 < n_here; e0 += 32) {
          const int e = e0 + lane;
          const bool v = e < n_here;
          const uint64_t rec = v ? sc.records[(int64_t)c * kChunk + e] : 0ull;
          const int r = (int)(rec >> 61);
          const uint32_t j = (uint32_t)rec;
          const uint32_t k = (uint32_t)(rec >> 32) & 0x1FFFFFFFu;
#pragma unroll
          for (int rr = 0; rr < R; ++rr) {
            const uint32_t m = __ballot_sync(kFull, v && r == rr);
            if (v && r == rr) {
              const int64_t p = base[rr] + __popc(m & lt);
              pair_j[p] = j;
              pair_k[p] = k;
            }
            base[rr] += __popc(m);
          }
        }
        consumed += n_here;
        c = sc.next[c];
      }
    }
  }
}

cudaError_t launch_pairs_compact(const PairScratch& sc, const char* stage, const StageHeader& L, int64_t rb,
                                 int64_t rows, const int64_t* row_ptr, uint32_t* pair_j, uint32_t* pair_k,
                                 int64_t capacity, cudaStream_t s) {
  const int64_t batches = nb_max(rows);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((batches + 7) / 8, (int64_t)num_sms() * 8));
  pairs_compact_kernel<<<blocks, 256, 0, s>>>(sc, rows, row_ptr, (const int32_t*)(stage + L.off_perm),
                                              (const unsigned long long*)(stage + L.off_counters) + 2, rb,
                                              nb_max(rows), pair_j, pair_k, capacity,
                                              (int32_t*)(stage + offsetof(StageHeader, status)));
  return cudaGetLastError();
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
  PairScratch sc;
  SearchArgs emit;  // pair_j, pair_k, sc for emit_round
};

constexpr int kBatchThreads = 512;
constexpr int kBatchWarps = kBatchThreads / 32;

template <int W, int MODE>
__device__ __forceinline__ void batch_verify(const uint32_t* items, int n_items, int64_t (&acc)[R], EmitState& es,
                                             RowCache<W>* rc, const BatchArgs& a) {
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
    emit_round<MODE, W>(found, r, j, id, acc, es, rc, a.emit);
  }
}

template <int W, int MODE>
__global__ void __launch_bounds__(kBatchThreads) pairs_batch_kernel(const BatchArgs a) {
  if (MODE == kFill && (*(volatile int32_t*)a.status & kStatusCapacity)) return;  // buffers too small
  __shared__ RowCache<W> caches[kBatchWarps];
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
  RowCache<W>* rc = caches + warp;
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
    EmitState es{-1, 0, -1, 0};
    if (a.has_diag) {
      const bool d = lane < R && r0 + lane < a.row_end;
      emit_round<MODE, W>(d, lane, (uint32_t)(r0 + lane), 0u, acc, es, rc, a.emit);
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
          // expand and verify (same order rules as the LoopOverTerms flush)
          int xn = 0;
          for (int s0 = 0; s0 < qn; s0 += 32) {
            if (xn + 32 * R > kXbufCap) {
              __syncwarp();
              batch_verify<W, MODE>(xbuf, xn, acc, es, rc, a);
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
          batch_verify<W, MODE>(xbuf, xn, acc, es, rc, a);
          __syncwarp();
          qn = 0;
        }
      }
    }
    __syncwarp();
    {
      int xn = 0;
      for (int s0 = 0; s0 < qn; s0 += 32) {
        if (xn + 32 * R > kXbufCap) {
          __syncwarp();
          batch_verify<W, MODE>(xbuf, xn, acc, es, rc, a);
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
      batch_verify<W, MODE>(xbuf, xn, acc, es, rc, a);
      __syncwarp();
    }
    if (MODE != kFill && lane < R && r0 + lane < a.row_end)
      a.rp[r0 + lane - a.row_begin] = (int64_t)rc->cnt[lane];
    if (MODE == kEmit && lane == 0) {
      a.sc.heads[bt] = es.first;
      if (es.chunk >= 0) a.sc.next[es.chunk] = -1;
    }
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

cudaError_t launch_pairs_batch(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, const char* stage,
                               const StageHeader& L, int64_t rb, int64_t re, int64_t* rp, uint32_t* pj,
                               uint32_t* pk, int mode, const PairScratch* sc, cudaStream_t s) {
  if (n_unq >= (int64_t(1) << 24)) return cudaErrorInvalidValue;
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
  a.batch_counter = (unsigned long long*)(stage + L.off_counters);
  if (sc) a.sc = *sc; else a.sc = PairScratch{0, nullptr, nullptr, nullptr, nullptr};
  std::memset(&a.emit, 0, sizeof(a.emit));
  a.emit.pair_j = pj;
  a.emit.pair_k = pk;
  a.emit.sc = a.sc;
  cudaError_t e = cudaMemsetAsync(a.batch_counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (mode == kEmit) {
    e = cudaMemsetAsync(sc->cursor, 0, 2 * sizeof(int64_t), s);
    if (e != cudaSuccess) return e;
  }
  const int64_t rows = re - rb;
#define NQS_BATCH(WW)                                                          \
  case WW:                                                                     \
    if (mode == kCount) return launch_batch_w<WW, kCount>(a, rows, s);         \
    if (mode == kFill) return launch_batch_w<WW, kFill>(a, rows, s);           \
    return launch_batch_w<WW, kEmit>(a, rows, s);
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
