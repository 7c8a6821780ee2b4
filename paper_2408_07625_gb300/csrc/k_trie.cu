// Prefix trees of U and of the unique XY patterns (Alg. 3) and the
// FindCoupledPairs schedule that walks them jointly (LoopOverTrie, Alg. 2C).
//
// Levels follow the qubit index: level i holds the prefixes x_0 .. x_{i-1}.
//
// Tree of U.  U is sorted in that lexicographic order (LSD radix sort, one
// byte of qubits per pass).  A node of level i is a maximal run of sorted
// positions sharing the first i qubits and is named by (t, i), t the run's
// first position.  lcp[t] = first qubit where S[t-1] and S[t] differ, so
// position t starts the nodes of levels lcp[t]+1 .. N.  The child of (t, i)
// along S[t]'s own bit is (t, i+1); the other child exists only if the run
// branches at level i, and then starts at the position m with lcp[m] = i.
// Per position a record keeps S[t], the set of levels at which (t, .)
// branches (bit mask) with the start m of each such branch (CSR), the lcp of
// the next position (node (t, i) holds one sample iff lcp[t+1] < i) and the
// sample's index in U.  This replaces the per-level parent/child arrays of
// the paper's GPU construction by one sort and three data-parallel passes.
//
// Tree of XY (static, built on the host in nqs_ham_load): nodes in level
// order, each {child0, child1, single}; single = pattern id when the node's
// subtree holds one pattern (its children are then not stored).
//
// Traversal (Alg. 2C).  A warp owns one sample x.  A node pair (u, p) of
// level i is kept iff both nodes exist; its children pair u's child along
// bit c with p's child along x_i XOR c.  When u holds a single sample j the
// pair (x, U_j) is coupled iff x XOR U_j is a pattern (one lookup in the XY
// hash set); when p holds a single pattern k, iff x XOR XY_k is in U (one
// lookup in the staged table of U).  Either shortcut ends the path early,
// with the same pair set as walking it to level N.  Pending node pairs live
// on a per-warp stack in shared memory; each step pops up to 32 (one per
// lane) and pushes their children in lane order, so a row's pairs come out in
// an order fixed by the row alone.
#include <algorithm>
#include <cstring>
#include <vector>

#include "device_util.cuh"
#include "nqs_internal.cuh"

namespace nqs {

// --------------------------------------------------------------------------
// host: prefix tree of the unique XY patterns
// --------------------------------------------------------------------------
static int first_diff(const uint64_t* a, const uint64_t* b, int W) {
  for (int w = 0; w < W; ++w) {
    const uint64_t d = a[w] ^ b[w];
    if (d) return 64 * w + __builtin_ctzll(d);
  }
  return -1;
}

static inline int bit_at(const uint64_t* v, int q) { return (int)((v[q >> 6] >> (q & 63)) & 1ull); }

void build_xy_trie(const std::vector<uint64_t>& xy, int64_t n_xy, int W, std::vector<int32_t>& nodes) {
  nodes.clear();
  if (n_xy == 0) return;
  std::vector<int64_t> order(n_xy);
  for (int64_t p = 0; p < n_xy; ++p) order[p] = p;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const int q = first_diff(&xy[a * W], &xy[b * W], W);
    return q >= 0 && bit_at(&xy[a * W], q) == 0;
  });
  struct Item { int64_t lo, hi; int level; };
  std::vector<Item> items{{0, n_xy, 0}};   // node id = position in items (level order)
  for (size_t id = 0; id < items.size(); ++id) {
    const Item it = items[id];
    int32_t c[2] = {-1, -1}, single = -1;
    if (it.hi - it.lo == 1) {
      single = (int32_t)order[it.lo];
    } else {  // distinct patterns: the run splits at some level >= it.level, so level < N
      int64_t m = it.lo;
      while (m < it.hi && bit_at(&xy[order[m] * W], it.level) == 0) ++m;
      if (m > it.lo) { c[0] = (int32_t)items.size(); items.push_back({it.lo, m, it.level + 1}); }
      if (m < it.hi) { c[1] = (int32_t)items.size(); items.push_back({m, it.hi, it.level + 1}); }
    }
    nodes.push_back(c[0]);
    nodes.push_back(c[1]);
    nodes.push_back(single);
    nodes.push_back(0);
  }
}

// --------------------------------------------------------------------------
// device: prefix tree of U
// --------------------------------------------------------------------------
template <int W>
struct alignas(16) TrieRec {
  uint64_t key[W];   // S[t]
  uint64_t bm[W];    // bit i set: node (t, i) branches at level i
  int32_t base;      // first entry of t's branch starts in child_m
  int32_t lcpn;      // lcp[t + 1] (-1 for the last position)
  int32_t orig;      // index of S[t] in U
  int32_t pad;
};

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per block

int64_t sort_blocks(int64_t n) { return (std::max<int64_t>(n, 1) + kSortTile - 1) / kSortTile; }

// v[idx] without dynamic indexing of a register array
template <int W>
__device__ __forceinline__ uint64_t word_at(const uint64_t (&v)[W], int idx) {
  uint64_t r = v[0];
#pragma unroll
  for (int w = 1; w < W; ++w) r = idx == w ? v[w] : r;
  return r;
}

// digit g of a key: byte g of the W-word value, either as is (numeric order,
// word W-1 most significant) or bit-reversed (qubit order: qubit 8g is the
// digit's most significant bit)
template <int W, bool QORDER>
__device__ __forceinline__ uint32_t sort_digit(const uint64_t (&v)[W], int g) {
  const uint32_t byte = (uint32_t)(word_at<W>(v, g >> 3) >> ((g & 7) * 8)) & 0xFFu;
  return QORDER ? __brev(byte) >> 24 : byte;
}

template <int W, bool QORDER>
__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                                                 int g, int32_t* __restrict__ hist, int nblk) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t e = t0 + k * kSortThreads + threadIdx.x;
    if (e < n) {
      uint64_t v[W];
      load_words<W>(keys + e * W, v);
      atomicAdd(&h[sort_digit<W, QORDER>(v, g)], 1);
    }
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of m ints in place (one block)
__global__ void __launch_bounds__(1024) sort_scan_kernel(int32_t* __restrict__ d, int64_t m) {
  __shared__ int32_t part[1024];
  const int64_t per = (m + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = std::min<int64_t>(b + per, m);
  int32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += d[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int32_t run = part[threadIdx.x] - s;
  for (int64_t i = b; i < e; ++i) {
    const int32_t v = d[i];
    d[i] = run;
    run += v;
  }
}

// Exclusive scan of a long int32 array by many blocks: each block scans a
// tile of kScanTileI keys (warp scans, then the warps' totals), one thread
// turns the tile totals into offsets, and every block adds its offset.
constexpr int kScanTileI = 2048;

__global__ void __launch_bounds__(1024) scan_tile_i32_kernel(int32_t* __restrict__ d, int64_t m,
                                                             int32_t* __restrict__ tile_sum) {
  __shared__ int32_t wsum[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTileI;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e0 = base + 2 * threadIdx.x;
  const int32_t v0 = e0 < m ? d[e0] : 0, v1 = e0 + 1 < m ? d[e0 + 1] : 0;
  const int32_t t = v0 + v1;
  int32_t incl = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int32_t w = wsum[lane];
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t x = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += x;
    }
    wsum[lane] = wi - w;
    if (lane == 31) tile_sum[blockIdx.x] = wi;
  }
  __syncthreads();
  const int32_t ex = wsum[warp] + incl - t;
  if (e0 < m) d[e0] = ex;
  if (e0 + 1 < m) d[e0 + 1] = ex + v0;
}

// exclusive scan of the tile totals, one block of 1024 threads: each thread sums a
// contiguous run of tiles, the runs' totals are scanned across the block, each thread
// writes its run's offsets
__global__ void __launch_bounds__(1024) scan_tile_offsets_kernel(int32_t* __restrict__ tile_sum, int64_t tiles) {
  __shared__ int32_t wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t per = (tiles + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = b + per < tiles ? b + per : tiles;
  int32_t s = 0;
  for (int64_t t = b; t < e; ++t) s += tile_sum[t];
  int32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int32_t w = wsum[lane];
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t x = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += x;
    }
    wsum[lane] = wi - w;
  }
  __syncthreads();
  int32_t run = wsum[warp] + incl - s;
  for (int64_t t = b; t < e; ++t) {
    const int32_t v = tile_sum[t];
    tile_sum[t] = run;
    run += v;
  }
}

__global__ void scan_tile_add_kernel(int32_t* __restrict__ d, int64_t m, const int32_t* __restrict__ tile_sum) {
  const int64_t e = (int64_t)blockIdx.x * kScanTileI + threadIdx.x;
  const int32_t off = tile_sum[blockIdx.x];
  if (e < m) d[e] += off;
  if (e + 1024 < m && threadIdx.x + 1024 < kScanTileI) d[e + 1024] += off;
}

// exclusive scan of m ints: one block when small, tiles (partial: ceil(m / 2048) ints) when large
static void scan_i32(int32_t* d, int64_t m, int32_t* partial, cudaStream_t s) {
  if (!partial || m <= (int64_t)1 << 18) {
    sort_scan_kernel<<<1, 1024, 0, s>>>(d, m);
    return;
  }
  const int64_t tiles = (m + kScanTileI - 1) / kScanTileI;
  scan_tile_i32_kernel<<<(unsigned)tiles, 1024, 0, s>>>(d, m, partial);
  scan_tile_offsets_kernel<<<1, 1024, 0, s>>>(partial, tiles);
  scan_tile_add_kernel<<<(unsigned)tiles, 1024, 0, s>>>(d, m, partial);
}

int64_t sort_scan_partials(int64_t n) { return 256 * sort_blocks(n) / kScanTileI + 1; }

cudaError_t launch_scan_i32(int32_t* d, int64_t m, int32_t* partial, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  scan_i32(d, m, partial, s);
  return cudaGetLastError();
}

// Stable scatter: warp w of a block owns keys [t0 + 256 w, t0 + 256 w + 256),
// visited in rounds of 32; equal digits are ranked by (round, lane).  The
// block's keys are first placed in shared memory in digit order (the block's
// own stable sort by this digit), then written out in that order, so that
// consecutive threads write consecutive positions of each digit's run and
// the global stores coalesce.  Dynamic shared memory: sort_scatter_smem(W).
template <int W>
constexpr size_t sort_scatter_smem() {
  return (size_t)kSortTile * (8 * W + 4 + 4);
}

template <int W, bool QORDER>
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const uint64_t* __restrict__ kin,
                                                                    const int32_t* __restrict__ iin, int64_t n, int g,
                                                                    const int32_t* __restrict__ hist, int nblk,
                                                                    uint64_t* __restrict__ kout,
                                                                    int32_t* __restrict__ iout) {
  __shared__ int32_t wcnt[kSortThreads / 32][256];
  __shared__ int32_t dstart[256];   // block-local start of each digit's run
  __shared__ int32_t gbase[256];    // global start of this block's run of each digit
  __shared__ int32_t wtot[kSortThreads / 32];
  extern __shared__ __align__(16) unsigned char sort_smem[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(sort_smem);                 // [kSortTile][W]
  int32_t* si = reinterpret_cast<int32_t*>(sk + (size_t)kSortTile * W);  // [kSortTile]
  int32_t* sd = si + kSortTile;                                          // [kSortTile] digits
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (int d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
  __syncwarp();
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
  const int64_t w0 = t0 + warp * (32 * kSortItems);
  uint32_t dig[kSortItems];
  int32_t rank[kSortItems];
  uint64_t key[kSortItems][W];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t e = w0 + k * 32 + lane;
    const bool live = e < n;
    uint32_t d = 256u + lane;  // never matches a live digit
    if (live) {
      load_words<W>(kin + e * W, key[k]);
      d = sort_digit<W, QORDER>(key[k], g);
    }
    const uint32_t peers = __match_any_sync(kFull, d);
    const int32_t prior = live ? wcnt[warp][d] : 0;
    __syncwarp();
    if (live && (peers & lt) == 0u) wcnt[warp][d] = prior + __popc(peers);
    __syncwarp();
    dig[k] = d;
    rank[k] = prior + __popc(peers & lt);
  }
  __syncthreads();
  {  // thread d: offsets of each warp within the block's run of digit d, then the runs' starts
    const int d = threadIdx.x;
    int32_t run = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) {
      const int32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
    gbase[d] = hist[(int64_t)d * nblk + blockIdx.x];
    int32_t incl = run;  // exclusive scan of the run lengths over digits (block scan)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t x = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += x;
    }
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    int32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wtot[w];
    dstart[d] = before + incl - run;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t e = w0 + k * 32 + lane;
    if (e < n) {
      const int32_t p = dstart[dig[k]] + wcnt[warp][dig[k]] + rank[k];
#pragma unroll
      for (int w = 0; w < W; ++w) sk[(size_t)p * W + w] = key[k][w];
      si[p] = iin ? __ldg(iin + e) : (int32_t)e;
      sd[p] = (int32_t)dig[k];
    }
  }
  __syncthreads();
  const int live = (int)(n - t0 < kSortTile ? n - t0 : kSortTile);
  for (int p = threadIdx.x; p < live; p += kSortThreads) {
    const int d = sd[p];
    const int64_t dst = (int64_t)gbase[d] + (p - dstart[d]);
#pragma unroll
    for (int w = 0; w < W; ++w) kout[dst * W + w] = sk[(size_t)p * W + w];
    iout[dst] = si[p];
  }
}

template <int W>
__device__ __forceinline__ int first_diff_dev(const uint64_t* __restrict__ a, const uint64_t* __restrict__ b,
                                              int n_qubits) {
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint64_t d = __ldg(a + w) ^ __ldg(b + w);
    if (d) return 64 * w + __ffsll((long long)d) - 1;
  }
  return n_qubits;  // equal samples (reported by staging as duplicates)
}

// records: key, sample index, lcp of the next position; lcp array; cleared masks
template <int W>
__global__ void trie_lcp_kernel(const uint64_t* __restrict__ S, const int32_t* __restrict__ idx, int64_t n,
                                int n_qubits, TrieRec<W>* __restrict__ rec, int32_t* __restrict__ lcp) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    TrieRec<W> r;
#pragma unroll
    for (int w = 0; w < W; ++w) { r.key[w] = __ldg(S + t * W + w); r.bm[w] = 0ull; }
    r.base = 0;
    r.lcpn = t + 1 < n ? first_diff_dev<W>(S + t * W, S + (t + 1) * W, n_qubits) : -1;
    r.orig = __ldg(idx + t);
    r.pad = 0;
    rec[t] = r;
    lcp[t] = t > 0 ? first_diff_dev<W>(S + (t - 1) * W, S + t * W, n_qubits) : -1;
  }
}

template <int W>
__device__ __forceinline__ bool same_prefix(const uint64_t* __restrict__ a, const uint64_t (&b)[W], int i) {
  bool eq = true;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int lo = 64 * w;
    const uint64_t m = i >= lo + 64 ? ~0ull : (i > lo ? ((1ull << (i - lo)) - 1ull) : 0ull);
    eq = eq && (((__ldg(a + w) ^ b[w]) & m) == 0ull);
  }
  return eq;
}

// Position m >= 1 starts the 1-child of the level-lcp[m] node holding m - 1;
// that node starts at the first position sharing m - 1's first lcp[m] qubits.
template <int W>
__global__ void trie_branch_kernel(const uint64_t* __restrict__ S, int64_t n, int n_qubits,
                                   const int32_t* __restrict__ lcp, TrieRec<W>* __restrict__ rec,
                                   int32_t* __restrict__ tpar) {
  for (int64_t m = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
    const int i = lcp[m];
    if (i >= n_qubits) { tpar[m] = -1; continue; }  // duplicate: no branch
    uint64_t target[W];
    load_words<W>(S + (m - 1) * W, target);
    int64_t lo = 0, hi = m - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (same_prefix<W>(S + mid * W, target, i)) hi = mid; else lo = mid + 1;
    }
    tpar[m] = (int32_t)lo;
    atomicOr((unsigned long long*)&rec[lo].bm[i >> 6], 1ull << (i & 63));
  }
}

template <int W>
__global__ void trie_count_kernel(const TrieRec<W>* __restrict__ rec, int64_t n, int64_t* __restrict__ cnt) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += __popcll(rec[t].bm[w]);
    cnt[t + 1] = c;
  }
}

template <int W>
__device__ __forceinline__ int popc_below(const uint64_t (&bm)[W], int i) {
  int c = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int lo = 64 * w;
    const uint64_t m = i >= lo + 64 ? ~0ull : (i > lo ? ((1ull << (i - lo)) - 1ull) : 0ull);
    c += __popcll(bm[w] & m);
  }
  return c;
}

template <int W>
__global__ void trie_child_kernel(TrieRec<W>* __restrict__ rec, int64_t n, const int64_t* __restrict__ cnt,
                                  const int32_t* __restrict__ lcp, const int32_t* __restrict__ tpar,
                                  int32_t* __restrict__ child_m) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
    rec[m].base = (int32_t)cnt[m];
    if (m == 0) continue;
    const int32_t t = tpar[m];
    if (t < 0) continue;
    uint64_t bm[W];
#pragma unroll
    for (int w = 0; w < W; ++w) bm[w] = rec[t].bm[w];
    child_m[cnt[t] + popc_below<W>(bm, lcp[m])] = (int32_t)m;
  }
}

struct TrieView {
  uint64_t* keys[2];
  int32_t* idx[2];
  int32_t* hist;
  char* rec;
  int32_t* child_m;
  int64_t* cnt;
  int32_t* lcp;
  int32_t* tpar;
  int nblk;
};

static TrieView trie_view(char* stage, const StageHeader& L) {
  TrieView v;
  const int64_t n = std::max<int64_t>(L.n_unq, 1);
  v.keys[0] = (uint64_t*)(stage + L.off_trie);
  v.keys[1] = v.keys[0] + n * L.W;
  v.idx[0] = (int32_t*)(v.keys[1] + n * L.W);
  v.idx[1] = v.idx[0] + n;
  v.lcp = v.idx[1] + n;
  v.tpar = v.lcp + n;
  v.child_m = v.tpar + n;
  v.hist = v.child_m + n;
  v.nblk = (int)((n + kSortTile - 1) / kSortTile);
  char* p = (char*)(v.hist + 256 * (int64_t)v.nblk);
  p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
  v.cnt = (int64_t*)p;
  p = (char*)(((uintptr_t)(v.cnt + n + 1) + 255) & ~(uintptr_t)255);
  v.rec = p;
  return v;
}

int64_t trie_bytes(int W, int64_t n) {
  n = std::max<int64_t>(n, 1);
  const int64_t nblk = (n + kSortTile - 1) / kSortTile;
  const int64_t rec = 16 * W + 16;
  return 2 * 8 * W * n + 5 * 4 * n + 4 * 256 * nblk + 256 + 8 * (n + 1) + 256 + rec * n + 256;
}

// the scatter's dynamic shared memory may exceed the default 48 KB (W > 1)
template <int W, bool QORDER>
static cudaError_t scatter_attr() {
  return cudaFuncSetAttribute(sort_scatter_kernel<W, QORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sort_scatter_smem<W>());
}

template <int W>
static cudaError_t trie_build_w(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                                const StageHeader& L, cudaStream_t s) {
  TrieView v = trie_view(stage, L);
  auto* rec = reinterpret_cast<TrieRec<W>*>(v.rec);
  const int G = (ham->n_qubits + 7) / 8;
  const uint64_t* kin = U;
  const int32_t* iin = nullptr;
  int cur = 0;
  cudaError_t e;
  for (int g = G - 1; g >= 0; --g) {  // least significant digit (highest qubits) first
    sort_hist_kernel<W, true><<<v.nblk, kSortThreads, 0, s>>>(kin, n, g, v.hist, v.nblk);
    sort_scan_kernel<<<1, 1024, 0, s>>>(v.hist, 256 * (int64_t)v.nblk);
    if ((e = scatter_attr<W, true>()) != cudaSuccess) return e;
    sort_scatter_kernel<W, true><<<v.nblk, kSortThreads, sort_scatter_smem<W>(), s>>>(kin, iin, n, g, v.hist, v.nblk,
                                                                                    v.keys[cur], v.idx[cur]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kin = v.keys[cur];
    iin = v.idx[cur];
    cur ^= 1;
  }
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * num_sms()));
  trie_lcp_kernel<W><<<blocks, 256, 0, s>>>(kin, iin, n, ham->n_qubits, rec, v.lcp);
  trie_branch_kernel<W><<<blocks, 256, 0, s>>>(kin, n, ham->n_qubits, v.lcp, rec, v.tpar);
  if ((e = cudaMemsetAsync(v.cnt, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
  trie_count_kernel<W><<<blocks, 256, 0, s>>>(rec, n, v.cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_scan(v.cnt + 1, n, stage, L, s)) != cudaSuccess) return e;
  trie_child_kernel<W><<<blocks, 256, 0, s>>>(rec, n, v.cnt, v.lcp, v.tpar, v.child_m);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaMemsetAsync(stage + offsetof(StageHeader, trie_ok), 0xFF, sizeof(int32_t), s);
}

cudaError_t launch_trie_build(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                              const StageHeader& L, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(stage + offsetof(StageHeader, trie_ok), 0xFF, sizeof(int32_t), s);
  switch (ham->W) {
    case 1: return trie_build_w<1>(ham, U, n, stage, L, s);
    case 2: return trie_build_w<2>(ham, U, n, stage, L, s);
    case 3: return trie_build_w<3>(ham, U, n, stage, L, s);
    default: return trie_build_w<4>(ham, U, n, stage, L, s);
  }
}

// --------------------------------------------------------------------------
// LSD radix sort of W-word keys in numeric order (word W-1 most significant),
// with an int32 payload, over the low n_bytes bytes of the keys (the higher
// ones must be zero): one histogram, scan and stable scatter per byte.
// Buffers: kbuf[2] of n*W words, ibuf[2] of n ints, hist of 256 * sort_blocks(n)
// ints.  The result is in kbuf[*out] / ibuf[*out].
// --------------------------------------------------------------------------

template <int W>
static cudaError_t sort_words_w(const uint64_t* kin, const int32_t* iin, int64_t n, int n_bytes, uint64_t* kbuf[2],
                                int32_t* ibuf[2], int32_t* hist, int32_t* partial, int* out, cudaStream_t s) {
  const int nblk = (int)sort_blocks(n);
  int cur = 0;
  for (int g = 0; g < n_bytes; ++g) {
    sort_hist_kernel<W, false><<<nblk, kSortThreads, 0, s>>>(kin, n, g, hist, nblk);
    scan_i32(hist, 256 * (int64_t)nblk, partial, s);
    cudaError_t e = scatter_attr<W, false>();
    if (e != cudaSuccess) return e;
    sort_scatter_kernel<W, false><<<nblk, kSortThreads, sort_scatter_smem<W>(), s>>>(kin, iin, n, g, hist, nblk,
                                                                                   kbuf[cur], ibuf[cur]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kin = kbuf[cur];
    iin = ibuf[cur];
    *out = cur;
    cur ^= 1;
  }
  return cudaSuccess;
}

cudaError_t launch_sort_words(const uint64_t* kin, const int32_t* iin, int64_t n, int W, int n_bytes,
                              uint64_t* kbuf[2], int32_t* ibuf[2], int32_t* hist, int32_t* partial, int* out,
                              cudaStream_t s) {
  *out = -1;
  if (n == 0 || n_bytes == 0) return cudaSuccess;
  switch (W) {
    case 1: return sort_words_w<1>(kin, iin, n, n_bytes, kbuf, ibuf, hist, partial, out, s);
    case 2: return sort_words_w<2>(kin, iin, n, n_bytes, kbuf, ibuf, hist, partial, out, s);
    case 3: return sort_words_w<3>(kin, iin, n, n_bytes, kbuf, ibuf, hist, partial, out, s);
    default: return sort_words_w<4>(kin, iin, n, n_bytes, kbuf, ibuf, hist, partial, out, s);
  }
}

// --------------------------------------------------------------------------
// LoopOverTrie search
// --------------------------------------------------------------------------
constexpr int kTrieThreads = 256;
constexpr int kTrieWarps = kTrieThreads / 32;
constexpr int kTrieStack = 1024;   // node pairs per warp (8 KB)

struct TrieArgs {
  const uint64_t* U;
  int64_t n;
  int n_qubits;
  const uint32_t* hx;
  const unsigned long long* table;   // staged table of U (buckets of 4 (tag, index) slots)
  int64_t capmask;
  const char* rec;
  const int32_t* child_m;
  const int4* xnode;
  int64_t n_xnodes;
  const uint64_t* xy;
  const uint32_t* xy_hash;
  const unsigned long long* xy_table;
  int64_t xy_capmask;
  int has_diag;
  int64_t row_begin, row_end;
  int64_t* rp;
  uint32_t* pair_j;
  uint32_t* pair_k;
  int32_t* status;
  const int32_t* trie_ok;
  unsigned long long* row_counter;
  int pop;                           // node pairs popped per step (<= 32)
};

// entry: t (23 bits) | level (9 bits) << 23 | XY node << 32
__device__ __forceinline__ uint64_t pack_entry(int64_t t, int i, int64_t p) {
  return (uint64_t)t | ((uint64_t)i << 23) | ((uint64_t)p << 32);
}

template <int W>
__device__ __forceinline__ bool xy_lookup(const uint64_t (&c)[W], uint32_t h, const TrieArgs& a, uint32_t& id) {
  int64_t slot = h & a.xy_capmask;
  for (int64_t it = 0; it <= a.xy_capmask; ++it) {
    const unsigned long long* sl = a.xy_table + slot * (W + 1);
    const unsigned long long tag = __ldg(sl + W);
    if (tag == ~0ull) return false;
    bool eq = true;
#pragma unroll
    for (int w = 0; w < W; ++w) eq = eq && (__ldg(sl + w) == c[w]);
    if (eq) { id = (uint32_t)tag; return true; }
    slot = (slot + 1) & a.xy_capmask;
  }
  atomicOr(a.status, kStatusLimit);
  return false;
}

template <int W>
__device__ __forceinline__ bool u_lookup(const uint64_t (&c)[W], uint32_t h, const TrieArgs& a, uint32_t& j) {
  int64_t b = h & a.capmask;
  for (int64_t it = 0; it <= a.capmask; ++it) {
    const uint2* bk = reinterpret_cast<const uint2*>(a.table + b * 4);
    for (int k = 0; k < 4; ++k) {
      const uint2 sl = __ldg(bk + k);
      if (sl.y == ~0u) return false;  // an empty slot ends the chain
      if (sl.x == h) {
        bool eq = true;
#pragma unroll
        for (int w = 0; w < W; ++w) eq = eq && (__ldg(a.U + (int64_t)sl.y * W + w) == c[w]);
        if (eq) { j = sl.y; return true; }
      }
    }
    b = (b + 1) & a.capmask;
  }
  atomicOr(a.status, kStatusLimit);
  return false;
}

template <int W, int MODE>
__global__ void __launch_bounds__(kTrieThreads) pairs_trie_kernel(const TrieArgs a) {
  if (*(volatile const int32_t*)a.trie_ok == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, kStatusNoTrie);
    return;
  }
  if (MODE == kFill && (*(volatile int32_t*)a.status & kStatusCapacity)) return;
  extern __shared__ __align__(16) uint64_t trie_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t* st = trie_smem + (int64_t)warp * kTrieStack;
  const TrieRec<W>* rec = reinterpret_cast<const TrieRec<W>*>(a.rec);
  const int n_rows = (int)(a.row_end - a.row_begin);
  const int64_t pbase = MODE == kFill ? a.rp[0] : 0;
  // deepest stack the step rule allows: below cap - N - 34 a step adds <= pop <= 32,
  // above it a single pop adds at most one entry per level still to descend
  const int dfs_from = kTrieStack - a.n_qubits - 34;
  while (true) {
    unsigned long long ru = 0;
    if (lane == 0) ru = atomicAdd(a.row_counter, 1ull);
    const int64_t rr = (int64_t)__shfl_sync(kFull, ru, 0);
    if (rr >= n_rows) break;
    const int64_t row = a.row_begin + rr;
    uint64_t x[W];
    load_words<W>(a.U + row * W, x);
    const uint32_t hxr = __ldg(a.hx + row);
    int64_t acc = MODE == kFill ? a.rp[rr] - pbase : 0;
    if (a.has_diag) {  // the diagonal pair comes first in every row
      if (MODE == kFill && lane == 0) { a.pair_j[acc] = (uint32_t)row; a.pair_k[acc] = 0u; }
      ++acc;
    }
    int sc = 0;
    if (a.n_xnodes > 0) {
      if (lane == 0) st[0] = pack_entry(0, 0, 0);
      sc = 1;
    }
    __syncwarp();
    bool ok = true;
    while (sc > 0) {
      const int k = (sc <= dfs_from) ? min(a.pop, sc) : 1;
      const bool act = lane < k;
      const uint64_t ent = act ? st[sc - k + lane] : 0ull;
      __syncwarp();
      sc -= k;
      bool found = false, pushA = false, pushB = false;
      uint32_t fj = 0, fk = 0;
      uint64_t eA = 0, eB = 0;
      if (act) {
        const int64_t t = (int64_t)(ent & 0x7FFFFFull);
        const int i = (int)((ent >> 23) & 0x1FF);
        const int64_t p = (int64_t)(ent >> 32);
        const TrieRec<W>& r = rec[t];
        uint64_t key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = r.key[w];
        const int lcpn = r.lcpn;
        const int4 xn = __ldg(a.xnode + p);
        if (lcpn < i) {  // u holds one sample: test x XOR S[t] against the patterns
          const uint32_t j = (uint32_t)r.orig;
          uint64_t c[W];
#pragma unroll
          for (int w = 0; w < W; ++w) c[w] = x[w] ^ key[w];
          uint32_t id = 0;
          found = xy_lookup<W>(c, hxr ^ __ldg(a.hx + j), a, id);
          fj = j;
          fk = id;
        } else if (xn.z >= 0) {  // p holds one pattern: test x XOR XY_k for membership in U
          const uint32_t kk = (uint32_t)xn.z;
          uint64_t c[W];
#pragma unroll
          for (int w = 0; w < W; ++w) c[w] = x[w] ^ __ldg(a.xy + (int64_t)kk * W + w);
          uint32_t j = 0;
          found = u_lookup<W>(c, hxr ^ __ldg(a.xy_hash + kk), a, j);
          fj = j;
          fk = kk;
        } else {  // both nodes branch below: expand to level i + 1
          const int b = (int)((word_at<W>(key, i >> 6) >> (i & 63)) & 1ull);
          const int xb = (int)((word_at<W>(x, i >> 6) >> (i & 63)) & 1ull);
          const int cA = (b ^ xb) ? xn.y : xn.x;
          if (cA >= 0) { pushA = true; eA = pack_entry(t, i + 1, cA); }
          uint64_t bm[W];
#pragma unroll
          for (int w = 0; w < W; ++w) bm[w] = r.bm[w];
          if ((word_at<W>(bm, i >> 6) >> (i & 63)) & 1ull) {  // S[t] has bit 0 here; the 1-child starts at m
            const int cB = xb ? xn.x : xn.y;
            if (cB >= 0) {
              const int32_t m = __ldg(a.child_m + r.base + popc_below<W>(bm, i));
              pushB = true;
              eB = pack_entry(m, i + 1, cB);
            }
          }
        }
        if (found && a.has_diag && fk == 0u) found = false;  // already listed first
      }
      const uint32_t bA = __ballot_sync(kFull, pushA), bB = __ballot_sync(kFull, pushB);
      const int total = __popc(bA) + __popc(bB);
      if (sc + total > kTrieStack) {  // unreachable under the step rule; refuse rather than overrun
        if (lane == 0) atomicOr(a.status, kStatusLimit);
        ok = false;
        break;
      }
      const int off = sc + __popc(bA & lt) + __popc(bB & lt);
      if (pushA) st[off] = eA;
      if (pushB) st[off + (pushA ? 1 : 0)] = eB;
      sc += total;
      const uint32_t bf = __ballot_sync(kFull, found);
      if (MODE == kFill && found) {
        const int64_t q = acc + __popc(bf & lt);
        a.pair_j[q] = fj;
        a.pair_k[q] = fk;
      }
      acc += __popc(bf);
      __syncwarp();
    }
    if (MODE == kCount && lane == 0) a.rp[rr] = ok ? acc : 0;
  }
}

template <int W, int MODE>
static cudaError_t launch_trie_w(const TrieArgs& args, int64_t rows, cudaStream_t s) {
  auto kern = pairs_trie_kernel<W, MODE>;
  const size_t smem = (size_t)kTrieWarps * kTrieStack * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTrieThreads, smem);
  if (occ < 1) occ = 1;
  const int64_t need = (rows + kTrieWarps - 1) / kTrieWarps;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * occ));
  kern<<<blocks, kTrieThreads, smem, s>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_pairs_trie(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage,
                              const StageHeader& L, int64_t rb, int64_t re, int64_t* rp, uint32_t* pj,
                              uint32_t* pk, int mode, cudaStream_t s, const SearchTune& tune) {
  if (n >= (int64_t(1) << 23) || ham->n_qubits > 255 || mode == kEmit) return cudaErrorInvalidValue;
  TrieView v = trie_view((char*)stage, L);
  TrieArgs a;
  a.U = U;
  a.n = n;
  a.n_qubits = ham->n_qubits;
  a.hx = (const uint32_t*)(stage + L.off_hx);
  a.table = (const unsigned long long*)(stage + L.off_table);
  a.capmask = L.cap - 1;
  a.rec = v.rec;
  a.child_m = v.child_m;
  a.xnode = ham->xy_trie;
  a.n_xnodes = ham->n_xy_nodes;
  a.xy = ham->xy;
  a.xy_hash = ham->xy_hash;
  a.xy_table = ham->xy_table;
  a.xy_capmask = ham->xy_cap - 1;
  a.has_diag = ham->has_diag;
  a.row_begin = rb;
  a.row_end = re;
  a.rp = rp;
  a.pair_j = pj;
  a.pair_k = pk;
  a.status = (int32_t*)(stage + offsetof(StageHeader, status));
  a.trie_ok = (const int32_t*)(stage + offsetof(StageHeader, trie_ok));
  a.row_counter = (unsigned long long*)(stage + L.off_counters) + kCtrTrie;
  a.pop = std::min(32, std::max(1, tune.trie_pop));
  cudaError_t e = cudaMemsetAsync(a.row_counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int64_t rows = re - rb;
#define NQS_TRIE(WW)                                                          \
  case WW:                                                                    \
    if (mode == kCount) return launch_trie_w<WW, kCount>(a, rows, s);         \
    return launch_trie_w<WW, kFill>(a, rows, s);
  switch (ham->W) {
    NQS_TRIE(1)
    NQS_TRIE(2)
    NQS_TRIE(3)
    default:
    NQS_TRIE(4)
  }
#undef NQS_TRIE
}

}  // namespace nqs
