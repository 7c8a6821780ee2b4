// One qubit of autoregressive sampling without replacement (Alg. 1,
// ARGumbelTopK, Sec. "Autoregressive sampling without replacement").
//
// Each kept vector x_<i (log-probability l, conditioned perturbed value L~)
// is extended by x_i = 0 and 1: l' = l + log p_i(x_i | x_<i), L' = l' + G,
// Z = max of the two L', L~' = -log(exp(-L~) - exp(-Z) + exp(-L')), evaluated
// as L~' = L~ - softplus(L~ - Z + log(expm1(Z - L'))) for L' < Z and L~' = L~
// for the larger extension (the same value; the printed form cancels exp(-Z)
// against exp(-L') and loses exp(-L~) once Z is far below L~).  The
// extensions are ordered by L~' descending (stable: equal values keep the
// extension order, vector-major, x_i = 0 first) and the first K kept.  An
// extension with l' = -inf (an impossible outcome) is not kept.
//
// Ordering.  The extensions' 64-bit keys order the doubles L~' descending;
// with the extension index they form a total order.  Bucket path (up to
// kBucketMax buckets): one block sorts a strided sample of the keys and takes
// splitters at even ranks of its possible keys; every extension goes to the
// bucket of its key (slots reserved per block with one atomic per bucket);
// one block per bucket sorts its bucket by (key, index) in shared memory
// (bitonic) and writes the children of its ranks below K directly, its offset
// being the sizes of the buckets before it.  Placement inside a bucket
// depends on timing, the sort by the total order removes that.  A bucket
// above kBucketCap (many equal keys) hands the level to the general path: an
// LSD radix sort of all keys carrying the extension index.  The Gumbel draws
// and the conditional log-probabilities are inputs (the ansatz is the
// caller's).
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <math_constants.h>

#include "device_util.cuh"
#include "nqs_internal.cuh"

namespace nqs {

constexpr int kSampleThreads = 256;
constexpr int kBucketCap = 2048;       // extensions a bucket can hold (the sorting block's shared memory)
constexpr int kBucketMax = 1024;       // buckets
constexpr int kBucketAvg = 512;        // extensions per bucket aimed at
constexpr int kSplitSamples = 2048;    // keys sampled for the splitters
constexpr int kSortBlock = 1024;       // threads of the splitter and bucket-sort blocks
constexpr int kScatterThreads = 512;
constexpr int kScatterItems = 4;

// sort key ordering doubles descending (NaN-free input); impossible extensions last
__device__ __forceinline__ uint64_t desc_key(double v) {
  if (v == 0.0) v = 0.0;   // -0 and +0 are one value
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const uint64_t asc = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
  return ~asc;
}

// L~' of the smaller extension (perturbed value L < Z = the larger one's)
__device__ __forceinline__ double conditioned_smaller(double lt, double Z, double L) {
  const double v = (lt - Z) + log(expm1(Z - L));
  return lt - (fmax(v, 0.0) + log1p(exp(-fabs(v))));
}

struct SampleScratch {
  uint64_t* keys[2];
  int32_t* idx[2];
  int32_t* hist;
  int32_t* partial;
  double* ext;                 // [2n][2]: l', L~' of every extension
  unsigned long long* valid;   // possible extensions (general path)
  // bucket path
  uint64_t* spl;               // [kBucketMax]: splitters 1 .. B-1
  unsigned int* cursor;        // [kBucketMax]: extensions placed in each bucket
  int* flag;                   // a bucket overflowed
  long long* result;           // [2]: kept count, 1 if the bucket path completed
  uint64_t* bkey;              // [B][kBucketCap]
  int32_t* bidx;
  int64_t bytes;
};

static inline int64_t a256s(int64_t v) { return (v + 255) & ~int64_t(255); }

// buckets for m extensions (0: the bucket path does not apply)
static int bucket_count(int64_t m) {
  int B = 1;
  while ((int64_t)B * kBucketAvg < m) B <<= 1;
  return B <= kBucketMax ? B : 0;
}

static SampleScratch sample_scratch_view(char* base, int64_t n_parents) {
  SampleScratch v;
  std::memset(&v, 0, sizeof(v));
  const int64_t m = std::max<int64_t>(2 * n_parents, 1);
  int64_t off = 0;
  auto take = [&](int64_t bytes) { char* p = base ? base + off : nullptr; off = a256s(off + bytes); return p; };
  v.valid = (unsigned long long*)take(256);
  v.keys[0] = (uint64_t*)take(8 * m);
  v.keys[1] = (uint64_t*)take(8 * m);
  v.idx[0] = (int32_t*)take(4 * m);
  v.idx[1] = (int32_t*)take(4 * m);
  v.hist = (int32_t*)take(4 * 256 * sort_blocks(m));
  v.partial = (int32_t*)take(4 * sort_scan_partials(m));
  v.ext = (double*)take(16 * m);
  const int B = std::max(bucket_count(m), 1);
  v.spl = (uint64_t*)take(8 * kBucketMax);
  v.cursor = (unsigned int*)take(4 * kBucketMax);
  v.flag = (int*)take(4);
  v.result = (long long*)take(16);
  v.bkey = (uint64_t*)take(8 * (int64_t)B * kBucketCap);
  v.bidx = (int32_t*)take(4 * (int64_t)B * kBucketCap);
  v.bytes = off;
  return v;
}

int64_t sample_scratch_bytes(int64_t n_parents) { return sample_scratch_view(nullptr, n_parents).bytes; }

// one thread per kept vector: both extensions, their sort keys and (l', L~')
__global__ void gumbel_extend_kernel(int64_t n, const long long* __restrict__ n_dev, const double* __restrict__ pl,
                                     const double* __restrict__ plt, const double* __restrict__ logp,
                                     const double* __restrict__ G, uint64_t* __restrict__ keys,
                                     int32_t* __restrict__ idx, double* __restrict__ ext,
                                     unsigned long long* __restrict__ valid) {
  if (n_dev) n = min(n, (int64_t)max(*n_dev, 0ll));   // the device-held count, at most the launch's bound
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double l = pl[p], lt = plt[p];
    const double l0 = l + logp[2 * p], l1 = l + logp[2 * p + 1];
    const double L0 = l0 + G[2 * p], L1 = l1 + G[2 * p + 1];
    const double Z = fmax(L0, L1);
    // the smaller extension is the only one whose L~' needs the logarithms
    // (x = 1 when the two are equal: then both keep L~)
    const int sx = L0 < L1 ? 0 : 1;
    const double Ls = sx ? L1 : L0;
    const double lts = Ls < Z ? conditioned_smaller(lt, Z, Ls) : lt;
    const double lc[2] = {l0, l1};
    int nv = 0;
#pragma unroll
    for (int xi = 0; xi < 2; ++xi) {
      const int64_t c = 2 * p + xi;
      if (idx) idx[c] = (int32_t)c;
      if (lc[xi] == -CUDART_INF) {
        keys[c] = ~0ull;
        ext[2 * c] = -CUDART_INF;
        ext[2 * c + 1] = -CUDART_INF;
        continue;
      }
      const double ltc = xi == sx ? lts : lt;
      keys[c] = desc_key(ltc);
      ext[2 * c] = lc[xi];
      ext[2 * c + 1] = ltc;
      ++nv;
    }
    if (valid && nv) atomicAdd(valid, (unsigned long long)nv);
  }
}

// (key, extension index): the total order of the extensions
__device__ __forceinline__ bool ext_less(uint64_t ka, int32_t ia, uint64_t kb, int32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// One block: a sample of the m keys (evenly spaced positions, the tail
// included), sorted by their upper 32 bits; splitter b (1 <= b < B) = the
// sample at rank b V / B among its V possible keys, its lower 32 bits zero
// (any ascending splitters are correct: they only balance the buckets);
// cursors and flag zeroed.
constexpr int kSplitPer = kSplitSamples / kSortBlock;   // samples per thread

__global__ void __launch_bounds__(kSortBlock) gumbel_splitters_kernel(int64_t m, const long long* __restrict__ n_dev,
                                                                     int B, const uint64_t* __restrict__ keys,
                                                                     uint64_t* __restrict__ spl,
                                                                     unsigned int* __restrict__ cursor,
                                                                     int* __restrict__ flag) {
  __shared__ uint32_t sk[kSplitSamples];
  __shared__ int32_t sp[kSplitSamples];
  __shared__ int s_v;
  const int tid = threadIdx.x;
  if (n_dev) m = min(m, 2 * (int64_t)max(*n_dev, 0ll));
  for (int b = tid; b < kBucketMax; b += kSortBlock) cursor[b] = 0u;
  if (tid == 0) {
    *flag = 0;
    s_v = 0;
  }
  if (B == 1) return;
  uint32_t key[kSplitPer];
  int32_t pay[kSplitPer];
#pragma unroll
  for (int u = 0; u < kSplitPer; ++u) {
    const int i = kSplitPer * tid + u;
    const int64_t q = m > kSplitSamples ? ((int64_t)i * m) / kSplitSamples : i;
    key[u] = q < m ? (uint32_t)(keys[q] >> 32) : 0xFFFFFFFFu;
    pay[u] = 0;
  }
  block_bitonic<kSplitPer, false>(key, pay, kSplitSamples, sk, sp);
  int nv = 0;
#pragma unroll
  for (int u = 0; u < kSplitPer; ++u) {
    sk[kSplitPer * tid + u] = key[u];
    nv += key[u] != 0xFFFFFFFFu;   // the upper half of an impossible extension's key (no double has it)
  }
  atomicAdd(&s_v, nv);
  __syncthreads();
  const int V = s_v;
  for (int b = 1 + tid; b < B; b += kSortBlock)
    spl[b] = V > 0 ? (uint64_t)sk[(int)(((int64_t)b * V) / B)] << 32 : ~0ull;
}

// bucket of a key: the number of splitters <= key (splitters ascend)
__device__ __forceinline__ int bucket_of(uint64_t k, const uint64_t* s_spl, int B) {
  int lo = 1, hi = B;   // first splitter index in [1, B) with spl > k, or B
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s_spl[mid] <= k) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

// every possible extension into its bucket; a block's slots of a bucket are
// reserved with one atomic, the block-local order by shared-memory atomics
__global__ void __launch_bounds__(kScatterThreads) gumbel_bucket_scatter_kernel(
    int64_t m, const long long* __restrict__ n_dev, int B, const uint64_t* __restrict__ keys,
    const uint64_t* __restrict__ spl, unsigned int* __restrict__ cursor, int* __restrict__ flag,
    uint64_t* __restrict__ bkey, int32_t* __restrict__ bidx) {
  __shared__ uint64_t s_spl[kBucketMax];
  __shared__ unsigned int s_cnt[kBucketMax];
  __shared__ unsigned int s_base[kBucketMax];
  const int tid = threadIdx.x;
  if (n_dev) m = min(m, 2 * (int64_t)max(*n_dev, 0ll));
  for (int b = tid; b < kBucketMax; b += kScatterThreads) {
    s_spl[b] = (b >= 1 && b < B) ? spl[b] : ~0ull;
    s_cnt[b] = 0u;
  }
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * (kScatterThreads * kScatterItems);
  uint64_t k[kScatterItems];
  int bk[kScatterItems];
  unsigned int rk[kScatterItems];
#pragma unroll
  for (int u = 0; u < kScatterItems; ++u) {
    const int64_t c = t0 + (int64_t)u * kScatterThreads + tid;
    k[u] = c < m ? keys[c] : ~0ull;
    bk[u] = -1;
    if (k[u] != ~0ull) {
      bk[u] = bucket_of(k[u], s_spl, B);
      rk[u] = atomicAdd(&s_cnt[bk[u]], 1u);
    }
  }
  __syncthreads();
  for (int b = tid; b < B; b += kScatterThreads)
    if (s_cnt[b]) s_base[b] = atomicAdd(&cursor[b], s_cnt[b]);
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kScatterItems; ++u) {
    if (bk[u] < 0) continue;
    const unsigned int slot = s_base[bk[u]] + rk[u];
    if (slot >= (unsigned)kBucketCap) {
      *flag = 1;
      continue;
    }
    const int64_t c = t0 + (int64_t)u * kScatterThreads + tid;
    bkey[(int64_t)bk[u] * kBucketCap + slot] = k[u];
    bidx[(int64_t)bk[u] * kBucketCap + slot] = (int32_t)c;
  }
}

// One block per bucket: sort it by (key, index) in shared memory (bitonic over
// the next power of two), then write the children of its global ranks below K;
// block 0 reports the kept count.  Nothing is written after an overflow.
constexpr int kBucketPer = 8;                            // elements per thread
constexpr int kBucketThreads = kBucketCap / kBucketPer;

template <int W>
__global__ void __launch_bounds__(kBucketThreads) gumbel_bucket_sort_kernel(
    int B, int level, int64_t K, const unsigned int* __restrict__ cursor, const int* __restrict__ flag,
    const uint64_t* __restrict__ bkey, const int32_t* __restrict__ bidx, const uint64_t* __restrict__ px,
    const double* __restrict__ ext, uint64_t* __restrict__ cx, double* __restrict__ cl, double* __restrict__ clt,
    long long* __restrict__ result) {
  __shared__ uint64_t sk[kBucketCap];
  __shared__ int32_t si[kBucketCap];
  __shared__ long long s_red[2][kBucketThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, b = blockIdx.x;
  const bool over = *flag != 0;
  // this bucket's offset (sizes of the buckets before it) and the total
  long long off = 0, tot = 0;
  for (int q = tid; q < B; q += kBucketThreads) {
    const long long v = cursor[q];
    tot += v;
    if (q < b) off += v;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    off += __shfl_xor_sync(0xFFFFFFFFu, off, o);
    tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
  }
  if (lane == 0) {
    s_red[0][warp] = off;
    s_red[1][warp] = tot;
  }
  __syncthreads();
  off = 0;
  tot = 0;
  for (int w = 0; w < kBucketThreads / 32; ++w) {
    off += s_red[0][w];
    tot += s_red[1][w];
  }
  const long long n_out = min((long long)K, tot);
  if (b == 0 && tid == 0) {
    result[0] = over ? 0 : n_out;
    result[1] = over ? 0 : 1;
  }
  if (over || off >= n_out) return;
  const int cnt = (int)cursor[b];
  int size = 2;
  while (size < cnt) size <<= 1;
  uint64_t key[kBucketPer];
  int32_t pay[kBucketPer];
#pragma unroll
  for (int u = 0; u < kBucketPer; ++u) {
    const int i = kBucketPer * tid + u;
    key[u] = i < cnt ? bkey[(int64_t)b * kBucketCap + i] : ~0ull;
    pay[u] = i < cnt ? bidx[(int64_t)b * kBucketCap + i] : 0x7FFFFFFF;
  }
  block_bitonic<kBucketPer, true>(key, pay, size, sk, si);
#pragma unroll
  for (int u = 0; u < kBucketPer; ++u) si[kBucketPer * tid + u] = pay[u];
  __syncthreads();
  for (int i = tid; i < cnt; i += kBucketThreads) {
    const long long r = off + i;
    if (r >= n_out) break;
    const int64_t c = si[i];
    const int64_t p = c >> 1;
    const uint64_t bit = (uint64_t)(c & 1);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint64_t v = px ? px[p * W + w] : 0ull;
      if (w == (level >> 6)) v |= bit << (level & 63);
      cx[r * W + w] = v;
    }
    cl[r] = ext[2 * c];
    clt[r] = ext[2 * c + 1];
  }
}

// the first n_out extensions in sorted order: x_<i with x_i set, l', L~'
template <int W>
__global__ void gumbel_gather_kernel(int64_t n_out, int level, const int32_t* __restrict__ order,
                                     const uint64_t* __restrict__ px, const double* __restrict__ ext,
                                     uint64_t* __restrict__ cx, double* __restrict__ cl, double* __restrict__ clt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_out; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = order[r];
    const int64_t p = c >> 1;
    const uint64_t bit = (uint64_t)(c & 1);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint64_t v = px ? px[p * W + w] : 0ull;
      if (w == (level >> 6)) v |= bit << (level & 63);
      cx[r * W + w] = v;
    }
    cl[r] = ext[2 * c];
    clt[r] = ext[2 * c + 1];
  }
}

template <int W>
static void launch_bucket_sort(int B, int level, int64_t K, const SampleScratch& sc, const uint64_t* px, uint64_t* cx,
                               double* cl, double* clt, long long* result, cudaStream_t s) {
  gumbel_bucket_sort_kernel<W><<<B, kBucketThreads, 0, s>>>(B, level, K, sc.cursor, sc.flag, sc.bkey, sc.bidx, px,
                                                            sc.ext, cx, cl, clt, result);
}

static void launch_bucket_sort_w(int W, int B, int level, int64_t K, const SampleScratch& sc, const uint64_t* px,
                                 uint64_t* cx, double* cl, double* clt, long long* result, cudaStream_t s) {
  switch (W) {
    case 1: launch_bucket_sort<1>(B, level, K, sc, px, cx, cl, clt, result, s); break;
    case 2: launch_bucket_sort<2>(B, level, K, sc, px, cx, cl, clt, result, s); break;
    case 3: launch_bucket_sort<3>(B, level, K, sc, px, cx, cl, clt, result, s); break;
    default: launch_bucket_sort<4>(B, level, K, sc, px, cx, cl, clt, result, s); break;
  }
}

// a small page-locked host buffer per host thread for the per-level count
// (never freed: it lives as long as the thread); nullptr if it cannot be had
static long long* pinned_readback() {
  thread_local long long* p = nullptr;
  thread_local bool tried = false;
  if (!tried) {
    tried = true;
    if (cudaMallocHost((void**)&p, 4 * sizeof(long long)) != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
    }
  }
  return p;
}

// The bucket path; *done = false when a bucket overflowed (the general path follows).
static cudaError_t gumbel_level_buckets(int W, int level, int64_t n, const uint64_t* px, int64_t K,
                                        const SampleScratch& sc, uint64_t* cx, double* cl, double* clt,
                                        int64_t* n_out, bool* done, cudaStream_t s) {
  *done = false;
  const int64_t m = 2 * n;
  const int B = bucket_count(m);
  gumbel_splitters_kernel<<<1, kSortBlock, 0, s>>>(m, nullptr, B, sc.keys[0], sc.spl, sc.cursor, sc.flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t per = (int64_t)kScatterThreads * kScatterItems;
  gumbel_bucket_scatter_kernel<<<(unsigned)((m + per - 1) / per), kScatterThreads, 0, s>>>(
      m, nullptr, B, sc.keys[0], sc.spl, sc.cursor, sc.flag, sc.bkey, sc.bidx);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  launch_bucket_sort_w(W, B, level, K, sc, px, cx, cl, clt, sc.result, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  long long local[2] = {0, 0};
  long long* res = pinned_readback();   // page-locked: the copy goes straight to it
  if (!res) res = local;
  res[0] = res[1] = 0;
  if ((e = cudaMemcpyAsync(res, sc.result, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if (res[1] == 1) {
    *n_out = res[0];
    *done = true;
  }
  return cudaSuccess;
}

cudaError_t launch_gumbel_level(int W, int level, int64_t n, const uint64_t* px, const double* pl, const double* plt,
                                const double* logp, const double* G, int64_t K, void* scratch, uint64_t* cx,
                                double* cl, double* clt, int64_t* n_out, cudaStream_t s) {
  SampleScratch sc = sample_scratch_view((char*)scratch, n);
  const int64_t m = 2 * n;
  const int sms = num_sms();
  const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((n + kSampleThreads - 1) / kSampleThreads, 8 * sms));
  cudaError_t e;
  if (bucket_count(m) > 0) {
    gumbel_extend_kernel<<<eb, kSampleThreads, 0, s>>>(n, nullptr, pl, plt, logp, G, sc.keys[0], nullptr, sc.ext,
                                                       nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bool done = false;
    if ((e = gumbel_level_buckets(W, level, n, px, K, sc, cx, cl, clt, n_out, &done, s)) != cudaSuccess || done)
      return e;
  }
  // general path: an LSD radix sort of all keys with the extension index
  if ((e = cudaMemsetAsync(sc.valid, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  gumbel_extend_kernel<<<eb, kSampleThreads, 0, s>>>(n, nullptr, pl, plt, logp, G, sc.keys[0], sc.idx[0], sc.ext,
                                                     sc.valid);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // stable descending order by L~' over all 8 key bytes
  uint64_t* kbuf[2] = {sc.keys[1], sc.keys[0]};
  int32_t* ibuf[2] = {sc.idx[1], sc.idx[0]};
  int out = -1;
  if ((e = launch_sort_words(sc.keys[0], sc.idx[0], m, 1, 8, kbuf, ibuf, sc.hist, sc.partial, &out, s)) !=
      cudaSuccess)
    return e;
  const int32_t* order = out >= 0 ? ibuf[out] : sc.idx[0];
  unsigned long long nv = 0;
  if ((e = cudaMemcpyAsync(&nv, sc.valid, sizeof(nv), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *n_out = std::min<int64_t>((int64_t)nv, K);
  if (*n_out == 0) return cudaSuccess;
  const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((*n_out + 255) / 256, 8 * sms));
  switch (W) {
    case 1: gumbel_gather_kernel<1><<<gb, 256, 0, s>>>(*n_out, level, order, px, sc.ext, cx, cl, clt); break;
    case 2: gumbel_gather_kernel<2><<<gb, 256, 0, s>>>(*n_out, level, order, px, sc.ext, cx, cl, clt); break;
    case 3: gumbel_gather_kernel<3><<<gb, 256, 0, s>>>(*n_out, level, order, px, sc.ext, cx, cl, clt); break;
    default: gumbel_gather_kernel<4><<<gb, 256, 0, s>>>(*n_out, level, order, px, sc.ext, cx, cl, clt); break;
  }
  return cudaGetLastError();
}

// The device-count form: the parent count is read from n_dev (at most
// max_n, which sizes the launches) and the kept count and status are written
// to counts[0], counts[1] on the device; no host synchronisation, so a run of
// levels (and the caller's work between them) can be enqueued or captured in
// a graph.  The bucket path only: status 0 marks a level whose buckets
// overflowed (nothing kept; later levels then start from no parents).
cudaError_t launch_gumbel_level_async(int W, int level, int64_t max_n, const long long* n_dev, const uint64_t* px,
                                      const double* pl, const double* plt, const double* logp, const double* G,
                                      int64_t K, void* scratch, uint64_t* cx, double* cl, double* clt,
                                      long long* counts, cudaStream_t s) {
  SampleScratch sc = sample_scratch_view((char*)scratch, max_n);
  const int64_t m = 2 * max_n;
  const int B = bucket_count(m);
  if (B == 0) return cudaErrorInvalidValue;
  const int sms = num_sms();
  const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((max_n + kSampleThreads - 1) / kSampleThreads, 8 * sms));
  gumbel_extend_kernel<<<eb, kSampleThreads, 0, s>>>(max_n, n_dev, pl, plt, logp, G, sc.keys[0], nullptr, sc.ext,
                                                     nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gumbel_splitters_kernel<<<1, kSortBlock, 0, s>>>(m, n_dev, B, sc.keys[0], sc.spl, sc.cursor, sc.flag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t per = (int64_t)kScatterThreads * kScatterItems;
  gumbel_bucket_scatter_kernel<<<(unsigned)((m + per - 1) / per), kScatterThreads, 0, s>>>(
      m, n_dev, B, sc.keys[0], sc.spl, sc.cursor, sc.flag, sc.bkey, sc.bidx);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  launch_bucket_sort_w(W, B, level, K, sc, px, cx, cl, clt, counts, s);
  return cudaGetLastError();
}

int64_t sample_async_limit() { return (int64_t)kBucketMax * kBucketAvg / 2; }

}  // namespace nqs
