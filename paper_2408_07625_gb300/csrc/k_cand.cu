// Exact local energy (Eq. local_energy): the candidates x' = x XOR XY of every
// sample x for every unique XY pattern (Sec. "Unique XY": term l couples x to
// x' exactly when x XOR x' = XY^(l), Eq. pauli_melem), their matrix elements,
// the candidates deduplicated over the batch, and
//   E_loc(x) = sum_k H_{x, x XOR XY_k} psi(x XOR XY_k) / psi(x).
// This is the estimator whose O(N_unq N_T) ansatz evaluations the surrogate
// E_loc^var of Sec. "Streamlined local energy calculations" avoids; the
// library produces the candidate set the ansatz must be evaluated on and the
// sum once those amplitudes are known.
//
// Layout: entry e = i * n_xy + k for sample i and pattern k (the library's
// pattern order).  Every sample has exactly n_xy entries, so the per-entry
// outputs are dense [n_unq][n_xy] arrays and need no offsets.
//
// Deduplication (all passes stream over the entries or the table):
//   1. insert: each entry's candidate goes into an open-addressing table of
//      64-bit slots (owner entry << 32 | 32-bit linear hash); the entry's slot
//      index is written to cand_id[e] and its matrix element to hval[e];
//   2. compact: occupied slots -> unsorted unique keys with their slots;
//   3. sort: LSD radix sort of the unique keys in numeric order (qubit 0 the
//      least significant bit) carrying the slot; candidate u = sorted rank;
//   4. assign: slot_uid[slot] = u; cand_in_u[u] = the candidate's index in U
//      (membership table of the staged batch) or -1;
//   5. relabel: cand_id[e] = slot_uid[cand_id[e]].
// The candidate order (numeric) and every entry's index are independent of
// thread timing.
#include <algorithm>
#include <cstring>

#include "device_util.cuh"
#include "melem.cuh"
#include "nqs_internal.cuh"

namespace nqs {

constexpr unsigned long long kEmptySlot = ~0ull;
constexpr int kCandThreads = 256;
constexpr int kCandWarps = kCandThreads / 32;

static inline int64_t a256c(int64_t v) { return (v + 255) & ~int64_t(255); }

static int64_t cand_table_cap(int64_t entries) {
  int64_t c = 1024;
  while (c < 2 * entries) c <<= 1;
  return c;
}

// scratch layout of nqs_full_candidates
struct CandScratch {
  unsigned long long* counters;   // [0] unique candidates, [1] probe limit hit
  unsigned long long* table;      // [cap] slots
  int64_t cap;
  int32_t* slot_uid;              // [cap]
  uint64_t* ukeys;                // [entries][W] unique keys before the sort (sort buffer)
  int32_t* uslot;                 // [entries] their slots (sort payload buffer)
  uint64_t* kb;                   // [entries][W] sort buffer
  int32_t* ib;                    // [entries] sort payload buffer
  int32_t* hist;                  // [256 * sort_blocks(entries)]
  int32_t* partial;               // [sort_scan_partials(entries)]
  int64_t bytes;
};

static CandScratch cand_scratch_view(char* base, int64_t entries, int W) {
  CandScratch v;
  std::memset(&v, 0, sizeof(v));
  const int64_t m = std::max<int64_t>(entries, 1);
  v.cap = cand_table_cap(m);
  int64_t off = 0;
  auto take = [&](int64_t bytes) { char* p = base ? base + off : nullptr; off = a256c(off + bytes); return p; };
  v.counters = (unsigned long long*)take(256);
  v.table = (unsigned long long*)take(8 * v.cap);
  v.slot_uid = (int32_t*)take(4 * v.cap);
  v.ukeys = (uint64_t*)take(8 * W * m);
  v.uslot = (int32_t*)take(4 * m);
  v.kb = (uint64_t*)take(8 * W * m);
  v.ib = (int32_t*)take(4 * m);
  v.hist = (int32_t*)take(4 * 256 * sort_blocks(m));
  v.partial = (int32_t*)take(4 * sort_scan_partials(m));
  v.bytes = off;
  return v;
}

int64_t cand_scratch_bytes(const nqs_ham* ham, int64_t n_unq) {
  return cand_scratch_view(nullptr, n_unq * ham->n_xy, ham->W).bytes;
}

// slot of a 32-bit linear hash: Fibonacci hashing spreads the (structured)
// linear hash over the table
__device__ __forceinline__ uint64_t cand_home(uint32_t h, int lg) {
  return (uint64_t)((h * 0x9E3779B97F4A7C15ull) >> (64 - lg));
}

struct CandArgs {
  const uint64_t* U;
  const uint32_t* hx;          // linear hash of each sample (staged)
  const uint64_t* xy;          // [n_xy][W]
  const uint32_t* xy_hash;     // [n_xy]
  int64_t n_unq, n_xy;
  unsigned long long* table;
  int lg;                      // log2 of the table size
  uint32_t* cand_id;           // [n_unq][n_xy]: slot, later the candidate index
  double* hval;                // [n_unq][n_xy] or null
  unsigned long long* counters;
};

// the candidate of entry e (row e / n_xy, pattern e % n_xy)
template <int W>
__device__ __forceinline__ void entry_key(const CandArgs& a, uint64_t e, uint64_t (&c)[W]) {
  const uint64_t i = e / (uint64_t)a.n_xy, k = e - i * (uint64_t)a.n_xy;
#pragma unroll
  for (int w = 0; w < W; ++w) c[w] = __ldg(a.U + i * W + w) ^ __ldg(a.xy + k * W + w);
}

// Insert key c (hash h) owned by entry e; returns the slot holding it.
template <int W>
__device__ __forceinline__ uint32_t cand_insert(const CandArgs& a, const uint64_t (&c)[W], uint32_t h, uint64_t e) {
  const uint64_t mask = (1ull << a.lg) - 1ull;
  uint64_t s = cand_home(h, a.lg);
  const unsigned long long mine = ((unsigned long long)e << 32) | h;
  for (uint64_t it = 0; it <= mask; ++it) {
    unsigned long long v = a.table[s];
    if (v == kEmptySlot) {
      v = atomicCAS(a.table + s, kEmptySlot, mine);
      if (v == kEmptySlot) return (uint32_t)s;
    }
    if ((uint32_t)v == h) {
      uint64_t o[W];
      entry_key<W>(a, v >> 32, o);
      bool eq = true;
#pragma unroll
      for (int w = 0; w < W; ++w) eq = eq && o[w] == c[w];
      if (eq) return (uint32_t)s;
    }
    s = (s + 1) & mask;
  }
  atomicOr(a.counters + 1, 1ull);  // table full: cannot happen at load <= 1/2
  return 0u;
}

// Work unit of a warp: one sample and a tile of kCandTile consecutive
// patterns (lanes take them in rounds of 32), so that few samples with many
// patterns still fill the GPU.  Matrix elements in FP64 as in the E_loc^var
// kernel (the diagonal by its quadratic form or term loop, heavy term-form
// patterns by the whole warp, the rest one lane each).
constexpr int kCandTile = 1024;

template <int W>
__global__ void __launch_bounds__(kCandThreads) cand_insert_kernel(const CandArgs a, const Melem M) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kCandWarps;
  const int64_t k_first = M.has_diag ? 1 : 0;
  const int64_t tpr = (a.n_xy - k_first + kCandTile - 1) / kCandTile;   // tiles per sample
  const int64_t n_tiles = a.n_unq * (tpr > 0 ? tpr : 1);
  for (int64_t t = blockIdx.x * (int64_t)kCandWarps + (threadIdx.x >> 5); t < n_tiles; t += nw) {
    const int64_t i = tpr > 0 ? t / tpr : t;
    const int64_t tc = tpr > 0 ? t - i * tpr : 0;
    uint64_t x[W];
    load_words<W>(a.U + i * W, x);
    const uint32_t hxi = __ldg(a.hx + i);
    const uint64_t e0 = (uint64_t)i * (uint64_t)a.n_xy;
    if (M.has_diag && tc == 0) {  // pattern 0: x' = x, with the sample's first tile
      const double hd = a.hval ? melem_diag<PolicyD, W>(x, M) : 0.0;
      if (lane == 0) {
        a.cand_id[e0] = cand_insert<W>(a, x, hxi ^ __ldg(a.xy_hash), e0);
        if (a.hval) a.hval[e0] = hd;
      }
    }
    const int64_t k_end = min(a.n_xy, k_first + (tc + 1) * kCandTile);
    for (int64_t kb = k_first + tc * kCandTile; kb < k_end; kb += 32) {
      const int64_t k = kb + lane;
      const bool have = k < k_end;
      uint64_t c[W];
#pragma unroll
      for (int w = 0; w < W; ++w) c[w] = have ? x[w] ^ __ldg(a.xy + k * W + w) : 0ull;
      const int4 fm = have ? __ldg(M.fm + k) : make_int4(0, 0, 0, 0);
      const bool coop = have && k < M.heavy_end && (fm.x & 15) == kForm::Terms;
      double h = 0.0;
      if (a.hval) {
        uint32_t hb = __ballot_sync(kFull, coop);
        while (hb) {
          const int src = __ffs(hb) - 1;
          hb &= hb - 1;
          uint64_t cc[W];
#pragma unroll
          for (int w = 0; w < W; ++w) cc[w] = __shfl_sync(kFull, c[w], src);
          const int64_t kk = __shfl_sync(kFull, k, src);
          const double hw = melem_warp<PolicyD, W>(cc, (int64_t)__ldg(M.t_ptr + kk), (int64_t)__ldg(M.t_ptr + kk + 1), M);
          if (lane == src) h = hw;
        }
        if (have && !coop) h = melem_lane<PolicyD, W>(c, (uint32_t)k, fm, M);
      }
      if (have) {
        const uint64_t e = e0 + (uint64_t)k;
        a.cand_id[e] = cand_insert<W>(a, c, hxi ^ __ldg(a.xy_hash + k), e);
        if (a.hval) a.hval[e] = h;
      }
    }
  }
}

// occupied slots -> unsorted unique keys and their slots.  A block owns a
// chunk of kCompactChunk consecutive slots: it counts them, takes its places
// with one atomic, then writes them in slot order (the chunk is re-read from
// L2).
constexpr int kCompactChunk = 8192;

template <int W>
__global__ void __launch_bounds__(256) cand_compact_kernel(const CandArgs a, uint64_t* __restrict__ ukeys,
                                                           int32_t* __restrict__ uslot) {
  __shared__ uint32_t wcnt[8];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t cap = 1ull << a.lg;
  const uint64_t s0 = (uint64_t)blockIdx.x * kCompactChunk;
  const uint64_t s1 = s0 + kCompactChunk < cap ? s0 + kCompactChunk : cap;
  uint32_t cnt = 0;
  for (uint64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) cnt += a.table[s] != kEmptySlot ? 1u : 0u;
  cnt = __reduce_add_sync(kFull, cnt);
  if (lane == 0) wcnt[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += wcnt[w];
    s_base = t ? atomicAdd(a.counters, (unsigned long long)t) : 0ull;
  }
  __syncthreads();
  unsigned long long run = s_base;
  for (uint64_t t0 = s0; t0 < s1; t0 += blockDim.x) {
    const uint64_t s = t0 + threadIdx.x;
    const unsigned long long v = s < s1 ? a.table[s] : kEmptySlot;
    const bool occ = v != kEmptySlot;
    const uint32_t m = __ballot_sync(kFull, occ);
    __syncthreads();
    if (lane == 0) wcnt[warp] = __popc(m);
    __syncthreads();
    uint32_t off = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
      off += w < warp ? wcnt[w] : 0u;
      total += wcnt[w];
    }
    if (occ) {
      const uint64_t u = run + off + __popc(m & ((1u << lane) - 1u));
      uint64_t c[W];
      entry_key<W>(a, v >> 32, c);
#pragma unroll
      for (int w = 0; w < W; ++w) ukeys[u * W + w] = c[w];
      uslot[u] = (int32_t)s;
    }
    run += total;
  }
}

// sorted rank u -> slot_uid[slot]; membership of the candidate in U
// (the candidate's linear hash, which the staged table of U is keyed by, is
// the tag its slot keeps)
template <int W>
__global__ void cand_assign_kernel(int64_t n_c, const uint64_t* __restrict__ keys, const int32_t* __restrict__ slots,
                                   int32_t* __restrict__ slot_uid, int32_t* __restrict__ in_u,
                                   const unsigned long long* __restrict__ utable, int64_t capmask,
                                   const unsigned long long* __restrict__ ctable, const uint64_t* __restrict__ U,
                                   unsigned long long* counters) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n_c; u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sl = slots[u];
    slot_uid[sl] = (int32_t)u;
    if (!in_u) continue;
    uint64_t c[W];
    const uint32_t h = (uint32_t)ctable[sl];
#pragma unroll
    for (int w = 0; w < W; ++w) c[w] = keys[u * W + w];
    int32_t j = -1;
    int64_t b = h & capmask;
    bool done = false;
    for (int64_t it = 0; it <= capmask && !done; ++it) {
      const uint2* bk = reinterpret_cast<const uint2*>(utable + b * 4);
      for (int q = 0; q < 4; ++q) {
        const uint2 sl = __ldg(bk + q);
        if (sl.y == ~0u) { done = true; break; }
        if (sl.x == h) {
          bool eq = true;
#pragma unroll
          for (int w = 0; w < W; ++w) eq = eq && (__ldg(U + (int64_t)sl.y * W + w) == c[w]);
          if (eq) { j = (int32_t)sl.y; done = true; break; }
        }
      }
      b = (b + 1) & capmask;
    }
    if (!done) atomicOr(counters + 1, 1ull);
    in_u[u] = j;
  }
}

__global__ void cand_relabel_kernel(int64_t entries, uint32_t* __restrict__ cand_id, const int32_t* __restrict__ slot_uid) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < entries; e += (int64_t)gridDim.x * blockDim.x)
    cand_id[e] = (uint32_t)__ldg(slot_uid + cand_id[e]);
}

template <int W>
static cudaError_t cand_w(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage, const StageHeader& L,
                          const CandScratch& sc, uint32_t* cand_id, double* hval, uint64_t* cand, int32_t* in_u,
                          int64_t capacity, int64_t* n_cand, int* limit_hit, cudaStream_t s) {
  const int64_t entries = n * ham->n_xy;
  CandArgs a;
  a.U = U;
  a.hx = (const uint32_t*)(stage + L.off_hx);
  a.xy = ham->xy;
  a.xy_hash = ham->xy_hash;
  a.n_unq = n;
  a.n_xy = ham->n_xy;
  a.table = sc.table;
  a.lg = 0;
  while ((1ll << a.lg) < sc.cap) ++a.lg;
  a.cand_id = cand_id;
  a.hval = hval;
  a.counters = sc.counters;
  cudaError_t e;
  if ((e = cudaMemsetAsync(sc.counters, 0, 256, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(sc.table, 0xFF, 8 * sc.cap, s)) != cudaSuccess) return e;
  const int sms = num_sms();
  const int64_t k_first = ham->has_diag ? 1 : 0;
  const int64_t tiles = n * std::max<int64_t>(1, (ham->n_xy - k_first + kCandTile - 1) / kCandTile);
  const int ins_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + kCandWarps - 1) / kCandWarps, 16 * sms));
  cand_insert_kernel<W><<<ins_blocks, kCandThreads, 0, s>>>(a, melem_tables(ham, n));
  cand_compact_kernel<W><<<(unsigned)((sc.cap + kCompactChunk - 1) / kCompactChunk), 256, 0, s>>>(a, sc.ukeys,
                                                                                                sc.uslot);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  unsigned long long ctr[2] = {0, 0};
  if ((e = cudaMemcpyAsync(ctr, sc.counters, sizeof(ctr), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *n_cand = (int64_t)ctr[0];
  *limit_hit = ctr[1] != 0;
  if (*limit_hit || *n_cand > capacity) return cudaSuccess;
  // numeric sort of the unique keys over their low ceil(N / 8) bytes, carrying the slots
  uint64_t* kbuf[2] = {cand, sc.kb};
  int32_t* ibuf[2] = {sc.ib, sc.uslot};
  // pass 0 reads ukeys/uslot; the payload ping-pong reuses uslot after pass 0
  int out = -1;
  const int n_bytes = (ham->n_qubits + 7) / 8;
  if ((e = launch_sort_words(sc.ukeys, sc.uslot, *n_cand, W, n_bytes, kbuf, ibuf, sc.hist, sc.partial, &out, s)) !=
      cudaSuccess)
    return e;
  const uint64_t* keys = out >= 0 ? kbuf[out] : sc.ukeys;
  const int32_t* slots = out >= 0 ? ibuf[out] : sc.uslot;
  if (keys != cand && *n_cand > 0 &&
      (e = cudaMemcpyAsync(cand, keys, 8 * W * *n_cand, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  const int ub = (int)std::max<int64_t>(1, std::min<int64_t>((*n_cand + 255) / 256, 8 * sms));
  cand_assign_kernel<W><<<ub, 256, 0, s>>>(*n_cand, cand, slots, sc.slot_uid, in_u,
                                           (const unsigned long long*)(stage + L.off_table), L.cap - 1,
                                           sc.table, U, sc.counters);
  const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((entries + 255) / 256, 16 * sms));
  cand_relabel_kernel<<<eb, 256, 0, s>>>(entries, cand_id, sc.slot_uid);
  return cudaGetLastError();
}

cudaError_t launch_full_candidates(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage,
                                   const StageHeader& L, void* scratch, uint32_t* cand_id, double* hval,
                                   uint64_t* cand, int32_t* in_u, int64_t capacity, int64_t* n_cand,
                                   int* limit_hit, cudaStream_t s) {
  const CandScratch sc = cand_scratch_view((char*)scratch, n * ham->n_xy, ham->W);
  switch (ham->W) {
    case 1: return cand_w<1>(ham, U, n, stage, L, sc, cand_id, hval, cand, in_u, capacity, n_cand, limit_hit, s);
    case 2: return cand_w<2>(ham, U, n, stage, L, sc, cand_id, hval, cand, in_u, capacity, n_cand, limit_hit, s);
    case 3: return cand_w<3>(ham, U, n, stage, L, sc, cand_id, hval, cand, in_u, capacity, n_cand, limit_hit, s);
    default: return cand_w<4>(ham, U, n, stage, L, sc, cand_id, hval, cand, in_u, capacity, n_cand, limit_hit, s);
  }
}

// --------------------------------------------------------------------------
// E_loc(x) = sum_k H_{x, x_k} psi(x_k) / psi(x) over the candidates x_k.
// psi(x_k) = P_c 2^{K_c} per candidate (FP64 mantissa in [1, 2) and exponent,
// one exp per candidate), 1/psi(x) = Q_x 2^{-K_x} per sample from the batch
// workspace's amplitude records; per entry a complex product and an exact
// power-of-two scaling (a contribution below the FP64 range is zero).  One
// warp per sample, lanes over the patterns, fixed summation order.
// --------------------------------------------------------------------------
__global__ void cand_amp_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                AmpD* __restrict__ P) {
  const double kLn2 = 0.6931471805599453094;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ai = a[i];
    const double k = floor(ai / kLn2);
    const double m = exp(ai - k * kLn2);
    double c = 1.0, s = 0.0;
    if (b) sincos(b[i], &s, &c);
    P[i].v = make_double2(m * c, m * s);
    P[i].k = (int)fmax(fmin(k, 2.0e9), -2.0e9);
  }
}

// one block per sample: thread t takes entries t, t + 256, ...; the warps'
// sums are added in warp order (a fixed reduction order)
template <bool CPLX>
__global__ void __launch_bounds__(kCandThreads) eloc_full_kernel(int64_t n, int64_t n_xy, const uint32_t* __restrict__ cand_id,
                                                                 const double* __restrict__ hval,
                                                                 const AmpD* __restrict__ P, const AmpD* __restrict__ Q,
                                                                 int64_t n_cand, double* __restrict__ er,
                                                                 double* __restrict__ ei, int32_t* __restrict__ status) {
  __shared__ double s_r[kCandWarps], s_i[kCandWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double2 q = __ldg(&Q[i].v);
    const int kq = __ldg(&Q[i].k);
    double sr = 0.0, si = 0.0;
    const uint64_t e0 = (uint64_t)i * (uint64_t)n_xy;
    for (int64_t k = threadIdx.x; k < n_xy; k += kCandThreads) {
      const uint32_t c = __ldg(cand_id + e0 + k);
      const double h = __ldg(hval + e0 + k);
      if ((int64_t)c >= n_cand) { atomicOr(status, kStatusLimit); continue; }
      const double2 p = __ldg(&P[c].v);
      const int ex = __ldg(&P[c].k) - kq;
      if (CPLX) {
        const double rr = p.x * q.x - p.y * q.y, ri = p.x * q.y + p.y * q.x;
        sr += h * scalbn(rr, ex);
        si += h * scalbn(ri, ex);
      } else {
        sr += h * scalbn(p.x * q.x, ex);
      }
    }
    sr = warp_sum(sr);
    if (CPLX) si = warp_sum(si);
    if (lane == 0) {
      s_r[warp] = sr;
      s_i[warp] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0, ti = 0.0;
      for (int w = 0; w < kCandWarps; ++w) {
        tr += s_r[w];
        ti += s_i[w];
      }
      er[i] = tr;
      if (ei) ei[i] = CPLX ? ti : 0.0;
    }
    __syncthreads();
  }
}

cudaError_t launch_local_energy_full(int64_t n, int64_t n_xy, const char* stage, const StageHeader& L,
                                     const double* a, const double* b, const uint32_t* cand_id, const double* hval,
                                     int64_t n_cand, const double* ca, const double* cb, void* scratch,
                                     double* er, double* ei, cudaStream_t s) {
  AmpD* P = (AmpD*)scratch;
  const int sms = num_sms();
  cudaError_t e = launch_amplitudes(a, b, n, NQS_PREC_FP64, (char*)stage, L, s);
  if (e != cudaSuccess) return e;
  if (n_cand > 0)
    cand_amp_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((n_cand + 255) / 256, 8 * sms)), 256, 0, s>>>(
        n_cand, ca, cb, P);
  const int rb = (int)std::max<int64_t>(1, std::min<int64_t>(n, 16 * sms));
  const AmpD* Q = (const AmpD*)(stage + L.off_ampQ);
  int32_t* status = (int32_t*)(stage + offsetof(StageHeader, status));
  if (b || cb)
    eloc_full_kernel<true><<<rb, kCandThreads, 0, s>>>(n, n_xy, cand_id, hval, P, Q, n_cand, er, ei, status);
  else
    eloc_full_kernel<false><<<rb, kCandThreads, 0, s>>>(n, n_xy, cand_id, hval, P, Q, n_cand, er, ei, status);
  return cudaGetLastError();
}

}  // namespace nqs
