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
// Deduplication by sorting (every pass streams):
//   1. generate: each entry's candidate key (and its matrix element);
//   2. sort: LSD radix sort of the keys in numeric order (qubit 0 the least
//      significant bit), carrying the entry index (stable: equal keys keep
//      entry order);
//   3. mark: a sorted position starts a candidate when its key differs from
//      the previous one; an exclusive scan of the marks numbers them;
//   4. scatter: cand_id[entry] = number of its key; each candidate's key and
//      its membership in U (the staged table of U) from its first position.
// The candidate order (numeric) and every entry's index are independent of
// thread timing.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_util.cuh"
#include "melem.cuh"
#include "nqs_internal.cuh"

namespace nqs {

constexpr int kCandThreads = 256;
constexpr int kCandWarps = kCandThreads / 32;

static inline int64_t a256c(int64_t v) { return (v + 255) & ~int64_t(255); }

// scratch layout of nqs_full_candidates
struct CandScratch {
  unsigned long long* counters;   // [1] probe limit hit
  uint64_t* keys[2];              // [entries][W] sort buffers (keys[0]: generated keys)
  int32_t* idx[2];                // [entries] sort payload buffers (entry index)
  int32_t* mark;                  // [entries + 1] candidate starts, then their exclusive scan
  int32_t* hist;                  // [256 * sort_blocks(entries)]
  int32_t* partial;               // [scan partials]
  int64_t bytes;
};

static CandScratch cand_scratch_view(char* base, int64_t entries, int W) {
  CandScratch v;
  std::memset(&v, 0, sizeof(v));
  const int64_t m = std::max<int64_t>(entries, 1);
  int64_t off = 0;
  auto take = [&](int64_t bytes) { char* p = base ? base + off : nullptr; off = a256c(off + bytes); return p; };
  v.counters = (unsigned long long*)take(256);
  v.keys[0] = (uint64_t*)take(8 * W * m);
  v.keys[1] = (uint64_t*)take(8 * W * m);
  v.idx[0] = (int32_t*)take(4 * m);
  v.idx[1] = (int32_t*)take(4 * m);
  v.mark = (int32_t*)take(4 * (m + 1));
  v.hist = (int32_t*)take(4 * 256 * sort_blocks(m));
  v.partial = (int32_t*)take(4 * std::max<int64_t>(sort_scan_partials(m), (m + 1) / 2048 + 2));
  // the E_loc sum reuses the scratch for 32 bytes per candidate (at most one per entry)
  v.bytes = std::max<int64_t>(off, 32 * m + 256);
  return v;
}

int64_t cand_scratch_bytes(const nqs_ham* ham, int64_t n_unq) {
  return cand_scratch_view(nullptr, n_unq * ham->n_xy, ham->W).bytes;
}

struct CandArgs {
  const uint64_t* U;
  const uint64_t* xy;          // [n_xy][W]
  int64_t n_unq, n_xy;
  uint64_t* keys;              // [entries][W] generated keys
  double* hval;                // [n_unq][n_xy] or null
};

// Work unit of a warp: one sample and a tile of kCandTile consecutive
// patterns (lanes take them in rounds of 32), so that few samples with many
// patterns still fill the GPU.  Matrix elements in FP64 as in the E_loc^var
// kernel (the diagonal by its quadratic form or term loop, heavy term-form
// patterns by the whole warp, the rest one lane each).
constexpr int kCandTile = 1024;

template <int W>
__global__ void __launch_bounds__(kCandThreads) cand_gen_kernel(const CandArgs a, const Melem M) {
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
    const uint64_t e0 = (uint64_t)i * (uint64_t)a.n_xy;
    if (M.has_diag && tc == 0) {  // pattern 0: x' = x, with the sample's first tile
      const double hd = a.hval ? melem_diag<PolicyD, W>(x, M) : 0.0;
      if (lane == 0) {
#pragma unroll
        for (int w = 0; w < W; ++w) a.keys[e0 * W + w] = x[w];
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
#pragma unroll
        for (int w = 0; w < W; ++w) a.keys[e * W + w] = c[w];
        if (a.hval) a.hval[e] = h;
      }
    }
  }
}

// mark[p] = 1 where sorted position p starts a candidate (its key differs from p - 1)
template <int W>
__global__ void cand_mark_kernel(int64_t m, const uint64_t* __restrict__ keys, int32_t* __restrict__ mark) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
    bool start = p == 0;
    if (!start) {
#pragma unroll
      for (int w = 0; w < W; ++w) start = start || __ldg(keys + p * W + w) != __ldg(keys + (p - 1) * W + w);
    }
    mark[p] = start ? 1 : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) mark[m] = 0;
}

// sorted position p (entry idx[p]); scan = exclusive scan of the marks (m + 1 values),
// so position p starts a candidate when scan[p + 1] - scan[p] = 1 and its candidate is
// u = scan[p] + start - 1: the entry's candidate index; at a candidate's first position
// its key and its index in U (or -1)
template <int W>
__global__ void cand_scatter_kernel(int64_t m, const uint64_t* __restrict__ keys, const int32_t* __restrict__ idx,
                                    const int32_t* __restrict__ scan, uint32_t* __restrict__ cand_id, uint64_t* __restrict__ cand,
                                    int32_t* __restrict__ in_u, const uint32_t* __restrict__ hx,
                                    const uint32_t* __restrict__ xy_hash, int64_t n_xy,
                                    const unsigned long long* __restrict__ utable, int64_t capmask,
                                    const uint64_t* __restrict__ U, unsigned long long* counters) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sc = scan[p];
    const bool first = scan[p + 1] - sc == 1;
    const int32_t e = idx[p];
    const int32_t u = sc + (first ? 1 : 0) - 1;
    cand_id[e] = (uint32_t)u;
    if (!first) continue;
    uint64_t c[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      c[w] = keys[p * W + w];
      cand[(int64_t)u * W + w] = c[w];
    }
    if (!in_u) continue;
    // x' = U_i XOR XY_k has the linear hash h(U_i) ^ h(XY_k), the key of the staged table of U
    const int64_t i = e / n_xy, k = e - i * n_xy;
    const uint32_t h = __ldg(hx + i) ^ __ldg(xy_hash + k);
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
    if (!done) atomicOr(counters, 1ull);
    in_u[u] = j;
  }
}

template <int W>
static cudaError_t cand_w(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage, const StageHeader& L,
                          const CandScratch& sc, uint32_t* cand_id, double* hval, uint64_t* cand, int32_t* in_u,
                          int64_t capacity, int64_t* n_cand, int* limit_hit, cudaStream_t s) {
  const int64_t entries = n * ham->n_xy;
  CandArgs a;
  a.U = U;
  a.xy = ham->xy;
  a.n_unq = n;
  a.n_xy = ham->n_xy;
  a.keys = sc.keys[0];
  a.hval = hval;
  cudaError_t e;
  if ((e = cudaMemsetAsync(sc.counters, 0, 256, s)) != cudaSuccess) return e;
  const int sms = num_sms();
  const int64_t k_first = ham->has_diag ? 1 : 0;
  const int64_t tiles = n * std::max<int64_t>(1, (ham->n_xy - k_first + kCandTile - 1) / kCandTile);
  const int gen_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + kCandWarps - 1) / kCandWarps, 16 * sms));
  cand_gen_kernel<W><<<gen_blocks, kCandThreads, 0, s>>>(a, melem_tables(ham, n));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // numeric sort of all entries' keys over their low ceil(N / 8) bytes, carrying the entry index
  uint64_t* kbuf[2] = {sc.keys[1], sc.keys[0]};
  int32_t* ibuf[2] = {sc.idx[1], sc.idx[0]};
  int out = -1;
  const int n_bytes = (ham->n_qubits + 7) / 8;
  if ((e = launch_sort_words(sc.keys[0], nullptr, entries, W, n_bytes, kbuf, ibuf, sc.hist, sc.partial, &out, s)) !=
      cudaSuccess)
    return e;
  const uint64_t* keys = out >= 0 ? kbuf[out] : sc.keys[0];
  const int32_t* idx = out >= 0 ? ibuf[out] : nullptr;   // n_bytes >= 1, so at least one pass ran
  const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((entries + 255) / 256, 16 * sms));
  cand_mark_kernel<W><<<eb, 256, 0, s>>>(entries, keys, sc.mark);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_scan_i32(sc.mark, entries + 1, sc.partial, s)) != cudaSuccess) return e;
  int32_t total = 0;
  if ((e = cudaMemcpyAsync(&total, sc.mark + entries, sizeof(total), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *n_cand = total;
  *limit_hit = 0;
  if (*n_cand > capacity) return cudaSuccess;
  cand_scatter_kernel<W><<<eb, 256, 0, s>>>(entries, keys, idx, sc.mark, cand_id, cand, in_u,
                                            (const uint32_t*)(stage + L.off_hx), ham->xy_hash, ham->n_xy,
                                            (const unsigned long long*)(stage + L.off_table), L.cap - 1, U,
                                            sc.counters);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (in_u) {  // the membership probe's limit flag
    unsigned long long lim = 0;
    if ((e = cudaMemcpyAsync(&lim, sc.counters, sizeof(lim), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *limit_hit = lim != 0;
  }
  return cudaSuccess;
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
// psi(x_k) = P_c 2^{K_c} per candidate (FP64 mantissa in [1, 2.03) and exponent,
// one exponential per candidate), 1/psi(x) = Q_x 2^{-K_x} per sample from the batch
// workspace's amplitude records; per entry a complex product and an exact
// power-of-two scaling (a contribution below the FP64 range is zero).  One
// warp per sample, lanes over the patterns, fixed summation order.
// --------------------------------------------------------------------------
// e^a = 2^k m for one candidate per thread, mostly on the FP32 pipes (the candidates are
// many and this part's FP64 rate is low): table-driven reduction a = (64 k + j) ln2 / 64 + r,
// 0 <= r < ln2 / 64, so e^a = 2^k 2^(j/64) e^r; 2^(j/64) from a double-float table, e^r by
// its Taylor series (1 + r + r^2/2 in double-float, the terms of degree 3..6, below
// 2.2e-7 in all, in FP32), the product in double-float; about 1e-14 relative.  The
// reduction follows the published table-driven scheme (Tang) with 64 entries.
struct Exp2Table {
  float2 t[64];   // 2^(j/64) as (hi, lo)
};

__device__ __forceinline__ double exp_mantissa(double a, const Exp2Table& T, int& k) {
  const double kInvStep = 92.332482616893656877;            // 64 / ln 2
  const double kStep = 0.6931471805599453094 / 64.0;         // ln 2 / 64 (double; the division is exact)
  const double kStepHi = (double)0.010830424f;               // its leading 24 bits: K kStepHi is exact
  const double kStepLo = kStep - kStepHi;
  double K = floor(a * kInvStep);
  K = fmin(fmax(K, -1.0e11), 1.0e11);
  const double rd = fma(-K, kStepLo, fma(-K, kStepHi, a));   // in [0, ln 2 / 64) up to rounding
  const long long Ki = (long long)K;
  const int j = (int)(Ki & 63);
  k = (int)((Ki - j) >> 6);
  const float rh = __double2float_rn(rd);
  const df r = {rh, __double2float_rn(rd - (double)rh)};
  // e^r = 1 + r + r^2 / 2 + q with q = r^3 / 6 + r^4 / 24 + r^5 / 120 + r^6 / 720 (< 2.2e-7)
  float q = __fmaf_rn(rh, 1.f / 720.f, 1.f / 120.f);
  q = __fmaf_rn(q, rh, 1.f / 24.f);
  q = __fmaf_rn(q, rh, 1.f / 6.f);
  q = __fmul_rn(__fmul_rn(q, rh), __fmul_rn(rh, rh));
  const df r2 = df_mul(r, r);
  df e = df_add(r, df{0.5f * r2.hi, 0.5f * r2.lo});
  e = df_add(e, df{q, 0.f});
  e = df_add(df{1.f, 0.f}, e);
  const float2 t = T.t[j];
  const df m = df_mul(df{t.x, t.y}, e);
  return (double)m.hi + (double)m.lo;
}

__global__ void cand_amp_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                AmpD* __restrict__ P, const Exp2Table T) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int k;
    const double m = exp_mantissa(a[i], T, k);
    if (b) {
      double c, s;
      sincos(b[i], &s, &c);
      P[i].v = make_double2(m * c, m * s);
    } else {
      P[i].v = make_double2(m, 0.0);
    }
    P[i].k = k;
  }
}

static Exp2Table exp2_table() {
  Exp2Table T;
  for (int j = 0; j < 64; ++j) {
    const double v = std::exp2(j / 64.0);
    const float hi = (float)v;
    T.t[j] = make_float2(hi, (float)(v - (double)hi));
  }
  return T;
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
  cudaError_t e = launch_amplitudes(a, b, n, NQS_PREC_FP64, (char*)stage, L, s, nullptr);
  if (e != cudaSuccess) return e;
  if (n_cand > 0)
    cand_amp_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((n_cand + 255) / 256, 8 * sms)), 256, 0, s>>>(
        n_cand, ca, cb, P, exp2_table());
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
