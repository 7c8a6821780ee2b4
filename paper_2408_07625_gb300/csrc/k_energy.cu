// MatrixElement + ScatterAdd -> E_loc^var, the variational energy and the adjoint.
//
// MatrixElement (supplementary algorithm "Calculating the Hamiltonian matrix
// element"): H_xx' = sum_{l in P_XY} c_l (-1)^{|x' & YZ_l|}, c_l = h_l i^{|Y_l|}.
// ScatterAdd (Fig. scatter_local_energies) becomes a row-owned reduction: one
// warp owns row x and sums H_xx' psi(x')/psi(x) over its CSR pairs in a fixed
// order, so no atomics are needed and results are bitwise reproducible.
//
// Amplitude ratios: psi(x) = P_x 2^{K_x} with |P_x| in [1, 2) (precomputed per
// sample in FP64), 1/psi(x) = Q_x 2^{-K_x}; psi(x')/psi(x) = P_x' Q_x 2^{K_x'-K_x}.
// This replaces one exp per pair by a (double-float) product and an exact
// power-of-two scaling.
#include <cfloat>
#include <mutex>

#include "device_util.cuh"
#include "melem.cuh"
#include "nqs_internal.cuh"

namespace nqs {

constexpr int kEnergyThreads = 256;
constexpr int kEnergyWarps = kEnergyThreads / 32;

// --------------------------------------------------------------------------
// per-sample amplitude factors
// --------------------------------------------------------------------------

__global__ void amplitudes_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                  int64_t n, int fp64, AmpF* __restrict__ Pf, AmpF* __restrict__ Qf,
                                  AmpD* __restrict__ Pd, AmpD* __restrict__ Qd, const uint64_t* __restrict__ U,
                                  int W) {
  const double kLn2 = 0.6931471805599453094;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ai = a[i];
    const double k = floor(ai / kLn2);
    const double m = exp(ai - k * kLn2);     // in [1, 2) up to rounding
    double c = 1.0, s = 0.0;
    if (b) sincos(b[i], &s, &c);
    const double pr = m * c, pi = m * s;
    const double qr = c / m, qi = -s / m;
    const int ki = (int)k;
    if (fp64) {
      Pd[i].v = make_double2(pr, pi);
      Pd[i].k = ki;
      Qd[i].v = make_double2(qr, qi);
      Qd[i].k = ki;
    } else {
      df dpr = df_from_double(pr), dpi = df_from_double(pi);
      df dqr = df_from_double(qr), dqi = df_from_double(qi);
      Pf[i].v = make_float4(dpr.hi, dpr.lo, dpi.hi, dpi.lo);
      Pf[i].k = ki;
      Qf[i].v = make_float4(dqr.hi, dqr.lo, dqi.hi, dqi.lo);
      Qf[i].k = ki;
    }
    if (U) Pf[i].x0 = __ldg(U + i * W);  // same bytes in both layouts
  }
}

cudaError_t launch_amplitudes(const double* a, const double* b, int64_t n, int precision,
                              char* stage, const StageHeader& L, cudaStream_t s, const uint64_t* U) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * num_sms());
  const bool fp64 = precision == NQS_PREC_FP64;
  amplitudes_kernel<<<blocks, 256, 0, s>>>(
      a, b, n, fp64 ? 1 : 0, (AmpF*)(stage + L.off_ampP), (AmpF*)(stage + L.off_ampQ),
      (AmpD*)(stage + L.off_ampP), (AmpD*)(stage + L.off_ampQ), U, L.W);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// row schedule: rows of [rb, re) in decreasing order of their pair count
// (power-of-two classes, heaviest first).  Rows of at least kLongRow pairs
// (they lead the order) are taken one per block, whose warps share the row's
// rounds; the rest are handed out to warps one at a time from a counter, so
// the longest rows start first and no warp idles while others hold several
// long rows.  Results do not depend on the order: a row is a fixed-order
// reduction whose shape depends on its length alone.
// --------------------------------------------------------------------------
constexpr int kRowClasses = 32;
constexpr int kLongRowBits = 11;                 // rows with bit length >= 11: at least 1024 pairs
constexpr int64_t kLongRow = int64_t(1) << (kLongRowBits - 1);

__device__ __forceinline__ int row_class(int64_t c) {  // 0: heaviest
  const int lg = c > 0 ? 64 - __clzll((long long)c) : 0;    // bit length, 0..35 for c < 2^35
  const int k = kRowClasses - 1 - lg;
  return k < 0 ? 0 : k;
}

__global__ void row_class_count_kernel(const int64_t* __restrict__ rp, int64_t rows, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t h[kRowClasses];
  if (threadIdx.x < kRowClasses) h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[row_class(rp[r + 1] - rp[r])], 1u);
  __syncthreads();
  if (threadIdx.x < kRowClasses && h[threadIdx.x]) atomicAdd(cnt + threadIdx.x, h[threadIdx.x]);
}

// rows to their places in the order, class by class: a block counts its rows
// per class in shared memory, reserves that many places per class with one
// global atomic each, then writes its rows (the order inside a class is free)
__global__ void row_order_kernel(const int64_t* __restrict__ rp, int64_t rows, const uint32_t* __restrict__ cnt,
                                 uint32_t* __restrict__ cursor, int32_t* __restrict__ order) {
  __shared__ uint32_t off[kRowClasses];
  __shared__ uint32_t local[kRowClasses];
  if (threadIdx.x < kRowClasses) local[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t r0 = blockIdx.x * (int64_t)blockDim.x * 4;
  const int64_t r1 = r0 + (int64_t)blockDim.x * 4 < rows ? r0 + (int64_t)blockDim.x * 4 : rows;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) atomicAdd(&local[row_class(rp[r + 1] - rp[r])], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int k = 0; k < kRowClasses; ++k) {
      off[k] = run + (local[k] ? atomicAdd(cursor + k, local[k]) : 0u);
      run += cnt[k];
      local[k] = 0u;
    }
  }
  __syncthreads();
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int k = row_class(rp[r + 1] - rp[r]);
    order[off[k] + atomicAdd(&local[k], 1u)] = (int32_t)r;
  }
}

struct RowSched {
  const int32_t* order;
  const uint32_t* cnt;           // rows per class
  unsigned long long* next;      // warp rows taken
  unsigned long long* next_long; // block rows taken
  int64_t rows;
};

// sched region of the workspace: counts [32] u32, cursors [32] u32, two row counters u64
static cudaError_t launch_row_order(const int64_t* rp, int64_t rows, char* stage, const StageHeader& L,
                                    RowSched& rs, cudaStream_t s) {
  char* base = stage + L.off_sched;
  uint32_t* cnt = (uint32_t*)base;
  uint32_t* cur = cnt + kRowClasses;
  rs.cnt = cnt;
  rs.next = (unsigned long long*)(cur + kRowClasses);
  rs.next_long = rs.next + 1;
  rs.order = (const int32_t*)(stage + L.off_order);
  rs.rows = rows;
  cudaError_t e = cudaMemsetAsync(base, 0, 2 * kRowClasses * 4 + 16, s);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, 2 * num_sms()));
  row_class_count_kernel<<<blocks, 256, 0, s>>>(rp, rows, cnt);
  row_order_kernel<<<(unsigned)((rows + 1023) / 1024), 256, 0, s>>>(rp, rows, cnt, cur, (int32_t*)(stage + L.off_order));
  return cudaGetLastError();
}

// number of long rows (they lead the order)
__device__ __forceinline__ int64_t long_rows(const RowSched& rs) {
  int64_t n = 0;
  for (int k = 0; k <= kRowClasses - 1 - kLongRowBits; ++k) n += rs.cnt[k];
  return n;
}

// next long row for the whole block (-1: none left); all threads call it
__device__ __forceinline__ int64_t next_long_row(const RowSched& rs, int64_t n_long, int64_t* slot) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long v = atomicAdd(rs.next_long, 1ull);
    *slot = (int64_t)v < n_long ? (int64_t)__ldg(rs.order + v) : -1;
  }
  __syncthreads();
  return *slot;
}

__device__ __forceinline__ int64_t next_row(const RowSched& rs, int64_t n_long) {
  unsigned long long v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(rs.next, 1ull);
  const int64_t i = n_long + (int64_t)__shfl_sync(kFull, v, 0);
  return i < rs.rows ? (int64_t)__ldg(rs.order + i) : -1;
}

// matrix elements kept per pair for the adjoint: (hi, lo) floats or doubles
template <class Pol> struct HStore;
// (complex H: both parts, float4 or double2 per pair)
template <> struct HStore<PolicyF> {
  using V = float2;
  __device__ static void put(void* h, int64_t q, df v) { reinterpret_cast<float2*>(h)[q] = make_float2(v.hi, v.lo); }
  __device__ static df get(const void* h, int64_t q) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(h) + q);
    return {v.x, v.y};
  }
  __device__ static void put2(void* h, int64_t q, df r, df i) {
    reinterpret_cast<float4*>(h)[q] = make_float4(r.hi, r.lo, i.hi, i.lo);
  }
  __device__ static void get2(const void* h, int64_t q, df& r, df& i) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(h) + q);
    r = {v.x, v.y};
    i = {v.z, v.w};
  }
};
template <> struct HStore<PolicyD> {
  using V = double;
  __device__ static void put(void* h, int64_t q, double v) { reinterpret_cast<double*>(h)[q] = v; }
  __device__ static double get(const void* h, int64_t q) { return __ldg(reinterpret_cast<const double*>(h) + q); }
  __device__ static void put2(void* h, int64_t q, double r, double i) {
    reinterpret_cast<double2*>(h)[q] = make_double2(r, i);
  }
  __device__ static void get2(const void* h, int64_t q, double& r, double& i) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(h) + q);
    r = v.x;
    i = v.y;
  }
};

// Arithmetic modes of the energy and adjoint kernels (template CX): real H
// with real log psi (0), real H with complex log psi (1), complex H (2; the
// local energies are complex whatever log psi is).
constexpr int kReal = 0, kCplxPsi = 1, kCplxH = 2;

// Pair lists come as two uint32 arrays (pair_j: column, pair_k: pattern) or,
// with pair_k == NULL, as packed 64-bit words in pair_j (column << 32 | pattern).
__device__ __forceinline__ void load_pair(const uint32_t* __restrict__ pj, const uint32_t* __restrict__ pk,
                                          int64_t q, uint32_t& j, uint32_t& k) {
  if (pk) {
    j = __ldg(pj + q);
    k = __ldg(pk + q);
  } else {
    const unsigned long long v = __ldg(reinterpret_cast<const unsigned long long*>(pj) + q);
    j = (uint32_t)(v >> 32);
    k = (uint32_t)v;
  }
}
__device__ __forceinline__ uint32_t load_col(const uint32_t* __restrict__ pj, const uint32_t* __restrict__ pk,
                                             int64_t q) {
  return pk ? __ldg(pj + q) : (uint32_t)(__ldg(reinterpret_cast<const unsigned long long*>(pj) + q) >> 32);
}
__device__ __forceinline__ uint32_t load_pat(const uint32_t* __restrict__ pj, const uint32_t* __restrict__ pk,
                                             int64_t q) {
  return pk ? __ldg(pk + q) : (uint32_t)__ldg(reinterpret_cast<const unsigned long long*>(pj) + q);
}

// a term added to an exact row sum (Fx); a term out of its range flags the status
template <class Pol>
__device__ __forceinline__ void fx_term(Fx& a, typename Pol::T t, int32_t* status) {
  if (!Pol::fx(a, t)) atomicOr(status, kStatusRange);
}

// --------------------------------------------------------------------------
// E_loc^var over CSR pairs.  A row is a sequence of rounds of 32 pairs; each
// pair is evaluated by the lane that holds it (linear form or the pattern's
// terms), and heavy patterns without a linear form are summed by all lanes
// (then reduced across the warp).  The pair's lane adds H * ratio to its
// exact fixed-point sum and, if asked, stores H for the adjoint.  The next
// round's pair indices are loaded while the current round is evaluated.  A
// short row is one warp's rounds; a long row's rounds are dealt to the
// block's warps in turn.  The sums are exact, so a row's E_loc^var does not
// depend on the order of its pairs (sorted by column or as the search placed
// them) nor on the lane or warp that took each pair; it is rounded to FP64
// once at the end.
// --------------------------------------------------------------------------
template <class Pol, int W, int CX, bool STORE_H>
__device__ __forceinline__ void energy_rounds(const uint64_t* __restrict__ U, const Melem& M, const char* P,
                                              const char* Q, int64_t i, int64_t p, int64_t p1,
                                              int64_t first, int64_t stride, const uint32_t* __restrict__ pair_j,
                                              const uint32_t* __restrict__ pair_k, void* hpair, int32_t* status,
                                              Fx& acc_re, Fx& acc_im) {
  using T = typename Pol::T;
  const int lane = threadIdx.x & 31;
  uint32_t jn = 0u, kn = 0u;
  int64_t base = p + 32 * first;
  if (base + lane < p1) {
    load_pair(pair_j, pair_k, base + lane, jn, kn);
  }
  for (; base < p1; base += 32 * stride) {
    const int64_t q = base + lane;
    const uint32_t j = jn, k = kn;
    const bool have = q < p1 && pair_in_range(M, j, k, status);
    if (q + 32 * stride < p1) {
      load_pair(pair_j, pair_k, q + 32 * stride, jn, kn);
    }
    // N <= 64: the pattern's descriptor and sign mask are one 32-byte record, and the
    // column's bit word rides in its amplitude record (read with the ratio's factor)
    int4 fm = make_int4(0, 0, 0, 0);
    uint64_t amask = 0ull;
    if (W == 1) {
      if (have) {
        const int4* rec = M.fmx + 2 * (int64_t)k;
        fm = __ldg(rec);
        const int4 m2 = __ldg(rec + 1);
        amask = (uint64_t)(uint32_t)m2.x | ((uint64_t)(uint32_t)m2.y << 32);
      }
    } else if (have) {
      fm = __ldg(M.fm + k);
    }
    const bool coop = have && (int64_t)k < M.heavy_end && (fm.x & 15) == kForm::Terms;
    T h = Pol::zero(), h_im = Pol::zero();
    uint32_t hb = __ballot_sync(kFull, coop);
    while (hb) {  // heavy pattern in term form: all lanes share its term loop, its lane keeps H
      const int src = __ffs(hb) - 1;
      hb &= hb - 1;
      const uint32_t jj = __shfl_sync(kFull, j, src);
      const uint32_t kk = __shfl_sync(kFull, k, src);
      uint64_t xp[W];
      load_words<W>(U + (int64_t)jj * W, xp);
      const int64_t t0 = (int64_t)__ldg(M.t_ptr + kk), t1 = (int64_t)__ldg(M.t_ptr + kk + 1);
      if (CX == kCplxH) {
        T hwr, hwi;
        melem_warp_c<Pol, W>(xp, t0, t1, M, hwr, hwi);
        if (lane == src) { h = hwr; h_im = hwi; }
      } else {
        const T hw = melem_warp<Pol, W>(xp, t0, t1, M);
        if (lane == src) h = hw;
      }
    }
    if (have) {
      if (!coop) {
        uint64_t xp[W];
        if (W == 1) xp[0] = __ldg(reinterpret_cast<const uint64_t*>(P + 32 * (int64_t)j) + 3);
        else load_words<W>(U + (int64_t)j * W, xp);
        if (CX == kCplxH) melem_lane_c<Pol, W>(xp, k, fm, M, h, h_im);
        else if (W == 1 && (fm.x & 15) == kForm::Local) h = melem_local1<Pol>(xp[0], fm, amask, M);
        else h = melem_lane<Pol, W>(xp, k, fm, M);
      }
      T rr, ri;
      ratio<Pol, CX != kReal>(P, Q, j, i, rr, ri, status);
      if (CX == kCplxH) {  // (h + i h_im)(rr + i ri)
        fx_term<Pol>(acc_re, Pol::mul(h, rr), status);
        fx_term<Pol>(acc_re, Pol::neg(Pol::mul(h_im, ri)), status);
        fx_term<Pol>(acc_im, Pol::mul(h, ri), status);
        fx_term<Pol>(acc_im, Pol::mul(h_im, rr), status);
        if (STORE_H) HStore<Pol>::put2(hpair, q, h, h_im);
      } else {
        fx_term<Pol>(acc_re, Pol::mul(h, rr), status);
        if (CX == kCplxPsi) fx_term<Pol>(acc_im, Pol::mul(h, ri), status);
        if (STORE_H) HStore<Pol>::put(hpair, q, h);
      }
    }
  }
}

// the diagonal pair, if the row starts with it: H_xx added by lane 0 (psi(x)/psi(x) = 1)
template <class Pol, int W, int CX, bool STORE_H>
__device__ __forceinline__ bool energy_diag(const uint64_t* __restrict__ U, const Melem& M, int64_t i, int64_t p,
                                            int64_t p1, const uint32_t* __restrict__ pair_j,
                                            const uint32_t* __restrict__ pair_k, void* hpair,
                                            Fx& acc_re, double& hd, int32_t* status) {
  if (!(M.has_diag && p < p1 && load_pat(pair_j, pair_k, p) == 0u)) return false;
  uint64_t xi[W];
  load_words<W>(U + i * W, xi);
  const typename Pol::T h = melem_diag<Pol, W>(xi, M);
  hd = Pol::to_d(h);
  if ((threadIdx.x & 31) == 0) {
    fx_term<Pol>(acc_re, h, status);
    if (STORE_H) {
      if (CX == kCplxH) HStore<Pol>::put2(hpair, p, h, Pol::zero());  // H_xx is real
      else HStore<Pol>::put(hpair, p, h);
    }
  }
  return true;
}

// Real H and amplitudes on one-word samples are held to 48 registers (five
// blocks per SM, no spills); the other forms keep the compiler's choice, which
// a cap would make spill.
template <class Pol, int W, int CX, bool STORE_H>
__global__ void __launch_bounds__(kEnergyThreads, (W == 1 && CX == 0) ? 5 : 1)
local_energy_kernel(const uint64_t* __restrict__ U, const Melem M, const char* __restrict__ P,
                    const char* __restrict__ Q, int64_t row_begin, RowSched rs,
                    const int64_t* __restrict__ rp, const uint32_t* __restrict__ pair_j,
                    const uint32_t* __restrict__ pair_k, double* __restrict__ eloc_re,
                    double* __restrict__ eloc_im, double* __restrict__ hdiag, void* __restrict__ hpair,
                    int32_t* __restrict__ status) {
  __shared__ Fx s_re[kEnergyWarps], s_im[kEnergyWarps];
  __shared__ int64_t s_row;
  if (*(volatile int32_t*)status & kStatusCapacity) return;  // the pair list was not written
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t n_long = long_rows(rs);
  for (int64_t row = next_long_row(rs, n_long, &s_row); row >= 0; row = next_long_row(rs, n_long, &s_row)) {
    const int64_t i = row + row_begin;
    int64_t p = rp[row] - rp[0];
    const int64_t p1 = rp[row + 1] - rp[0];
    Fx acc_re = fx_zero(), acc_im = fx_zero();
    double hd = 0.0;
    if (warp == 0) energy_diag<Pol, W, CX, STORE_H>(U, M, i, p, p1, pair_j, pair_k, hpair, acc_re, hd, status);
    if (M.has_diag && p < p1 && load_pat(pair_j, pair_k, p) == 0u) ++p;
    energy_rounds<Pol, W, CX, STORE_H>(U, M, P, Q, i, p, p1, warp, kEnergyWarps, pair_j, pair_k, hpair,
                                       status, acc_re, acc_im);
    const Fx er = fx_warp_sum(acc_re);
    const Fx ei = CX != kReal ? fx_warp_sum(acc_im) : fx_zero();
    if (lane == 0) {
      s_re[warp] = er;
      s_im[warp] = ei;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Fx tr = s_re[0], ti = s_im[0];
      for (int w = 1; w < kEnergyWarps; ++w) {
        fx_add(tr, s_re[w]);
        fx_add(ti, s_im[w]);
      }
      eloc_re[i] = fx_to_double(tr);
      if (eloc_im) eloc_im[i] = fx_to_double(ti);
      if (hdiag) hdiag[i] = hd;
    }
  }
  for (int64_t row = next_row(rs, n_long); row >= 0; row = next_row(rs, n_long)) {
    const int64_t i = row + row_begin;
    int64_t p = rp[row] - rp[0];
    const int64_t p1 = rp[row + 1] - rp[0];
    Fx acc_re = fx_zero(), acc_im = fx_zero();
    double hd = 0.0;
    if (energy_diag<Pol, W, CX, STORE_H>(U, M, i, p, p1, pair_j, pair_k, hpair, acc_re, hd, status)) ++p;
    energy_rounds<Pol, W, CX, STORE_H>(U, M, P, Q, i, p, p1, 0, 1, pair_j, pair_k, hpair, status, acc_re,
                                         acc_im);
    const Fx er = fx_warp_sum(acc_re);
    const Fx ei = CX != kReal ? fx_warp_sum(acc_im) : fx_zero();
    if (lane == 0) {
      eloc_re[i] = fx_to_double(er);
      if (eloc_im) eloc_im[i] = fx_to_double(ei);
      if (hdiag) hdiag[i] = hd;
    }
  }
}

template <class Kern>
static int grid_for(Kern kern, int64_t rows) {
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kEnergyThreads, 0);
  if (occ < 1) occ = 1;
  return (int)std::max<int64_t>(1, std::min<int64_t>((rows + kEnergyWarps - 1) / kEnergyWarps,
                                                     (int64_t)num_sms() * occ));
}

template <class Pol, int W, int CX, bool STORE_H>
static void launch_le(const nqs_ham* ham, const uint64_t* U, const char* stage, const StageHeader& L,
                      int64_t rb, const RowSched& rs, const int64_t* rp, const uint32_t* pj,
                      const uint32_t* pk, double* er, double* ei, double* hd, void* hpair, cudaStream_t s) {
  auto kern = local_energy_kernel<Pol, W, CX, STORE_H>;
  kern<<<grid_for(kern, rs.rows), kEnergyThreads, 0, s>>>(
      U, melem_tables(ham, L.n_unq), stage + L.off_ampP, stage + L.off_ampQ, rb, rs, rp,
      pj, pk, er, ei, hd, hpair, (int32_t*)(stage + offsetof(StageHeader, status)));
}

template <class Pol, int CX, bool STORE_H>
static void launch_le_w(const nqs_ham* ham, const uint64_t* U, const char* stage, const StageHeader& L,
                        int64_t rb, const RowSched& rs, const int64_t* rp, const uint32_t* pj,
                        const uint32_t* pk, double* er, double* ei, double* hd, void* hpair, cudaStream_t s) {
  switch (ham->W) {
    case 1: launch_le<Pol, 1, CX, STORE_H>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s); break;
    case 2: launch_le<Pol, 2, CX, STORE_H>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s); break;
    case 3: launch_le<Pol, 3, CX, STORE_H>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s); break;
    default: launch_le<Pol, 4, CX, STORE_H>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s); break;
  }
}

template <class Pol>
static void launch_le_p(const nqs_ham* ham, const uint64_t* U, const char* stage, const StageHeader& L, bool cplx,
                        int64_t rb, const RowSched& rs, const int64_t* rp, const uint32_t* pj, const uint32_t* pk,
                        double* er, double* ei, double* hd, void* hpair, cudaStream_t s) {
  if (ham->cplx) {
    if (hpair) launch_le_w<Pol, kCplxH, true>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s);
    else launch_le_w<Pol, kCplxH, false>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s);
  } else if (cplx) {
    if (hpair) launch_le_w<Pol, kCplxPsi, true>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s);
    else launch_le_w<Pol, kCplxPsi, false>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s);
  } else {
    if (hpair) launch_le_w<Pol, kReal, true>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s);
    else launch_le_w<Pol, kReal, false>(ham, U, stage, L, rb, rs, rp, pj, pk, er, ei, hd, hpair, s);
  }
}

cudaError_t launch_local_energy(const nqs_ham* ham, const uint64_t* U, int64_t, const char* stage,
                                const StageHeader& L, bool cplx, int64_t rb, int64_t re,
                                const int64_t* rp, const uint32_t* pj, const uint32_t* pk,
                                int precision, double* er, double* ei, double* hd, void* hpair,
                                cudaStream_t s) {
  if (re <= rb) return cudaSuccess;
  RowSched rs;
  cudaError_t e = launch_row_order(rp, re - rb, (char*)stage, L, rs, s);
  if (e != cudaSuccess) return e;
  if (precision == NQS_PREC_FP64) launch_le_p<PolicyD>(ham, U, stage, L, cplx, rb, rs, rp, pj, pk, er, ei, hd, hpair, s);
  else launch_le_p<PolicyF>(ham, U, stage, L, cplx, rb, rs, rp, pj, pk, er, ei, hd, hpair, s);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// E^var: one block, FP64, fixed reduction order
// --------------------------------------------------------------------------
constexpr int kRedThreads = 1024;

__device__ double block_reduce_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  return sh[0];
}

__device__ double block_reduce_max(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = -DBL_MAX;
  if (warp == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : -DBL_MAX;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(kFull, r, o));
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  return sh[0];
}

// One pass: block b takes a contiguous chunk, finds its own max m_b and the
// sums S_b = sum exp(2 (a - m_b)), N_b = sum exp(2 (a - m_b)) E_loc; the last
// block to finish rescales them to the global max in block order.
__global__ void __launch_bounds__(kRedThreads)
evar_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ er,
            unsigned int* __restrict__ done, double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
  double m = -DBL_MAX;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) m = fmax(m, a[i]);
  const double mb = block_reduce_max(m, sh);
  double sw = 0.0, swe = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double w = exp(2.0 * (a[i] - mb));
    sw += w;
    swe += w * er[i];
  }
  const double Sb = block_reduce_sum(sw, sh);
  const double Nb = block_reduce_sum(swe, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = mb;
    part[3 * blockIdx.x + 1] = Sb;
    part[3 * blockIdx.x + 2] = Nb;
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int G = gridDim.x;
  double mm = -DBL_MAX;
  for (int b = threadIdx.x; b < G; b += blockDim.x) mm = fmax(mm, __ldcg(part + 3 * b));
  const double amax = block_reduce_max(mm, sh);
  double s1 = 0.0, s2 = 0.0;
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    const double mbb = __ldcg(part + 3 * b);
    const double f = (mbb == -DBL_MAX) ? 0.0 : exp(2.0 * (mbb - amax));
    s1 += __ldcg(part + 3 * b + 1) * f;
    s2 += __ldcg(part + 3 * b + 2) * f;
  }
  const double S = block_reduce_sum(s1, sh);
  const double N = block_reduce_sum(s2, sh);
  if (threadIdx.x == 0) {
    out[0] = N / S;
    out[1] = amax;
    out[2] = S;
    *done = 0u;  // ready for the next call
  }
}

cudaError_t launch_variational_energy(int64_t n, const double* a, const double* er, char* work,
                                      double* out, cudaStream_t s) {
  // one block per SM once there are 256 samples per SM: the FP64 exp per
  // sample runs on every SM (FP64 issue is scarce on this part)
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, std::min(kRedBlocks, num_sms())));
  unsigned int* done = (unsigned int*)(work + kRedOffset);
  double* part = (double*)(work + kRedOffset + 256);
  evar_kernel<<<G, kRedThreads, 0, s>>>(n, a, er, done, part, out);
  return cudaGetLastError();
}

// E^var of a batch from the triples of row blocks that partition it (one
// per rank when the rows are sharded): rescale every block's weight sum to
// the largest max, in block order.
__global__ void evar_combine_kernel(const double* __restrict__ parts, int k, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double amax = -DBL_MAX;
  for (int r = 0; r < k; ++r)
    if (parts[3 * r + 2] > 0.0) amax = fmax(amax, parts[3 * r + 1]);
  double S = 0.0, N = 0.0;
  for (int r = 0; r < k; ++r) {
    if (!(parts[3 * r + 2] > 0.0)) continue;
    const double f = exp(2.0 * (parts[3 * r + 1] - amax));
    S += parts[3 * r + 2] * f;
    N += parts[3 * r] * parts[3 * r + 2] * f;
  }
  out[0] = S > 0.0 ? N / S : 0.0;
  out[1] = amax;
  out[2] = S;
}

cudaError_t launch_evar_combine(const double* parts, int k, double* out, cudaStream_t s) {
  evar_combine_kernel<<<1, 32, 0, s>>>(parts, k, out);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// E^var without caller memory: the partial sums live in a file-scope device
// array instead of the batch workspace.  For callers that cannot allocate
// device memory (see nqs_variational_energy_noalloc in nqs.h).
// --------------------------------------------------------------------------
constexpr int kStaticRedBlocks = 1024;           // partial-sum slots in the array
constexpr int64_t kStaticRedChunk = 2048;        // samples per block
constexpr int64_t kStaticRedMax = kStaticRedBlocks * kStaticRedChunk;  // 2,097,152 samples
static __device__ __align__(256) unsigned char g_evar_scratch[256 + 3 * 8 * kStaticRedBlocks];

static std::mutex g_evar_scratch_mu;
static void* g_evar_scratch_addr[256] = {};      // device address of the array, per device

// Device address of g_evar_scratch on the current device; looked up once per
// device (the host-side name is only a stand-in for the device array).
static cudaError_t evar_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_evar_scratch_mu);
  if (!g_evar_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_evar_scratch);
    if (e != cudaSuccess) return e;
    g_evar_scratch_addr[dev] = p;
  }
  *out = g_evar_scratch_addr[dev];
  return cudaSuccess;
}

// --------------------------------------------------------------------------
// adjoint
// --------------------------------------------------------------------------
// per-sample effective upstream: ge(x) = g_re(x) + g_E w(x), gi(x) = g_im(x);
// and, for the rows y of [rb, re), the row's own terms of the gradient,
// D_yy = -(E_loc(y) - H_yy) and g_E 2 w_y (Re E_loc(y) - E):
//   own(y) = (ge_y Re D + gi_y Im D + g_E 2 w_y (Re E_loc(y) - E), gi_y Re D - ge_y Im D)
// (FP64 once per sample, all lanes busy, instead of in the row kernels' epilogue)
__global__ void geff_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ evar,
                            const double* __restrict__ g_re, const double* __restrict__ g_im,
                            const double* __restrict__ g_evar, int fp64, double2* __restrict__ gd,
                            float4* __restrict__ gf, int64_t rb, int64_t re, const double* __restrict__ er,
                            const double* __restrict__ ei, const double* __restrict__ hdiag,
                            double2* __restrict__ own, char* __restrict__ qrec) {
  const double gE = g_evar ? g_evar[0] : 0.0;
  const double E = evar[0], amax = evar[1], S = evar[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double w = exp(2.0 * (a[i] - amax)) / S;
    const double ge = (g_re ? g_re[i] : 0.0) + gE * w;
    const double gi = g_im ? g_im[i] : 0.0;
    if (fp64) {
      gd[i] = make_double2(ge, gi);
      if (qrec) *reinterpret_cast<double*>(qrec + 32 * i + 24) = ge;
    } else {
      df a1 = df_from_double(ge), a2 = df_from_double(gi);
      gf[i] = make_float4(a1.hi, a1.lo, a2.hi, a2.lo);
      if (qrec) *reinterpret_cast<float2*>(qrec + 32 * i + 24) = make_float2(a1.hi, a1.lo);
    }
    if (i >= rb && i < re) {
      const double Dr = -(er[i] - hdiag[i]);
      const double Di = ei ? -ei[i] : 0.0;
      own[i] = make_double2(ge * Dr + gi * Di + gE * 2.0 * w * (er[i] - E), gi * Dr - ge * Di);
    }
  }
}

// closed form: g(y) = g_E 2 w_y (E_loc(y) - E) (+ i g_E 2 w_y Im E_loc(y))
__global__ void backward_closed_kernel(int64_t rb, int64_t re, const double* __restrict__ a,
                                       const double* __restrict__ er, const double* __restrict__ ei,
                                       const double* __restrict__ evar, const double* __restrict__ g_evar,
                                       double* __restrict__ gre, double* __restrict__ gim) {
  const double gE = g_evar ? g_evar[0] : 0.0;
  const double E = evar[0], amax = evar[1], S = evar[2];
  for (int64_t y = rb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < re;
       y += (int64_t)gridDim.x * blockDim.x) {
    const double w = exp(2.0 * (a[y] - amax)) / S;
    gre[y] = gE * 2.0 * w * (er[y] - E);
    if (gim) gim[y] = ei ? gE * 2.0 * w * ei[y] : 0.0;
  }
}

template <class Pol>
__device__ __forceinline__ void load_geff(const char* G, int64_t i, typename Pol::T& ge, typename Pol::T& gi) {
  Pol::load_v(G, i, ge, gi);
}

// row y: sum over pairs (y, x), x != y, of ge(x) Re T + gi(x) Im T (and the
// Im-part analogue) with T = H_yx psi(y)/psi(x) = H_xy psi(y)/psi(x), summed
// exactly (fixed point, independent of the pairs' order); then the diagonal
// term D_yy = -(E_loc(y) - H_yy) and g_E 2 w_y (Re E_loc(y) - E).
// With LOAD_H the matrix elements come from the forward call's store (one
// lane per pair, no term loop); otherwise they are recomputed exactly as the
// forward computes them, so both forms give the same bits.
template <class Pol, int W, int CX, bool LOAD_H>
__device__ __forceinline__ void backward_rounds(const uint64_t* __restrict__ U, const Melem& M, const char* P,
                                                const char* Q, const char* G, int64_t y, int64_t p,
                                                int64_t p1, int64_t first, int64_t stride,
                                                const uint32_t* __restrict__ pair_j,
                                                const uint32_t* __restrict__ pair_k, const void* hpair,
                                                int32_t* status, Fx& da, Fx& db) {
  using T = typename Pol::T;
  const int lane = threadIdx.x & 31;
  uint32_t jn = 0u, kn = 0u;
  int64_t base = p + 32 * first;
  if (base + lane < p1) {
    if (LOAD_H) jn = load_col(pair_j, pair_k, base + lane);
    else load_pair(pair_j, pair_k, base + lane, jn, kn);
  }
  for (; base < p1; base += 32 * stride) {
    const int64_t q = base + lane;
    const uint32_t j = jn, k = kn;
    const bool have = q < p1 && pair_in_range(M, j, k, status);
    if (q + 32 * stride < p1) {
      if (LOAD_H) jn = load_col(pair_j, pair_k, q + 32 * stride);
      else load_pair(pair_j, pair_k, q + 32 * stride, jn, kn);
    }
    T h = Pol::zero(), h_im = Pol::zero();
    if (LOAD_H) {
      if (have) {
        if (CX == kCplxH) HStore<Pol>::get2(hpair, q, h, h_im);
        else h = HStore<Pol>::get(hpair, q);
      }
    } else {
      const int4 fm = have ? __ldg(M.fm + k) : make_int4(0, 0, 0, 0);
      const bool coop = have && (int64_t)k < M.heavy_end && (fm.x & 15) == kForm::Terms;
      uint32_t hb = __ballot_sync(kFull, coop);
      while (hb) {
        const int src = __ffs(hb) - 1;
        hb &= hb - 1;
        const uint32_t jj = __shfl_sync(kFull, j, src);
        const uint32_t kk = __shfl_sync(kFull, k, src);
        uint64_t xp[W];
        load_words<W>(U + (int64_t)jj * W, xp);
        const int64_t t0 = (int64_t)__ldg(M.t_ptr + kk), t1 = (int64_t)__ldg(M.t_ptr + kk + 1);
        if (CX == kCplxH) {
          T hwr, hwi;
          melem_warp_c<Pol, W>(xp, t0, t1, M, hwr, hwi);
          if (lane == src) { h = hwr; h_im = hwi; }
        } else {
          const T hw = melem_warp<Pol, W>(xp, t0, t1, M);
          if (lane == src) h = hw;
        }
      }
      if (have && !coop) {
        uint64_t xp[W];
        load_words<W>(U + (int64_t)j * W, xp);
        if (CX == kCplxH) melem_lane_c<Pol, W>(xp, k, fm, M, h, h_im);
        else h = melem_lane<Pol, W>(xp, k, fm, M);
      }
    }
    if (have) {
      T rr, ri, ge, gi;
      ratio<Pol, CX != kReal>(P, Q, y, j, rr, ri, status);
      if (CX == kReal) ge = Pol::load_slot(Q, j);   // the adjoint weight rides in the record of 1/psi(j)
      else load_geff<Pol>(G, j, ge, gi);
      if (CX == kCplxH) {
        // row y holds H_yj; the pair's term uses H_jy = conj(H_yj) (H Hermitian):
        // T = conj(h) psi(y)/psi(j) = (h rr + h_im ri) + i (h ri - h_im rr)
        const T tr = Pol::add(Pol::mul(h, rr), Pol::mul(h_im, ri));
        const T ti = Pol::add(Pol::mul(h, ri), Pol::neg(Pol::mul(h_im, rr)));
        fx_term<Pol>(da, Pol::mul(ge, tr), status);
        fx_term<Pol>(da, Pol::mul(gi, ti), status);
        fx_term<Pol>(db, Pol::neg(Pol::mul(ge, ti)), status);
        fx_term<Pol>(db, Pol::mul(gi, tr), status);
      } else {
        const T tr = Pol::mul(h, rr);
        fx_term<Pol>(da, Pol::mul(ge, tr), status);
        if (CX == kCplxPsi) {
          const T ti = Pol::mul(h, ri);
          fx_term<Pol>(da, Pol::mul(gi, ti), status);
          fx_term<Pol>(db, Pol::neg(Pol::mul(ge, ti)), status);
          fx_term<Pol>(db, Pol::mul(gi, tr), status);
        }
      }
    }
  }
}

// the pair sums plus the row's own terms (from geff_kernel)
template <bool CPLX>
__device__ __forceinline__ void backward_finish(int64_t y, double sa, double sb, const double2* own, double* gre,
                                                double* gim) {
  const double2 o = own[y];
  gre[y] = sa + o.x;
  if (gim) gim[y] = CPLX ? sb + o.y : 0.0;
}

template <class Pol, int W, int CX, bool LOAD_H>
__global__ void __launch_bounds__(kEnergyThreads)
backward_pairs_kernel(const uint64_t* __restrict__ U, const Melem M,
                      const char* __restrict__ P, const char* __restrict__ Q, const char* __restrict__ G,
                      int64_t row_begin, RowSched rs, const int64_t* __restrict__ rp,
                      const uint32_t* __restrict__ pair_j, const uint32_t* __restrict__ pair_k,
                      const void* __restrict__ hpair, const double2* __restrict__ own,
                      double* __restrict__ gre, double* __restrict__ gim, int32_t* __restrict__ status) {
  __shared__ Fx s_a[kEnergyWarps], s_b[kEnergyWarps];
  __shared__ int64_t s_row;
  if (*(volatile int32_t*)status & kStatusCapacity) return;  // the pair list was not written
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t n_long = long_rows(rs);
  for (int64_t row = next_long_row(rs, n_long, &s_row); row >= 0; row = next_long_row(rs, n_long, &s_row)) {
    const int64_t y = row + row_begin;
    int64_t p = rp[row] - rp[0];
    const int64_t p1 = rp[row + 1] - rp[0];
    if (M.has_diag && p < p1 && load_pat(pair_j, pair_k, p) == 0u) ++p;
    Fx da = fx_zero(), db = fx_zero();
    backward_rounds<Pol, W, CX, LOAD_H>(U, M, P, Q, G, y, p, p1, warp, kEnergyWarps, pair_j, pair_k, hpair,
                                          status, da, db);
    da = fx_warp_sum(da);
    db = CX != kReal ? fx_warp_sum(db) : fx_zero();
    if (lane == 0) {
      s_a[warp] = da;
      s_b[warp] = db;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Fx ta = s_a[0], tb = s_b[0];
      for (int w = 1; w < kEnergyWarps; ++w) {
        fx_add(ta, s_a[w]);
        fx_add(tb, s_b[w]);
      }
      backward_finish<CX != kReal>(y, fx_to_double(ta), CX != kReal ? fx_to_double(tb) : 0.0, own, gre, gim);
    }
  }
  for (int64_t row = next_row(rs, n_long); row >= 0; row = next_row(rs, n_long)) {
    const int64_t y = row + row_begin;
    int64_t p = rp[row] - rp[0];
    const int64_t p1 = rp[row + 1] - rp[0];
    if (M.has_diag && p < p1 && load_pat(pair_j, pair_k, p) == 0u) ++p;
    Fx da = fx_zero(), db = fx_zero();
    backward_rounds<Pol, W, CX, LOAD_H>(U, M, P, Q, G, y, p, p1, 0, 1, pair_j, pair_k, hpair, status, da, db);
    const double sa = fx_to_double(fx_warp_sum(da));
    const double sb = CX != kReal ? fx_to_double(fx_warp_sum(db)) : 0.0;
    if (lane == 0) backward_finish<CX != kReal>(y, sa, sb, own, gre, gim);
  }
}

struct BwArgs {
  const double2* own;
  double *gre, *gim;
  const void* hpair;
};

template <class Pol, int W, int CX, bool LOAD_H>
static void launch_bw(const nqs_ham* ham, const uint64_t* U, char* stage, const StageHeader& L, int64_t rb,
                      const RowSched& rs, const int64_t* rp, const uint32_t* pj, const uint32_t* pk,
                      const BwArgs& b, cudaStream_t s) {
  auto kern = backward_pairs_kernel<Pol, W, CX, LOAD_H>;
  kern<<<grid_for(kern, rs.rows), kEnergyThreads, 0, s>>>(
      U, melem_tables(ham, L.n_unq), stage + L.off_ampP, stage + L.off_ampQ, stage + L.off_geff, rb, rs, rp, pj, pk, b.hpair, b.own, b.gre, b.gim,
      (int32_t*)(stage + offsetof(StageHeader, status)));
}

template <class Pol, int CX, bool LOAD_H>
static void launch_bw_w(const nqs_ham* ham, const uint64_t* U, char* stage, const StageHeader& L, int64_t rb,
                        const RowSched& rs, const int64_t* rp, const uint32_t* pj, const uint32_t* pk,
                        const BwArgs& b, cudaStream_t s) {
  switch (ham->W) {
    case 1: launch_bw<Pol, 1, CX, LOAD_H>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s); break;
    case 2: launch_bw<Pol, 2, CX, LOAD_H>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s); break;
    case 3: launch_bw<Pol, 3, CX, LOAD_H>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s); break;
    default: launch_bw<Pol, 4, CX, LOAD_H>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s); break;
  }
}

template <class Pol>
static void launch_bw_p(const nqs_ham* ham, const uint64_t* U, char* stage, const StageHeader& L, bool cplx,
                        int64_t rb, const RowSched& rs, const int64_t* rp, const uint32_t* pj, const uint32_t* pk,
                        const BwArgs& b, cudaStream_t s) {
  if (ham->cplx) {
    if (b.hpair) launch_bw_w<Pol, kCplxH, true>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s);
    else launch_bw_w<Pol, kCplxH, false>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s);
  } else if (cplx) {
    if (b.hpair) launch_bw_w<Pol, kCplxPsi, true>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s);
    else launch_bw_w<Pol, kCplxPsi, false>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s);
  } else {
    if (b.hpair) launch_bw_w<Pol, kReal, true>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s);
    else launch_bw_w<Pol, kReal, false>(ham, U, stage, L, rb, rs, rp, pj, pk, b, s);
  }
}

cudaError_t launch_backward(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                            const StageHeader& L, bool cplx, const double* a, const double*,
                            int64_t rb, int64_t re, const int64_t* rp, const uint32_t* pj,
                            const uint32_t* pk, const double* er, const double* ei, const double* hd,
                            const double* evar, const double* g_re, const double* g_im,
                            const double* g_evar, int precision, const void* hpair, double* gre,
                            double* gim, cudaStream_t s) {
  const int64_t rows = re - rb;
  if (rows <= 0) return cudaSuccess;
  if (!g_re && !g_im) {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, 8 * num_sms()));
    backward_closed_kernel<<<blocks, 256, 0, s>>>(rb, re, a, er, ei, evar, g_evar, gre, gim);
    return cudaGetLastError();
  }
  const bool fp64 = precision == NQS_PREC_FP64;
  {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * num_sms()));
    geff_kernel<<<blocks, 256, 0, s>>>(n, a, evar, g_re, g_im, g_evar, fp64 ? 1 : 0,
                                       (double2*)(stage + L.off_geff), (float4*)(stage + L.off_geff), rb, re, er,
                                       ei, hd, (double2*)(stage + L.off_own), stage + L.off_ampQ);
  }
  RowSched rs;
  cudaError_t e = launch_row_order(rp, rows, stage, L, rs, s);
  if (e != cudaSuccess) return e;
  const BwArgs b{(const double2*)(stage + L.off_own), gre, gim, hpair};
  if (fp64) launch_bw_p<PolicyD>(ham, U, stage, L, cplx, rb, rs, rp, pj, pk, b, s);
  else launch_bw_p<PolicyF>(ham, U, stage, L, cplx, rb, rs, rp, pj, pk, b, s);
  return cudaGetLastError();
}


// --------------------------------------------------------------------------
// Half-stored pairs (i < j form): each unordered coupled pair {x_i, x_j} is
// one record (i, j, k).  Its matrix element is evaluated once and both rows
// receive their terms by FP64 atomic addition (symmetric scatter):
//   E_loc(i) += H_ij psi(j)/psi(i),   E_loc(j) += H_ji psi(i)/psi(j),
// with H_ji = conj(H_ij) (H Hermitian).  The diagonal is set first, one warp
// per sample.  Atomic addition makes the summation order, and so the last
// bits of a row's sum, depend on thread timing; the per-pair terms are the
// CSR path's to the bit.
// --------------------------------------------------------------------------
template <class Pol, int W>
__global__ void __launch_bounds__(kEnergyThreads)
half_diag_kernel(const uint64_t* __restrict__ U, const Melem M, int64_t n, double* __restrict__ er,
                 double* __restrict__ ei, double* __restrict__ hd) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kEnergyWarps;
  for (int64_t i = blockIdx.x * (int64_t)kEnergyWarps + (threadIdx.x >> 5); i < n; i += nw) {
    double h = 0.0;
    if (M.has_diag) {
      uint64_t x[W];
      load_words<W>(U + i * W, x);
      h = Pol::to_d(melem_diag<Pol, W>(x, M));
    }
    if (lane == 0) {
      er[i] = h;
      if (ei) ei[i] = 0.0;
      if (hd) hd[i] = h;
    }
  }
}

// H_ij of the record held by this lane (x' = U_j, pattern k): heavy term-form
// patterns by the whole warp, the rest by the lane
template <class Pol, int W, int CX>
__device__ __forceinline__ void half_melem(const uint64_t* __restrict__ U, const Melem& M, bool have, uint32_t j,
                                           uint32_t k, typename Pol::T& h, typename Pol::T& h_im) {
  using T = typename Pol::T;
  const int lane = threadIdx.x & 31;
  const int4 fm = have ? __ldg(M.fm + k) : make_int4(0, 0, 0, 0);
  const bool coop = have && (int64_t)k < M.heavy_end && (fm.x & 15) == kForm::Terms;
  h = Pol::zero();
  h_im = Pol::zero();
  uint32_t hb = __ballot_sync(kFull, coop);
  while (hb) {
    const int src = __ffs(hb) - 1;
    hb &= hb - 1;
    const uint32_t jj = __shfl_sync(kFull, j, src);
    const uint32_t kk = __shfl_sync(kFull, k, src);
    uint64_t xp[W];
    load_words<W>(U + (int64_t)jj * W, xp);
    const int64_t t0 = (int64_t)__ldg(M.t_ptr + kk), t1 = (int64_t)__ldg(M.t_ptr + kk + 1);
    if (CX == kCplxH) {
      T hwr, hwi;
      melem_warp_c<Pol, W>(xp, t0, t1, M, hwr, hwi);
      if (lane == src) { h = hwr; h_im = hwi; }
    } else {
      const T hw = melem_warp<Pol, W>(xp, t0, t1, M);
      if (lane == src) h = hw;
    }
  }
  if (have && !coop) {
    uint64_t xp[W];
    load_words<W>(U + (int64_t)j * W, xp);
    if (CX == kCplxH) melem_lane_c<Pol, W>(xp, k, fm, M, h, h_im);
    else h = melem_lane<Pol, W>(xp, k, fm, M);
  }
}

// the two terms of a record: t_i = H_ij psi(j)/psi(i) and t_j = conj(H_ij) psi(i)/psi(j)
template <class Pol, int CX>
__device__ __forceinline__ void half_terms(const char* P, const char* Q, int64_t i, int64_t j, typename Pol::T h,
                                           typename Pol::T h_im, int32_t* status, double& ir, double& ii,
                                           double& jr, double& ji) {
  using T = typename Pol::T;
  T rr, ri, sr, si;
  ratio<Pol, CX != kReal>(P, Q, j, i, rr, ri, status);   // psi(j)/psi(i)
  ratio<Pol, CX != kReal>(P, Q, i, j, sr, si, status);   // psi(i)/psi(j)
  if (CX == kCplxH) {
    ir = Pol::to_d(Pol::add(Pol::mul(h, rr), Pol::neg(Pol::mul(h_im, ri))));
    ii = Pol::to_d(Pol::add(Pol::mul(h, ri), Pol::mul(h_im, rr)));
    jr = Pol::to_d(Pol::add(Pol::mul(h, sr), Pol::mul(h_im, si)));
    ji = Pol::to_d(Pol::add(Pol::mul(h, si), Pol::neg(Pol::mul(h_im, sr))));
  } else {
    ir = Pol::to_d(Pol::mul(h, rr));
    jr = Pol::to_d(Pol::mul(h, sr));
    ii = CX == kCplxPsi ? Pol::to_d(Pol::mul(h, ri)) : 0.0;
    ji = CX == kCplxPsi ? Pol::to_d(Pol::mul(h, si)) : 0.0;
  }
}

__device__ __forceinline__ bool half_record(const uint32_t* __restrict__ ri, const uint32_t* __restrict__ rj,
                                            const uint32_t* __restrict__ rk, int64_t s, int64_t n_slots,
                                            const Melem& M, int32_t* status, uint32_t& i, uint32_t& j,
                                            uint32_t& k) {
  i = s < n_slots ? __ldg(ri + s) : kNoRecordSlot;
  if (i == kNoRecordSlot) return false;
  j = __ldg(rj + s);
  k = __ldg(rk + s);
  const bool ok = (int64_t)i < M.n_unq && pair_in_range(M, j, k, status);
  if (!ok && (int64_t)i >= M.n_unq) atomicOr(status, kStatusLimit);
  return ok;
}

template <class Pol, int W, int CX, bool STORE_H>
__global__ void __launch_bounds__(kEnergyThreads)
half_energy_kernel(const uint64_t* __restrict__ U, const Melem M, const char* __restrict__ P,
                   const char* __restrict__ Q, const uint32_t* __restrict__ ri, const uint32_t* __restrict__ rj,
                   const uint32_t* __restrict__ rk, int64_t n_slots, double* __restrict__ er,
                   double* __restrict__ ei, void* __restrict__ hrec, int32_t* __restrict__ status) {
  using T = typename Pol::T;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * kEnergyThreads;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; b < n_slots; b += stride) {
    const int64_t s = b + lane;
    uint32_t i = 0, j = 0, k = 0;
    const bool have = half_record(ri, rj, rk, s, n_slots, M, status, i, j, k);
    T h, h_im;
    half_melem<Pol, W, CX>(U, M, have, j, k, h, h_im);
    if (!have) continue;
    double a_r, a_i, b_r, b_i;
    half_terms<Pol, CX>(P, Q, i, j, h, h_im, status, a_r, a_i, b_r, b_i);
    atomicAdd(er + i, a_r);
    atomicAdd(er + j, b_r);
    if (CX != kReal) {
      atomicAdd(ei + i, a_i);
      atomicAdd(ei + j, b_i);
    }
    if (STORE_H) {
      if (CX == kCplxH) HStore<Pol>::put2(hrec, s, h, h_im);
      else HStore<Pol>::put(hrec, s, h);
    }
  }
}

template <class Pol, int W, int CX, bool STORE_H>
static void launch_half_le(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage, const StageHeader& L,
                           const uint32_t* ri, const uint32_t* rj, const uint32_t* rk, int64_t n_slots, double* er,
                           double* ei, void* hrec, cudaStream_t s) {
  const Melem M = melem_tables(ham, n);
  auto kern = half_energy_kernel<Pol, W, CX, STORE_H>;
  const int64_t warps = (n_slots + 31) / 32;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((warps + kEnergyWarps - 1) / kEnergyWarps,
                                                                  (int64_t)grid_for(kern, INT64_MAX / 2)));
  kern<<<blocks, kEnergyThreads, 0, s>>>(U, M, stage + L.off_ampP, stage + L.off_ampQ, ri, rj, rk, n_slots, er, ei,
                                         hrec, (int32_t*)(stage + offsetof(StageHeader, status)));
}

template <class Pol, int CX, bool STORE_H>
static void launch_half_le_w(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage,
                             const StageHeader& L, const uint32_t* ri, const uint32_t* rj, const uint32_t* rk,
                             int64_t n_slots, double* er, double* ei, double* hd, void* hrec, cudaStream_t s) {
  const Melem M = melem_tables(ham, n);
  const int db = (int)std::max<int64_t>(1, std::min<int64_t>((n + kEnergyWarps - 1) / kEnergyWarps, 8 * num_sms()));
  switch (ham->W) {
    case 1: half_diag_kernel<Pol, 1><<<db, kEnergyThreads, 0, s>>>(U, M, n, er, ei, hd);
            launch_half_le<Pol, 1, CX, STORE_H>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hrec, s); break;
    case 2: half_diag_kernel<Pol, 2><<<db, kEnergyThreads, 0, s>>>(U, M, n, er, ei, hd);
            launch_half_le<Pol, 2, CX, STORE_H>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hrec, s); break;
    case 3: half_diag_kernel<Pol, 3><<<db, kEnergyThreads, 0, s>>>(U, M, n, er, ei, hd);
            launch_half_le<Pol, 3, CX, STORE_H>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hrec, s); break;
    default: half_diag_kernel<Pol, 4><<<db, kEnergyThreads, 0, s>>>(U, M, n, er, ei, hd);
             launch_half_le<Pol, 4, CX, STORE_H>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hrec, s); break;
  }
}

template <class Pol>
static void launch_half_le_p(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage,
                             const StageHeader& L, bool cplx, const uint32_t* ri, const uint32_t* rj,
                             const uint32_t* rk, int64_t n_slots, double* er, double* ei, double* hd, void* hrec,
                             cudaStream_t s) {
  if (ham->cplx) {
    if (hrec) launch_half_le_w<Pol, kCplxH, true>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hd, hrec, s);
    else launch_half_le_w<Pol, kCplxH, false>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hd, hrec, s);
  } else if (cplx) {
    if (hrec) launch_half_le_w<Pol, kCplxPsi, true>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hd, hrec, s);
    else launch_half_le_w<Pol, kCplxPsi, false>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hd, hrec, s);
  } else {
    if (hrec) launch_half_le_w<Pol, kReal, true>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hd, hrec, s);
    else launch_half_le_w<Pol, kReal, false>(ham, U, n, stage, L, ri, rj, rk, n_slots, er, ei, hd, hrec, s);
  }
}

cudaError_t launch_local_energy_half(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage,
                                     const StageHeader& L, bool cplx, const uint32_t* ri, const uint32_t* rj,
                                     const uint32_t* rk, int64_t n_slots, int precision, double* er, double* ei,
                                     double* hd, void* hrec, cudaStream_t s) {
  if (precision == NQS_PREC_FP64)
    launch_half_le_p<PolicyD>(ham, U, n, stage, L, cplx, ri, rj, rk, n_slots, er, ei, hd, hrec, s);
  else
    launch_half_le_p<PolicyF>(ham, U, n, stage, L, cplx, ri, rj, rk, n_slots, er, ei, hd, hrec, s);
  return cudaGetLastError();
}

// Adjoint over half-stored records.  The row terms of the CSR adjoint, for a
// record (i, j): row j gets ge(i) Re T + gi(i) Im T (and -ge(i) Im T + gi(i) Re T
// for Im log psi) with T = H_ij psi(j)/psi(i), row i the same with the roles
// of i and j swapped and T = conj(H_ij) psi(i)/psi(j).  The rows' own terms
// (geff_kernel) initialise the gradient.
__global__ void half_grad_init_kernel(int64_t n, const double2* __restrict__ own, double* __restrict__ gre,
                                      double* __restrict__ gim) {
  for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < n; y += (int64_t)gridDim.x * blockDim.x) {
    const double2 o = own[y];
    gre[y] = o.x;
    if (gim) gim[y] = o.y;
  }
}

template <class Pol, int W, int CX, bool LOAD_H>
__global__ void __launch_bounds__(kEnergyThreads)
half_backward_kernel(const uint64_t* __restrict__ U, const Melem M, const char* __restrict__ P,
                     const char* __restrict__ Q, const char* __restrict__ G, const uint32_t* __restrict__ ri,
                     const uint32_t* __restrict__ rj, const uint32_t* __restrict__ rk, int64_t n_slots,
                     const void* __restrict__ hrec, double* __restrict__ gre, double* __restrict__ gim,
                     int32_t* __restrict__ status) {
  using T = typename Pol::T;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * kEnergyThreads;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; b < n_slots; b += stride) {
    const int64_t s = b + lane;
    uint32_t i = 0, j = 0, k = 0;
    const bool have = half_record(ri, rj, rk, s, n_slots, M, status, i, j, k);
    T h = Pol::zero(), h_im = Pol::zero();
    if (LOAD_H) {
      if (have) {
        if (CX == kCplxH) HStore<Pol>::get2(hrec, s, h, h_im);
        else h = HStore<Pol>::get(hrec, s);
      }
    } else {
      half_melem<Pol, W, CX>(U, M, have, j, k, h, h_im);
    }
    if (!have) continue;
    double a_r, a_i, b_r, b_i;   // T_ij (row j's term) and T_ji (row i's term)
    half_terms<Pol, CX>(P, Q, i, j, h, h_im, status, a_r, a_i, b_r, b_i);
    T gei, gii, gej, gij;
    Pol::load_v(G, i, gei, gii);
    Pol::load_v(G, j, gej, gij);
    const double ge_i = Pol::to_d(gei), gi_i = Pol::to_d(gii), ge_j = Pol::to_d(gej), gi_j = Pol::to_d(gij);
    atomicAdd(gre + j, ge_i * a_r + gi_i * a_i);
    atomicAdd(gre + i, ge_j * b_r + gi_j * b_i);
    if (gim) {
      atomicAdd(gim + j, -ge_i * a_i + gi_i * a_r);
      atomicAdd(gim + i, -ge_j * b_i + gi_j * b_r);
    }
  }
}

template <class Pol, int CX, bool LOAD_H>
static void launch_half_bw_w(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage, const StageHeader& L,
                             const uint32_t* ri, const uint32_t* rj, const uint32_t* rk, int64_t n_slots,
                             const void* hrec, double* gre, double* gim, cudaStream_t s) {
  const Melem M = melem_tables(ham, n);
  const int64_t warps = (n_slots + 31) / 32;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((warps + kEnergyWarps - 1) / kEnergyWarps,
                                                                  (int64_t)8 * num_sms()));
  int32_t* status = (int32_t*)(stage + offsetof(StageHeader, status));
#define NQS_HALF_BW(WW)                                                                                          \
  half_backward_kernel<Pol, WW, CX, LOAD_H><<<blocks, kEnergyThreads, 0, s>>>(                                    \
      U, M, stage + L.off_ampP, stage + L.off_ampQ, stage + L.off_geff, ri, rj, rk, n_slots, hrec, gre, gim, status)
  switch (ham->W) {
    case 1: NQS_HALF_BW(1); break;
    case 2: NQS_HALF_BW(2); break;
    case 3: NQS_HALF_BW(3); break;
    default: NQS_HALF_BW(4); break;
  }
#undef NQS_HALF_BW
}

cudaError_t launch_backward_half(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                                 const StageHeader& L, bool cplx, const double* a, const uint32_t* ri,
                                 const uint32_t* rj, const uint32_t* rk, int64_t n_slots, const void* hrec,
                                 const double* er, const double* ei, const double* hd, const double* evar,
                                 const double* g_re, const double* g_im, const double* g_evar, int precision,
                                 double* gre, double* gim, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * num_sms()));
  if (!g_re && !g_im) {
    backward_closed_kernel<<<blocks, 256, 0, s>>>(0, n, a, er, ei, evar, g_evar, gre, gim);
    return cudaGetLastError();
  }
  const bool fp64 = precision == NQS_PREC_FP64;
  geff_kernel<<<blocks, 256, 0, s>>>(n, a, evar, g_re, g_im, g_evar, fp64 ? 1 : 0, (double2*)(stage + L.off_geff),
                                     (float4*)(stage + L.off_geff), 0, n, er, ei, hd, (double2*)(stage + L.off_own),
                                     nullptr);
  half_grad_init_kernel<<<blocks, 256, 0, s>>>(n, (const double2*)(stage + L.off_own), gre, gim);
  const int cx = ham->cplx ? kCplxH : (cplx ? kCplxPsi : kReal);
#define NQS_HALF_BW_P(POL)                                                                                        \
  if (cx == kCplxH) {                                                                                             \
    if (hrec) launch_half_bw_w<POL, kCplxH, true>(ham, U, n, stage, L, ri, rj, rk, n_slots, hrec, gre, gim, s);   \
    else launch_half_bw_w<POL, kCplxH, false>(ham, U, n, stage, L, ri, rj, rk, n_slots, hrec, gre, gim, s);       \
  } else if (cx == kCplxPsi) {                                                                                    \
    if (hrec) launch_half_bw_w<POL, kCplxPsi, true>(ham, U, n, stage, L, ri, rj, rk, n_slots, hrec, gre, gim, s); \
    else launch_half_bw_w<POL, kCplxPsi, false>(ham, U, n, stage, L, ri, rj, rk, n_slots, hrec, gre, gim, s);     \
  } else {                                                                                                        \
    if (hrec) launch_half_bw_w<POL, kReal, true>(ham, U, n, stage, L, ri, rj, rk, n_slots, hrec, gre, gim, s);    \
    else launch_half_bw_w<POL, kReal, false>(ham, U, n, stage, L, ri, rj, rk, n_slots, hrec, gre, gim, s);        \
  }
  if (fp64) {
    NQS_HALF_BW_P(PolicyD)
  } else {
    NQS_HALF_BW_P(PolicyF)
  }
#undef NQS_HALF_BW_P
  return cudaGetLastError();
}


}  // namespace nqs

extern "C" int nqs_variational_energy_noalloc(int64_t n, const double* a, const double* eloc_re,
                                              double* out, void* stream) {
  using namespace nqs;
  if (n <= 0 || !a || !eloc_re || !out) return fail(NQS_ERR_ARG, "bad argument");
  if (n > kStaticRedMax)
    return fail(NQS_ERR_CAPACITY, "n_unq exceeds the 2097152-sample limit of the built-in scratch; "
                                  "use nqs_variational_energy with a workspace");
  void* base = nullptr;
  cudaError_t e = evar_scratch_address(&base);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (E^var scratch)");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int* done = (unsigned int*)base;
  double* part = (double*)((char*)base + 256);
  e = cudaMemsetAsync(done, 0, sizeof(unsigned int), s);  // the completion counter starts at zero
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (E^var scratch)");
  const int G = (int)((n + kStaticRedChunk - 1) / kStaticRedChunk);
  evar_kernel<<<G, kRedThreads, 0, s>>>(n, a, eloc_re, done, part, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "E^var kernel");
  return NQS_OK;
}
