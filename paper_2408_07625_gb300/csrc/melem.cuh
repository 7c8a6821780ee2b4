// MatrixElement evaluation shared by the energy, adjoint and candidate kernels:
// per-sample amplitude records, the FP32-compensated and FP64 arithmetic
// policies, the amplitude ratio, and H_xx' in the pattern's evaluation form
// (supplementary algorithm "Calculating the Hamiltonian matrix element",
// Eq. pauli_melem, evaluated in exact regroupings chosen at load time).
#pragma once

#include "device_util.cuh"
#include "nqs_internal.cuh"

namespace nqs {

// A factor (P or Q, FP32 compensated or FP64, real and imaginary parts) with
// the sample's power-of-two exponent K in one 32-byte record (one L2
// sector): a pair's gather of P_j and K_j, or Q_j and K_j, is one request.
// Per-sample amplitude record (one 32-byte L2 sector): the factor, its power-of-two
// exponent, and the sample's first bit word (read with the factor by the energy
// kernel when N <= 64, so a pair's column costs one gather)
struct __align__(32) AmpF {
  float4 v;
  int k;
  int pad;
  uint64_t x0;
};
struct __align__(32) AmpD {
  double2 v;
  int k;
  int pad;
  uint64_t x0;
};
static_assert(sizeof(AmpF) == 32 && sizeof(AmpD) == 32, "one sector per amplitude record");

// --------------------------------------------------------------------------
// arithmetic policies: FP32 compensated (double-float) and FP64
// --------------------------------------------------------------------------
struct PolicyF {
  using T = df;
  static constexpr int kMaxExp = 100;
  __device__ static T zero() { return {0.f, 0.f}; }
  __device__ static T coef(const float2* cf, const double*, int64_t l, uint32_t par) {
    return df_signflip(__ldg(cf + l), par);
  }
  __device__ static T val(const float2* f, const double*, int64_t i) {
    const float2 v = __ldg(f + i);
    return {v.x, v.y};
  }
  __device__ static void acc(T& a, T t) { df_acc(a, t); }
  // exact addition of both parts to a fixed-point sum; false if a part is out of its range
  __device__ static bool fx(Fx& a, T t) { return fx_add(a, t.hi, t.lo); }
  __device__ static T add(T a, T b) { return df_add(a, b); }
  __device__ static T mul(T a, T b) { return df_mul(a, b); }
  __device__ static T neg(T a) { return df_neg(a); }
  __device__ static T scale(T a, int e) { return df_ldexp(a, e); }
  __device__ static T fin(T a) { return df_norm(a); }
  __device__ static T warp_sum(T a) { return nqs::warp_sum(df_norm(a)); }
  __device__ static double to_d(T a) { return df_to_double(a); }
  __device__ static T from_d(double v) { return df_from_double(v); }
  __device__ static void load_v(const char* G, int64_t i, T& re, T& im) {  // 16-byte (re, im) entries
    const float4 v = __ldg(reinterpret_cast<const float4*>(G) + i);
    re = {v.x, v.y};
    im = {v.z, v.w};
  }
  // the record's last 8 bytes as a value (the real adjoint weight in the records of 1/psi)
  __device__ static T load_slot(const char* R, int64_t i) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(R + 32 * i + 24));
    return {v.x, v.y};
  }
  __device__ static void load_amp(const char* P, int64_t i, T& re, T& im, int& k) {
    const AmpF* r = reinterpret_cast<const AmpF*>(P) + i;
    const float4 v = __ldg(&r->v);
    k = __ldg(&r->k);
    re = {v.x, v.y};
    im = {v.z, v.w};
  }
};

struct PolicyD {
  using T = double;
  static constexpr int kMaxExp = 1000;
  __device__ static T zero() { return 0.0; }
  __device__ static T coef(const float2*, const double* cd, int64_t l, uint32_t par) {
    return dsignflip(__ldg(cd + l), par);
  }
  __device__ static T val(const float2*, const double* d, int64_t i) { return __ldg(d + i); }
  __device__ static void acc(T& a, T t) { a += t; }
  __device__ static bool fx(Fx& a, T t) { return fx_add(a, t); }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T neg(T a) { return -a; }
  __device__ static T scale(T a, int e) { return a * pow2d(e); }  // |e| <= kMaxExp
  __device__ static T fin(T a) { return a; }
  __device__ static T warp_sum(T a) { return nqs::warp_sum(a); }
  __device__ static double to_d(T a) { return a; }
  __device__ static T from_d(double v) { return v; }
  __device__ static void load_v(const char* G, int64_t i, T& re, T& im) {  // 16-byte (re, im) entries
    const double2 v = __ldg(reinterpret_cast<const double2*>(G) + i);
    re = v.x;
    im = v.y;
  }
  __device__ static T load_slot(const char* R, int64_t i) {
    return __ldg(reinterpret_cast<const double*>(R + 32 * i + 24));
  }
  __device__ static void load_amp(const char* P, int64_t i, T& re, T& im, int& k) {
    const AmpD* r = reinterpret_cast<const AmpD*>(P) + i;
    const double2 v = __ldg(&r->v);
    k = __ldg(&r->k);
    re = v.x;
    im = v.y;
  }
};

// complex ratio psi(num) / psi(den) = P_num Q_den 2^{K_num - K_den}
template <class Pol, bool CPLX>
__device__ __forceinline__ void ratio(const char* P, const char* Q, int64_t num, int64_t den,
                                      typename Pol::T& rr, typename Pol::T& ri, int32_t* status) {
  using T = typename Pol::T;
  T pr, pi, qr, qi;
  int kn, kd;
  Pol::load_amp(P, num, pr, pi, kn);
  Pol::load_amp(Q, den, qr, qi, kd);
  int e = kn - kd;
  if (e > Pol::kMaxExp || e < -Pol::kMaxExp) {
    atomicOr(status, kStatusRange);
    e = e > 0 ? Pol::kMaxExp : -Pol::kMaxExp;
  }
  if (CPLX) {
    rr = Pol::add(Pol::mul(pr, qr), Pol::neg(Pol::mul(pi, qi)));
    ri = Pol::add(Pol::mul(pr, qi), Pol::mul(pi, qr));
    rr = Pol::scale(rr, e);
    ri = Pol::scale(ri, e);
  } else {
    rr = Pol::scale(Pol::mul(pr, qr), e);
    ri = Pol::zero();
  }
}

// MatrixElement tables of a Hamiltonian (device pointers)
struct Melem {
  const uint32_t* t_ptr;   // P_XY of pattern k: terms t_ptr[k] .. t_ptr[k+1]-1
  const uint64_t* yz;
  const float2* cf;
  const double* cd;
  int has_diag;
  int64_t heavy_end;
  const int4* fm;          // per pattern: {kind | nb << 4, table offset, mask offset, packed qubits}
  const int4* fmx;         // N <= 64: per pattern {fm, sign mask A (low, high)}, 32 bytes
  const float2* fv_f;
  const double* fv_d;
  const uint64_t* fz;
  int diag_quad;
  const float2* quad_f;
  const double* quad_d;
  int64_t n_xy;            // patterns (pair indices k are below it)
  int64_t n_unq;           // samples of the batch (pair columns j are below it)
  // imaginary parts of the coefficients and local tables (complex H: terms with odd |Y|)
  const float2* cf_im;
  const double* cd_im;
  const float2* fv_f_im;
  const double* fv_d_im;
};

inline Melem melem_tables(const nqs_ham* h, int64_t n_unq) {
  return Melem{h->row_ptr, h->yz, h->coef_f, h->coef, h->has_diag, h->heavy_end, h->fm, h->fmx,
               h->fv_f, h->fv_d, h->fz, h->diag_quad, h->quad_f, h->quad_d, h->n_xy, n_unq,
               h->coef_f_im, h->coef_im, h->fv_f_im, h->fv_d_im};
}

// A pair's column and pattern index lie in range by construction of the
// lists; one that does not (a list not built for this batch) is flagged
// and skipped instead of indexing outside the tables.
__device__ __forceinline__ bool pair_in_range(const Melem& M, uint32_t j, uint32_t k, int32_t* status) {
  const bool ok = (int64_t)j < M.n_unq && (int64_t)k < M.n_xy;
  if (!ok) atomicOr(status, kStatusLimit);
  return ok;
}

// The terms [t0, t1) of one pattern summed by the whole warp: lane t adds
// terms t0 + t, t0 + t + 32, ... in order, four loads in flight at a time;
// every lane runs the same number of steps (terms past t1 add nothing).
// Every lane returns the same value.
// N <= 64, local form with its sign mask at hand (from the pattern's 32-byte record)
template <class Pol>
__device__ __forceinline__ typename Pol::T melem_local1(uint64_t xp, int4 fm, uint64_t amask, const Melem& M) {
  const int nb = fm.x >> 4;
  uint32_t u = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < nb) u |= (uint32_t)((xp >> ((fm.w >> (8 * i)) & 255)) & 1ull) << i;
  const typename Pol::T h = Pol::val(M.fv_f, M.fv_d, (int64_t)fm.y + u);
  return (__popcll(xp & amask) & 1) ? Pol::neg(h) : h;
}

template <class Pol, int W>
__device__ __forceinline__ typename Pol::T melem_warp(const uint64_t (&xp)[W], int64_t t0, int64_t t1,
                                                       const Melem& M);

// H of one pair by one lane, in the pattern's form (fm = its descriptor):
// local (one table value) or the pattern's terms (loads of four terms in
// flight).
template <class Pol, int W>
__device__ __forceinline__ typename Pol::T melem_lane(const uint64_t (&xp)[W], uint32_t k, int4 fm,
                                                       const Melem& M) {
  using T = typename Pol::T;
  const int kind = fm.x & 15;
  if (kind == kForm::Local) {
    const int nb = fm.x >> 4;
    uint32_t u = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < nb) {
        const int q = (fm.w >> (8 * i)) & 255;
        u |= (uint32_t)((xp[q >> 6] >> (q & 63)) & 1ull) << i;
      }
    }
    const T h = Pol::val(M.fv_f, M.fv_d, (int64_t)fm.y + u);
    return parity_and<W>(xp, M.fz + (int64_t)fm.z * W) ? Pol::neg(h) : h;
  }
  T h = Pol::zero();
  const int64_t t0 = __ldg(M.t_ptr + k), t1 = __ldg(M.t_ptr + k + 1);
#pragma unroll 4
  for (int64_t l = t0; l < t1; ++l) Pol::acc(h, Pol::coef(M.cf, M.cd, l, parity_and<W>(xp, M.yz + l * W)));
  return Pol::fin(h);
}

template <class Pol, int W>
__device__ __forceinline__ typename Pol::T melem_warp(const uint64_t (&xp)[W], int64_t t0, int64_t t1,
                                                       const Melem& M) {
  using T = typename Pol::T;
  const int lane = threadIdx.x & 31;
  T h = Pol::zero();
  for (int64_t b = t0; b < t1; b += 4 * 32) {
    T c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t l = b + 32 * u + lane;
      c[u] = l < t1 ? Pol::coef(M.cf, M.cd, l, parity_and<W>(xp, M.yz + l * W)) : Pol::zero();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) Pol::acc(h, c[u]);
  }
  return Pol::warp_sum(h);
}

// H_xx by the whole warp: the quadratic form (lane t takes the occupied
// qubits r of rank t, t + 32, .. and adds b_r + sum_{s > r occupied} B_rs;
// the lanes work side by side) or the diagonal pattern's terms; every lane
// returns the same value.
template <class Pol, int W>
__device__ __forceinline__ typename Pol::T melem_diag(const uint64_t (&x)[W], const Melem& M) {
  using T = typename Pol::T;
  const int lane = threadIdx.x & 31;
  if (!M.diag_quad) return melem_warp<Pol, W>(x, (int64_t)__ldg(M.t_ptr), (int64_t)__ldg(M.t_ptr + 1), M);
  constexpr int NQ = 64 * W;
  T h = lane == 0 ? Pol::val(M.quad_f, M.quad_d, 0) : Pol::zero();
  int before = 0;  // occupied qubits in the words before w
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int cnt = __popcll(x[w]);
    for (int t = lane; t < before + cnt; t += 32) {  // this lane's occupied qubits in word w
      if (t < before) continue;
      const int n = t - before;                     // rank inside the word
      const uint32_t lo = (uint32_t)x[w], hi = (uint32_t)(x[w] >> 32);
      const int nlo = __popc(lo);
      const int b = n < nlo ? (int)__fns(lo, 0, n + 1) : 32 + (int)__fns(hi, 0, n - nlo + 1);
      const int r = 64 * w + b;
      Pol::acc(h, Pol::val(M.quad_f, M.quad_d, 1 + r));
      const int64_t row = 1 + NQ + (int64_t)r * NQ;
      const uint64_t above = b == 63 ? 0ull : (x[w] & (~0ull << (b + 1)));
#pragma unroll
      for (int w2 = w; w2 < W; ++w2)
        for (uint64_t u = (w2 == w) ? above : x[w2]; u; u &= u - 1)
          Pol::acc(h, Pol::val(M.quad_f, M.quad_d, row + 64 * w2 + (__ffsll((long long)u) - 1)));
    }
    before += cnt;
  }
  return Pol::warp_sum(h);
}

// Complex H (terms with an odd number of Y): the same forms with both parts.
// A term's coefficient h i^{|Y|} is real or imaginary; the sign
// (-1)^{|x' & YZ|} applies to both parts alike.
template <class Pol, int W>
__device__ __forceinline__ void melem_lane_c(const uint64_t (&xp)[W], uint32_t k, int4 fm, const Melem& M,
                                             typename Pol::T& hr, typename Pol::T& hi) {
  using T = typename Pol::T;
  const int kind = fm.x & 15;
  if (kind == kForm::Local) {
    const int nb = fm.x >> 4;
    uint32_t u = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < nb) {
        const int q = (fm.w >> (8 * i)) & 255;
        u |= (uint32_t)((xp[q >> 6] >> (q & 63)) & 1ull) << i;
      }
    }
    const T vr = Pol::val(M.fv_f, M.fv_d, (int64_t)fm.y + u);
    const T vi = Pol::val(M.fv_f_im, M.fv_d_im, (int64_t)fm.y + u);
    const bool neg = parity_and<W>(xp, M.fz + (int64_t)fm.z * W);
    hr = neg ? Pol::neg(vr) : vr;
    hi = neg ? Pol::neg(vi) : vi;
    return;
  }
  hr = Pol::zero();
  hi = Pol::zero();
  const int64_t t0 = __ldg(M.t_ptr + k), t1 = __ldg(M.t_ptr + k + 1);
#pragma unroll 2
  for (int64_t l = t0; l < t1; ++l) {
    const uint32_t par = parity_and<W>(xp, M.yz + l * W);
    Pol::acc(hr, Pol::coef(M.cf, M.cd, l, par));
    Pol::acc(hi, Pol::coef(M.cf_im, M.cd_im, l, par));
  }
  hr = Pol::fin(hr);
  hi = Pol::fin(hi);
}

template <class Pol, int W>
__device__ __forceinline__ void melem_warp_c(const uint64_t (&xp)[W], int64_t t0, int64_t t1, const Melem& M,
                                             typename Pol::T& hr, typename Pol::T& hi) {
  using T = typename Pol::T;
  const int lane = threadIdx.x & 31;
  T ar = Pol::zero(), ai = Pol::zero();
  for (int64_t b = t0; b < t1; b += 2 * 32) {
    T cr[2], ci[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t l = b + 32 * u + lane;
      const uint32_t par = l < t1 ? parity_and<W>(xp, M.yz + l * W) : 0u;
      cr[u] = l < t1 ? Pol::coef(M.cf, M.cd, l, par) : Pol::zero();
      ci[u] = l < t1 ? Pol::coef(M.cf_im, M.cd_im, l, par) : Pol::zero();
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      Pol::acc(ar, cr[u]);
      Pol::acc(ai, ci[u]);
    }
  }
  hr = Pol::warp_sum(ar);
  hi = Pol::warp_sum(ai);
}

}  // namespace nqs
