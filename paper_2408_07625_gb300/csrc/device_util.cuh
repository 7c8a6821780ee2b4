// Device helpers: bit-vector words, parities, compensated FP32 arithmetic,
// exact fixed-point sums, a block-wide bitonic sort.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nqs {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <int W>
__device__ __forceinline__ void load_words(const uint64_t* __restrict__ p, uint64_t (&v)[W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) v[w] = __ldg(p + w);
}

// parity of |x AND m| (the sign (-1)^{|x' & YZ|} of Eq. pauli_melem)
template <int W>
__device__ __forceinline__ uint32_t parity_and(const uint64_t (&x)[W], const uint64_t* __restrict__ m) {
  uint64_t t = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) t ^= x[w] & __ldg(m + w);
  return __popc((uint32_t)t ^ (uint32_t)(t >> 32)) & 1u;
}

// three bits of a 32-bit blocked Bloom word per key (the word itself from the
// low bits of the hash): for each 5-bit field f of the hash at bits 15, 20 and
// 25, bit f - 1 (mod 32), which a right rotation by f brings to bit 31
__device__ __forceinline__ uint32_t bloom_bits(uint32_t h) {
  return (1u << (((h >> 15) - 1u) & 31u)) | (1u << (((h >> 20) - 1u) & 31u)) | (1u << (((h >> 25) - 1u) & 31u));
}

// --------------------------------------------------------------------------
// double-float ("df"): value = hi + lo with |lo| <= ulp(hi)/2.
// Error-free transformations: Knuth's TwoSum and the FMA-based TwoProduct.
// --------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo);
  return fast_two_sum(s.hi, lo);
}

// accumulate a df term without renormalising (renormalise once at the end)
__device__ __forceinline__ void df_acc(df& acc, df t) {
  df s = two_sum(acc.hi, t.hi);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ df df_norm(df a) { return fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_from_double(double v) {
  float hi = __double2float_rn(v);
  float lo = __double2float_rn(v - (double)hi);
  return {hi, lo};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// a * 2^e for |e| <= 126: multiplication by the power of two built from its
// IEEE-754 exponent field (exact unless the product leaves the normal range)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ df df_ldexp(df a, int e) {
  const float s = pow2f(e);
  return {a.hi * s, a.lo * s};
}
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// flip the sign of both parts when bit is 1 (exact)
__device__ __forceinline__ df df_signflip(float2 c, uint32_t bit) {
  uint32_t m = bit << 31;
  return {__uint_as_float(__float_as_uint(c.x) ^ m), __uint_as_float(__float_as_uint(c.y) ^ m)};
}

__device__ __forceinline__ double dsignflip(double c, uint32_t bit) {
  return __longlong_as_double(__double_as_longlong(c) ^ ((unsigned long long)bit << 63));
}

// warp all-reduce (butterfly): every lane ends with the same, order-fixed value
__device__ __forceinline__ df warp_sum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df u;
    u.hi = __shfl_xor_sync(kFull, v.hi, o);
    u.lo = __shfl_xor_sync(kFull, v.lo, o);
    v = df_add(v, u);
  }
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// --------------------------------------------------------------------------
// Exact sums ("Fx"): a signed 128-bit integer counting units of 2^-64
// (64 integer bits with the sign, 64 fraction bits).  A float, double or
// double-float term is turned into a whole number of units (the magnitude's
// bits below one unit are cut off, so a term is off by less than 2^-64) and
// added exactly.  Integer addition is associative, so a sum of terms does not
// depend on their order, on how they are dealt to lanes or on the reduction
// tree: a row's E_loc^var is the same whatever order its pairs are listed in.
// A term of magnitude 2^55 or more is not taken; the add functions then
// return false and leave the sum alone.  The conversions are branch-free
// (selects only), so the lanes of a warp do not diverge on the terms' scales.
// --------------------------------------------------------------------------
struct Fx {
  unsigned long long lo;
  long long hi;
};

__device__ __forceinline__ Fx fx_zero() { return {0ull, 0ll}; }

__device__ __forceinline__ void fx_add(Fx& a, const Fx& b) {
  unsigned long long ahi = (unsigned long long)a.hi;
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(ahi) : "l"(b.lo), "l"((unsigned long long)b.hi));
  a.hi = (long long)ahi;
}

// a += (neg ? -1 : 1) * floor(v 2^t) units, t <= 63
__device__ __forceinline__ void fx_add_scaled(Fx& a, unsigned long long v, int t, bool neg) {
  const int tp = t > 0 ? t : 0;
  const int tn = t < 0 ? -t : 0;
  const unsigned long long up = v << tp;
  const unsigned long long uh = (v >> 1) >> (63 - tp);
  const unsigned long long dn = tn < 64 ? v >> tn : 0ull;
  const unsigned long long mask = neg ? ~0ull : 0ull;
  const unsigned long long lo = (t >= 0 ? up : dn) ^ mask;
  const unsigned long long hi = (t >= 0 ? uh : 0ull) ^ mask;
  unsigned long long ahi = (unsigned long long)a.hi;
  // a + ~x + 1 = a - x when neg
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(ahi) : "l"(lo), "l"(hi));
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(a.lo), "+l"(ahi) : "l"(neg ? 1ull : 0ull));
  a.hi = (long long)ahi;
}

// f = +-m 2^(e - 150), m < 2^24: +-(m 2^40) 2^(e - 126) units
__device__ __forceinline__ bool fx_add(Fx& a, float f) {
  const uint32_t u = __float_as_uint(f);
  const int e = (int)((u >> 23) & 0xFFu);
  if (e > 181) return false;
  const unsigned long long m = (u & 0x7FFFFFu) | (e ? 0x800000u : 0u);
  fx_add_scaled(a, m << 40, e - 126, (u >> 31) != 0u);
  return true;
}

// d = +-m 2^(e - 1075), m < 2^53: +-(m 2^11) 2^(e - 1022) units
__device__ __forceinline__ bool fx_add(Fx& a, double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((u >> 52) & 0x7FFull);
  if (e > 1077) return false;
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  fx_add_scaled(a, m << 11, e - 1022, (u >> 63) != 0ull);
  return true;
}

// a normalised double-float hi + lo (|lo| <= ulp(hi)/2, so lo's exponent is at
// least 24 below hi's) as one 64-bit magnitude on hi's scale: m_hi 2^40 plus
// or minus lo's mantissa shifted to that scale (at most 2^40); anything else
// (zero hi, a part out of order) is added part by part
__device__ __forceinline__ bool fx_add(Fx& a, float hi, float lo) {
  const uint32_t uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
  const int d = el - eh + 40;
  if (eh == 0 || eh > 181 || d > 16) return fx_add(a, hi) & fx_add(a, lo);
  const unsigned long long mh = (unsigned long long)((uh & 0x7FFFFFu) | 0x800000u) << 40;
  const unsigned long long ml = (ul & 0x7FFFFFu) | (el ? 0x800000u : 0u);
  const unsigned long long l = d >= 0 ? ml << d : (d > -64 ? ml >> (-d) : 0ull);
  const bool same = ((uh ^ ul) >> 31) == 0u;
  fx_add_scaled(a, same ? mh + l : mh - l, eh - 126, (uh >> 31) != 0u);
  return true;
}

// warp all-reduce: every lane ends with the exact sum
__device__ __forceinline__ Fx fx_warp_sum(Fx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Fx w;
    w.lo = __shfl_xor_sync(kFull, v.lo, o);
    w.hi = __shfl_xor_sync(kFull, v.hi, o);
    fx_add(v, w);
  }
  return v;
}

// the sum rounded once to the nearest double: the magnitude's leading 64
// bits, with a sticky bit for any lower ones, rounded by the conversion, then
// scaled by a power of two (exact)
__device__ __forceinline__ double fx_to_double(Fx a) {
  const bool neg = a.hi < 0;
  unsigned long long lo = a.lo, hi = (unsigned long long)a.hi;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  if ((hi | lo) == 0ull) return 0.0;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  unsigned long long top, rest;
  if (lz >= 64) {
    top = lo << (lz - 64);
    rest = 0ull;
  } else if (lz == 0) {
    top = hi;
    rest = lo;
  } else {
    top = (hi << lz) | (lo >> (64 - lz));
    rest = lo << lz;
  }
  top |= rest != 0ull ? 1ull : 0ull;
  // the magnitude is (top + a fraction) 2^(64 - lz) units of 2^-64, i.e. about top 2^-lz
  const double r = __ull2double_rn(top) * __longlong_as_double((long long)(1023 - lz) << 52);
  return neg ? -r : r;
}

// Bitonic sort of N elements (a power of two, N <= E * blockDim.x) by (key,
// payload) ascending (by key alone when PAY is false), E per thread: thread t
// holds elements E t .. E t + E - 1.  Partners within a thread are compared
// in registers, partners in another lane of the warp through shuffles, and
// only partners in another warp through shared memory (sk, sp: N entries).
// Warps whose elements all lie past N skip the comparisons (their partners
// lie past N too) but take part in every barrier.
template <int E, bool PAY, class Key>
__device__ __forceinline__ void block_bitonic(Key (&key)[E], int32_t (&pay)[E], int N, Key* sk, int32_t* sp) {
  const int tid = threadIdx.x;
  const bool live = E * 32 * (tid >> 5) < N;
  auto less = [&](Key ka, int32_t pa, Key kb, int32_t pb) {
    if (PAY) return ka < kb || (ka == kb && pa < pb);
    return ka < kb;
  };
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < 32 * E) {
        if (!live) continue;
        if (j < E) {
#pragma unroll
          for (int jj = 1; jj < E; jj <<= 1) {
            if (jj != j) continue;
#pragma unroll
            for (int u = 0; u < E; ++u) {
              const int w = u ^ jj;   // known at compile time: the arrays stay in registers
              if (w > u) {
                const int i = E * tid + u;
                if (((i & k) == 0) == less(key[w], pay[w], key[u], pay[u])) {
                  const Key tk = key[u];
                  key[u] = key[w];
                  key[w] = tk;
                  if (PAY) {
                    const int32_t tp = pay[u];
                    pay[u] = pay[w];
                    pay[w] = tp;
                  }
                }
              }
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < E; ++u) {
            const Key ok = __shfl_xor_sync(0xFFFFFFFFu, key[u], j / E);
            const int32_t op = PAY ? __shfl_xor_sync(0xFFFFFFFFu, pay[u], j / E) : 0;
            const int i = E * tid + u;
            const bool take_min = ((i & k) == 0) == ((i & j) == 0);
            if (take_min == less(ok, op, key[u], pay[u])) {
              key[u] = ok;
              if (PAY) pay[u] = op;
            }
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < E; ++u) {
          if (E * tid + u < N) {
            sk[E * tid + u] = key[u];
            if (PAY) sp[E * tid + u] = pay[u];
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < E; ++u) {
          const int i = E * tid + u;
          if (i < N) {
            const int l = i ^ j;
            const Key ok = sk[l];
            const int32_t op = PAY ? sp[l] : 0;
            const bool take_min = ((i & k) == 0) == ((i & j) == 0);
            if (take_min == less(ok, op, key[u], pay[u])) {
              key[u] = ok;
              if (PAY) pay[u] = op;
            }
          }
        }
        __syncthreads();
      }
    }
  }
}

}  // namespace nqs
