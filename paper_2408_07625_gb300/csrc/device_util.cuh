// Device helpers: bit-vector words, parities, compensated FP32 arithmetic, a
// block-wide bitonic sort.
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
