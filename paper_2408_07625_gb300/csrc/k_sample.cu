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
// The ordering is an LSD radix sort of 64-bit keys that order the doubles
// L~' descending, carrying the extension index; the Gumbel draws and the
// conditional log-probabilities are inputs (the ansatz is the caller's).
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <math_constants.h>

#include "nqs_internal.cuh"

namespace nqs {

constexpr int kSampleThreads = 256;

// sort key ordering doubles descending (NaN-free input); impossible extensions last
__device__ __forceinline__ uint64_t desc_key(double v) {
  if (v == 0.0) v = 0.0;   // -0 and +0 are one value
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const uint64_t asc = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
  return ~asc;
}

struct SampleScratch {
  uint64_t* keys[2];
  int32_t* idx[2];
  int32_t* hist;
  int32_t* partial;
  double* ext;                 // [2n][2]: l', L~' of every extension
  unsigned long long* valid;   // possible extensions
  int64_t bytes;
};

static inline int64_t a256s(int64_t v) { return (v + 255) & ~int64_t(255); }

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
  v.bytes = off;
  return v;
}

int64_t sample_scratch_bytes(int64_t n_parents) { return sample_scratch_view(nullptr, n_parents).bytes; }

// one thread per kept vector: both extensions, their sort keys and (l', L~')
__global__ void gumbel_extend_kernel(int64_t n, const double* __restrict__ pl, const double* __restrict__ plt,
                                     const double* __restrict__ logp, const double* __restrict__ G,
                                     uint64_t* __restrict__ keys, int32_t* __restrict__ idx, double* __restrict__ ext,
                                     unsigned long long* __restrict__ valid) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double l = pl[p], lt = plt[p];
    const double l0 = l + logp[2 * p], l1 = l + logp[2 * p + 1];
    const double L0 = l0 + G[2 * p], L1 = l1 + G[2 * p + 1];
    const double Z = fmax(L0, L1);
    const double lc[2] = {l0, l1}, L[2] = {L0, L1};
    int nv = 0;
#pragma unroll
    for (int xi = 0; xi < 2; ++xi) {
      const int64_t c = 2 * p + xi;
      idx[c] = (int32_t)c;
      if (lc[xi] == -CUDART_INF) {
        keys[c] = ~0ull;
        ext[2 * c] = -CUDART_INF;
        ext[2 * c + 1] = -CUDART_INF;
        continue;
      }
      double ltc = lt;
      if (L[xi] < Z) {
        const double v = (lt - Z) + log(expm1(Z - L[xi]));
        ltc = lt - (fmax(v, 0.0) + log1p(exp(-fabs(v))));
      }
      keys[c] = desc_key(ltc);
      ext[2 * c] = lc[xi];
      ext[2 * c + 1] = ltc;
      ++nv;
    }
    if (nv) atomicAdd(valid, (unsigned long long)nv);
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

cudaError_t launch_gumbel_level(int W, int level, int64_t n, const uint64_t* px, const double* pl, const double* plt,
                                const double* logp, const double* G, int64_t K, void* scratch, uint64_t* cx,
                                double* cl, double* clt, int64_t* n_out, cudaStream_t s) {
  SampleScratch sc = sample_scratch_view((char*)scratch, n);
  const int64_t m = 2 * n;
  const int sms = num_sms();
  cudaError_t e = cudaMemsetAsync(sc.valid, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  gumbel_extend_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((n + kSampleThreads - 1) / kSampleThreads,
                                                                     8 * sms)),
                         kSampleThreads, 0, s>>>(n, pl, plt, logp, G, sc.keys[0], sc.idx[0], sc.ext, sc.valid);
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

}  // namespace nqs
