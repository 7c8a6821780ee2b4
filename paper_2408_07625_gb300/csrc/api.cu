// C ABI entry points and host-side preparation (Sec. "Preparation", Fig. ham_prep).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "nqs_internal.cuh"

namespace nqs {

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }

int fail(int code, const std::string& msg) {
  g_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_error = std::string(what) + ": " + cudaGetErrorString(e);
  return NQS_ERR_CUDA;
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

static inline int64_t align256(int64_t v) { return (v + 255) & ~int64_t(255); }

static inline int64_t next_pow2(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

StageHeader stage_layout(const nqs_ham* ham, int64_t n) {
  StageHeader L;
  std::memset(&L, 0, sizeof(L));
  L.magic = kStageMagic;
  L.n_unq = n;
  L.W = ham->W;
  L.cap = next_pow2(std::max<int64_t>(n, 16));        // buckets of 4 slots, <= 1 key per bucket on average
  // one filter of all samples: about two keys per word, at most 128 KB (shared memory of the search)
  L.nwords = std::min<int64_t>(std::max<int64_t>(next_pow2(std::max<int64_t>(n / 2, 1)), 32), 32768);
  const int64_t n1 = std::max<int64_t>(n, 1);
  int64_t off = align256(kRedOffset + kRedBytes);
  L.off_hx = off;     off = align256(off + 4 * n1);
  L.off_table = off;  off = align256(off + 32 * L.cap);
  L.off_bloom = off;  off = align256(off + 4 * L.nwords);
  L.scan_blocks = (n1 + 1023) / 1024 + 1;
  L.off_scan = off;   off = align256(off + 8 * L.scan_blocks);
  L.off_ampP = off;   off = align256(off + 32 * n1);  // 32-byte records: factor and exponent
  L.off_ampQ = off;   off = align256(off + 32 * n1);
  L.off_geff = off;   off = align256(off + 16 * n1);
  L.off_own = off;    off = align256(off + 16 * n1);
  L.off_counters = off; off = align256(off + 256);
  L.off_q = off;      off = align256(off + 2 * 4 * 64 * kMaxWords);
  L.off_qrows = off;  off = align256(off + 4 * n1 * (int64_t)ham->n_qubits);
  L.off_big = off;    off = align256(off + 4 * n1);
  L.off_rowcur = off; off = align256(off + 8 * n1);
  L.off_trie = off;   off = align256(off + trie_bytes(ham->W, n));
  L.off_sched = off;  off = align256(off + 512);
  L.off_order = off;  off = align256(off + 4 * n1);
  L.total_bytes = off;
  return L;
}

// --------------------------------------------------------------------------
// Hamiltonian preparation
// --------------------------------------------------------------------------

static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static int popc_words(const uint64_t* v, int W) {
  int c = 0;
  for (int w = 0; w < W; ++w) c += __builtin_popcountll(v[w]);
  return c;
}

static bool words_less(const uint64_t* a, const uint64_t* b, int W) {
  for (int w = W - 1; w >= 0; --w)
    if (a[w] != b[w]) return a[w] < b[w];
  return false;
}

static bool words_equal(const uint64_t* a, const uint64_t* b, int W) {
  for (int w = 0; w < W; ++w)
    if (a[w] != b[w]) return false;
  return true;
}

template <typename T>
static int upload(T** dst, const std::vector<T>& src) {
  size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)dst, bytes);
  if (e != cudaSuccess) return fail(NQS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  if (!src.empty()) {
    e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (ham tables)");
  }
  return NQS_OK;
}

static void free_ham(nqs_ham* h) {
  if (!h) return;
  cudaFree(h->xy); cudaFree(h->row_ptr); cudaFree(h->yz); cudaFree(h->coef);
  cudaFree(h->coef_f); cudaFree(h->srch_hash); cudaFree(h->srch_id); cudaFree(h->srch_rec); cudaFree(h->hash_basis);
  cudaFree(h->xy_table); cudaFree(h->wmask); cudaFree(h->xy_trie); cudaFree(h->xy_hash); cudaFree(h->segs);
  cudaFree(h->fm); cudaFree(h->fmx); cudaFree(h->fv_d); cudaFree(h->fv_f); cudaFree(h->fz); cudaFree(h->quad_d);
  cudaFree(h->quad_f); cudaFree(h->coef_im); cudaFree(h->coef_f_im); cudaFree(h->fv_d_im); cudaFree(h->fv_f_im);
  delete h;
}

}  // namespace nqs

using namespace nqs;

extern "C" {

const char* nqs_last_error(void) { return g_error.c_str(); }
int nqs_version(void) { return NQS_VERSION; }

int nqs_search_timing(int on) {
  search_timing(on != 0);
  return NQS_OK;
}

int nqs_search_time(double* total_ms, int64_t* launches) {
  if (!total_ms || !launches) return fail(NQS_ERR_ARG, "null argument");
  cudaError_t e = search_time(total_ms, launches);
  if (e != cudaSuccess) return cuda_fail(e, "search timing events");
  return NQS_OK;
}

int nqs_probe_peaks(double* out, void* stream) {
  if (!out) return fail(NQS_ERR_ARG, "null argument");
  cudaError_t e = probe_peaks(out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "integer peak kernels");
  return NQS_OK;
}

int nqs_ham_load(int n_qubits, int64_t n_terms, const uint64_t* x_mask, const uint64_t* z_mask,
                 const double* coef, nqs_ham** out) {
  if (!out) return fail(NQS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1) return fail(NQS_ERR_ARG, "n_qubits must be >= 1");
  if (n_qubits > 64 * kMaxWords) return fail(NQS_ERR_UNSUPPORTED, "n_qubits > 256");
  if (n_terms < 0) return fail(NQS_ERR_ARG, "n_terms < 0");
  if (n_terms > 0 && (!x_mask || !z_mask || !coef)) return fail(NQS_ERR_ARG, "null term array");
  if (n_terms >= (int64_t(1) << 31)) return fail(NQS_ERR_UNSUPPORTED, "more than 2^31 terms");
  const int W = (n_qubits + 63) / 64;
  const int tail = n_qubits - 64 * (W - 1);
  const uint64_t tail_mask = tail == 64 ? ~0ull : ((1ull << tail) - 1);

  for (int64_t t = 0; t < n_terms; ++t) {
    if ((x_mask[t * W + W - 1] & ~tail_mask) || (z_mask[t * W + W - 1] & ~tail_mask))
      return fail(NQS_ERR_ARG, "term " + std::to_string(t) + " has bits >= n_qubits");
    if (!std::isfinite(coef[t])) return fail(NQS_ERR_ARG, "non-finite coefficient");
  }

  // merge identical (x, z) strings: stable sort keeps input order inside a key
  std::vector<int64_t> idx(n_terms);
  std::iota(idx.begin(), idx.end(), 0);
  auto key_less = [&](int64_t a, int64_t b) {
    const uint64_t* xa = x_mask + a * W; const uint64_t* xb = x_mask + b * W;
    if (!words_equal(xa, xb, W)) return words_less(xa, xb, W);
    return words_less(z_mask + a * W, z_mask + b * W, W);
  };
  std::stable_sort(idx.begin(), idx.end(), key_less);
  struct Merged { int64_t first; double h; };
  std::vector<Merged> merged;
  for (int64_t a = 0; a < n_terms;) {
    int64_t b = a;
    // Neumaier-compensated sum in input order
    double s = 0.0, c = 0.0;
    while (b < n_terms && words_equal(x_mask + idx[a] * W, x_mask + idx[b] * W, W) &&
           words_equal(z_mask + idx[a] * W, z_mask + idx[b] * W, W)) {
      double v = coef[idx[b]];
      double t = s + v;
      c += (std::fabs(s) >= std::fabs(v)) ? (s - t) + v : (v - t) + s;
      s = t;
      ++b;
    }
    double h = s + c;
    if (h != 0.0) merged.push_back({idx[a], h});
    a = b;
  }
  nqs_ham* h = new nqs_ham();
  // a string with an odd number of Y has an imaginary coefficient h i^{|Y|}: complex H
  for (auto& m : merged) {
    uint64_t y[kMaxWords];
    for (int w = 0; w < W; ++w) y[w] = x_mask[m.first * W + w] & z_mask[m.first * W + w];
    if (popc_words(y, W) & 1) h->cplx = 1;
  }
  h->n_qubits = n_qubits;
  h->W = W;
  cudaGetDevice(&h->device);

  // group by XY = x mask; classes: diagonal, heavy (|P_XY| > kHeavyTerms), light
  const int64_t M = (int64_t)merged.size();
  std::vector<int64_t> grp_start;
  for (int64_t a = 0; a < M; ++a) {
    if (a == 0 || !words_equal(x_mask + merged[a].first * W, x_mask + merged[a - 1].first * W, W))
      grp_start.push_back(a);
  }
  const int64_t G = (int64_t)grp_start.size();
  grp_start.push_back(M);
  std::vector<int> cls(G);
  for (int64_t g = 0; g < G; ++g) {
    const uint64_t* xg = x_mask + merged[grp_start[g]].first * W;
    int64_t sz = grp_start[g + 1] - grp_start[g];
    bool zero = true;
    for (int w = 0; w < W; ++w) zero = zero && xg[w] == 0;
    cls[g] = zero ? 0 : (sz > kHeavyTerms ? 1 : 2);
  }
  std::vector<int64_t> order(G);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cls[a] < cls[b]; });

  h->n_xy = G;
  h->n_terms = M;
  h->has_diag = (G > 0 && cls[order[0]] == 0) ? 1 : 0;
  h->heavy_end = h->has_diag;
  for (int64_t p = 0; p < G; ++p) if (cls[order[p]] == 1) h->heavy_end = p + 1;
  if (h->heavy_end < h->has_diag) h->heavy_end = h->has_diag;

  h->h_xy.assign(G * W, 0);
  h->h_row_ptr.assign(G + 1, 0);
  h->h_yz.assign(M * W, 0);
  h->h_coef.assign(M, 0.0);
  h->h_coef_im.assign(M, 0.0);
  std::vector<float2> coef_f(M), coef_f_im(M);
  int64_t t = 0;
  for (int64_t p = 0; p < G; ++p) {
    int64_t g = order[p];
    const uint64_t* xg = x_mask + merged[grp_start[g]].first * W;
    for (int w = 0; w < W; ++w) h->h_xy[p * W + w] = xg[w];
    h->h_row_ptr[p] = t;
    h->max_group = std::max<int64_t>(h->max_group, grp_start[g + 1] - grp_start[g]);
    for (int64_t a = grp_start[g]; a < grp_start[g + 1]; ++a, ++t) {
      const int64_t src = merged[a].first;
      uint64_t y[kMaxWords];
      for (int w = 0; w < W; ++w) {
        h->h_yz[t * W + w] = z_mask[src * W + w];
        y[w] = x_mask[src * W + w] & z_mask[src * W + w];
      }
      // <x|P|x'> = i^{|Y|} (-1)^{|x' & YZ|}: |Y| even -> i^{|Y|} = (-1)^{|Y|/2} (real),
      // |Y| odd -> i^{|Y|} = i (-1)^{(|Y|-1)/2} (imaginary)
      const int ny = popc_words(y, W);
      const double c = merged[a].h * (((ny / 2) & 1) ? -1.0 : 1.0);
      double& dst = (ny & 1) ? h->h_coef_im[t] : h->h_coef[t];
      dst = c;
      float hi = (float)c;
      float lo = (float)(c - (double)hi);
      ((ny & 1) ? coef_f_im[t] : coef_f[t]) = make_float2(hi, lo);
    }
  }
  h->h_row_ptr[G] = t;

  // MatrixElement forms.  Each regroups the sum of Eq. pauli_melem exactly;
  // coefficients are summed with Neumaier compensation in a fixed order.
  //   local: YZ_l = A XOR B_l with B_l inside the pattern's qubits, so
  //     c (-1)^{x'.YZ_l} = c (-1)^{x'.A} (-1)^{u.B_l}, u = x' on those qubits;
  //   quadratic diagonal: every diagonal term a Z string on at most two
  //     qubits: c (-1)^{x_r + x_s} = c (1 - 2 x_r)(1 - 2 x_s).
  struct CSum {
    double s = 0.0, c = 0.0;
    void add(double v) {
      const double t = s + v;
      c += (std::fabs(s) >= std::fabs(v)) ? (s - t) + v : (v - t) + s;
      s = t;
    }
    double value() const { return s + c; }
  };
  const int NQ = 64 * W;
  std::vector<int4> fm(G, make_int4(kForm::Terms, 0, 0, 0));
  std::vector<double> fv, fv_im;   // real and imaginary parts of the local tables
  std::vector<uint64_t> fz;
  for (int64_t p = h->has_diag; p < G; ++p) {
    const int64_t t0 = h->h_row_ptr[p], t1 = h->h_row_ptr[p + 1];
    const uint64_t* xy = &h->h_xy[p * W];
    const int nb = popc_words(xy, W);
    // local: every YZ_l agrees with YZ_0 outside XY
    bool local = nb <= 4;
    for (int64_t t = t0; t < t1 && local; ++t)
      for (int w = 0; w < W; ++w)
        if ((h->h_yz[t * W + w] ^ h->h_yz[t0 * W + w]) & ~xy[w]) local = false;
    if (local) {
      int q[4], n = 0;
      for (int w = 0; w < W; ++w)
        for (uint64_t m = xy[w]; m; m &= m - 1) q[n++] = 64 * w + __builtin_ctzll(m);
      uint32_t packed = 0;
      for (int i = 0; i < nb; ++i) packed |= (uint32_t)q[i] << (8 * i);
      std::vector<CSum> T(1u << nb), Ti(1u << nb);
      for (int64_t t = t0; t < t1; ++t) {
        uint32_t bl = 0;  // YZ_l on the pattern's qubits, compressed
        for (int i = 0; i < nb; ++i) bl |= (uint32_t)((h->h_yz[t * W + q[i] / 64] >> (q[i] % 64)) & 1ull) << i;
        for (uint32_t u = 0; u < (1u << nb); ++u) {
          const bool neg = __builtin_popcount(u & bl) & 1;
          if (h->h_coef[t] != 0.0) T[u].add(neg ? -h->h_coef[t] : h->h_coef[t]);
          if (h->h_coef_im[t] != 0.0) Ti[u].add(neg ? -h->h_coef_im[t] : h->h_coef_im[t]);
        }
      }
      fm[p] = make_int4(kForm::Local | (nb << 4), (int)fv.size(), (int)(fz.size() / W), (int)packed);
      for (auto& v : T) fv.push_back(v.value());
      for (auto& v : Ti) fv_im.push_back(v.value());
      for (int w = 0; w < W; ++w) fz.push_back(h->h_yz[t0 * W + w] & ~xy[w]);
      ++h->n_local;
    }
  }
  if (fv.size() >= (size_t)INT32_MAX || fz.size() / W >= (size_t)INT32_MAX) {
    std::fill(fm.begin(), fm.end(), make_int4(kForm::Terms, 0, 0, 0));  // tables too large to index
    fv.clear();
    fv_im.clear();
    fz.clear();
  }
  std::vector<int4> fmx;  // N <= 64: the descriptor and the local sign mask in one record
  if (W == 1) {
    fmx.resize(2 * (size_t)G);
    for (int64_t p = 0; p < G; ++p) {
      const uint64_t a = (fm[p].x & 15) == kForm::Local ? fz[(size_t)fm[p].z] : 0ull;
      fmx[2 * p] = fm[p];
      fmx[2 * p + 1] = make_int4((int)(uint32_t)a, (int)(uint32_t)(a >> 32), 0, 0);
    }
  }
  std::vector<double> quad_d;
  if (h->has_diag) {
    const int64_t t0 = h->h_row_ptr[0], t1 = h->h_row_ptr[1];
    std::vector<CSum> acc(1 + NQ + (size_t)NQ * NQ);
    bool ok = true;
    for (int64_t t = t0; t < t1 && ok; ++t) {
      int q[2], nq = 0;
      for (int w = 0; w < W && ok; ++w)
        for (uint64_t m = h->h_yz[t * W + w]; m; m &= m - 1) {
          if (nq == 2) { ok = false; break; }
          q[nq++] = 64 * w + __builtin_ctzll(m);
        }
      if (!ok) break;
      const double c = h->h_coef[t];
      acc[0].add(c);
      for (int u = 0; u < nq; ++u) acc[1 + q[u]].add(-2.0 * c);
      if (nq == 2) acc[1 + NQ + (size_t)q[0] * NQ + q[1]].add(4.0 * c);
    }
    if (ok) {
      h->diag_quad = 1;
      quad_d.resize(acc.size());
      for (size_t e = 0; e < acc.size(); ++e) quad_d[e] = acc[e].value();
    }
  }
  auto split = [](const std::vector<double>& v) {
    std::vector<float2> f(v.size());
    for (size_t e = 0; e < v.size(); ++e) {
      const float hi = (float)v[e];
      f[e] = make_float2(hi, (float)(v[e] - (double)hi));
    }
    return f;
  };
  const std::vector<float2> fv_f = split(fv), quad_f = split(quad_d), fv_f_im = split(fv_im);

  // linear hash basis: h(v) = XOR over set bits b of R[b] (GF(2)-linear, so
  // h(x ^ xy) = h(x) ^ h(xy) and a candidate's hash costs one XOR)
  h->h_hash_basis.resize(64 * W);
  uint64_t seed = 0x243F6A8885A308D3ull;
  for (int b = 0; b < 64 * W; ++b) h->h_hash_basis[b] = (uint32_t)(splitmix64(seed) >> 32);
  std::vector<uint32_t> hxy(G);
  for (int64_t p = 0; p < G; ++p) {
    uint32_t v = 0;
    for (int w = 0; w < W; ++w) {
      uint64_t m = h->h_xy[p * W + w];
      while (m) { int b = __builtin_ctzll(m); v ^= h->h_hash_basis[64 * w + b]; m &= m - 1; }
    }
    hxy[p] = v;
  }

  // search table of the oriented LoopOverTerms search: the non-diagonal
  // patterns grouped by their highest set qubit t (a pair {x, x'} with
  // x ^ x' = XY is searched from the one of the two with bit t set), one
  // segment per t, largest first.  A segment is cut into groups of 32 slots
  // holding at most two patterns per hash residue mod 32, so the 32 lanes of
  // a warp probing one sample touch each shared-memory bank of the
  // membership filter at most twice; short groups are padded with dummy slots.
  std::vector<uint32_t> srch_hash, srch_id;
  std::vector<uint64_t> srch_rec;
  h->rec_words = 2 * ((1 + W + 1) / 2);
  std::vector<std::vector<uint32_t>> by_top(64 * W);
  for (int64_t p = h->has_diag; p < G; ++p) {
    int top = -1;
    for (int w = W - 1; w >= 0 && top < 0; --w)
      if (h->h_xy[p * W + w]) top = 64 * w + 63 - __builtin_clzll(h->h_xy[p * W + w]);
    by_top[top].push_back((uint32_t)p);
  }
  std::vector<int> tord;
  for (int t = 0; t < 64 * W; ++t)
    if (!by_top[t].empty()) tord.push_back(t);
  std::stable_sort(tord.begin(), tord.end(), [&](int a, int b) { return by_top[a].size() > by_top[b].size(); });
  std::vector<int4> segs;
  for (int t : tord) {
    // striping the patterns, ordered by residue, over G groups puts at most
    // ceil(|residue class| / G) <= 2 of a residue into each group
    std::vector<uint32_t> pats = by_top[t];
    std::stable_sort(pats.begin(), pats.end(), [&](uint32_t a, uint32_t b) { return (hxy[a] & 31) < (hxy[b] & 31); });
    size_t maxb = 0;
    {
      size_t cnt[32] = {0};
      for (uint32_t p : pats) maxb = std::max(maxb, ++cnt[hxy[p] & 31]);
    }
    const size_t Gs = std::max((pats.size() + 31) / 32, (maxb + 1) / 2);
    std::vector<std::vector<uint32_t>> groups(Gs);
    for (size_t q = 0; q < pats.size(); ++q) groups[q % Gs].push_back(pats[q]);
    const int64_t g0 = (int64_t)srch_hash.size() / 32;
    for (auto& grp : groups) {
      for (int l = 0; l < 32; ++l) {
        if (l < (int)grp.size()) {
          const uint32_t id = grp[l];
          srch_hash.push_back(hxy[id]);
          srch_id.push_back(id);
          srch_rec.push_back((uint64_t)hxy[id] | ((uint64_t)id << 32));
          for (int w = 0; w < W; ++w) srch_rec.push_back(h->h_xy[(int64_t)id * W + w]);
          for (int w = 1 + W; w < h->rec_words; ++w) srch_rec.push_back(0);
        } else {
          const uint32_t dh = (uint32_t)l;
          srch_hash.push_back(dh);
          srch_id.push_back(kDummy);
          srch_rec.push_back((uint64_t)dh | ((uint64_t)kDummy << 32));
          for (int w = 1; w < h->rec_words; ++w) srch_rec.push_back(0);
        }
      }
    }
    segs.push_back(make_int4(t, (int)g0, (int)(srch_hash.size() / 32), 0));
  }
  h->n_segs = (int)segs.size();
  h->n_srch = (int64_t)srch_hash.size();

  // XY hash set for the batch schedule (Alg. 2B): same linear hash, so the
  // hash of x ^ x' is h(x) ^ h(x'); slot = W key words, then id | hash << 32
  h->xy_cap = 64;
  while (h->xy_cap < 2 * std::max<int64_t>(G, 1)) h->xy_cap <<= 1;
  std::vector<unsigned long long> xy_table((size_t)h->xy_cap * (W + 1), ~0ull);
  std::vector<unsigned long long> wmask(5, 0ull);
  for (int64_t p = 0; p < G; ++p) {
    int64_t slot = hxy[p] & (h->xy_cap - 1);
    while (xy_table[slot * (W + 1) + W] != ~0ull) slot = (slot + 1) & (h->xy_cap - 1);
    for (int w = 0; w < W; ++w) xy_table[slot * (W + 1) + w] = h->h_xy[p * W + w];
    xy_table[slot * (W + 1) + W] = (unsigned long long)p | ((unsigned long long)hxy[p] << 32);
    const int wt = popc_words(&h->h_xy[p * W], W);
    wmask[wt >> 6] |= 1ull << (wt & 63);
  }

  std::vector<uint32_t> rp32(G + 1);
  for (int64_t p = 0; p <= G; ++p) rp32[p] = (uint32_t)h->h_row_ptr[p];

  // prefix tree of the patterns for LoopOverTrie (Alg. 3)
  std::vector<int32_t> xy_nodes;
  build_xy_trie(h->h_xy, G, W, xy_nodes);
  h->n_xy_nodes = (int64_t)xy_nodes.size() / 4;
  std::vector<int4> xy_trie(h->n_xy_nodes);
  for (int64_t v = 0; v < h->n_xy_nodes; ++v)
    xy_trie[v] = make_int4(xy_nodes[4 * v], xy_nodes[4 * v + 1], xy_nodes[4 * v + 2], 0);

  int rc;
  if ((rc = upload(&h->xy, h->h_xy)) || (rc = upload(&h->row_ptr, rp32)) ||
      (rc = upload(&h->yz, h->h_yz)) || (rc = upload(&h->coef, h->h_coef)) ||
      (rc = upload(&h->coef_f, coef_f)) || (rc = upload(&h->srch_hash, srch_hash)) ||
      (rc = upload(&h->srch_id, srch_id)) || (rc = upload(&h->srch_rec, srch_rec)) ||
      (rc = upload(&h->hash_basis, h->h_hash_basis)) || (rc = upload(&h->xy_table, xy_table)) ||
      (rc = upload(&h->wmask, wmask)) || (rc = upload(&h->xy_trie, xy_trie)) ||
      (rc = upload(&h->xy_hash, hxy)) || (rc = upload(&h->segs, segs)) || (rc = upload(&h->fm, fm)) || (rc = upload(&h->fmx, fmx)) ||
      (rc = upload(&h->fv_d, fv)) || (rc = upload(&h->fv_f, fv_f)) || (rc = upload(&h->fz, fz)) ||
      (rc = upload(&h->quad_d, quad_d)) || (rc = upload(&h->quad_f, quad_f)) ||
      (rc = upload(&h->coef_im, h->h_coef_im)) || (rc = upload(&h->coef_f_im, coef_f_im)) ||
      (rc = upload(&h->fv_d_im, fv_im)) || (rc = upload(&h->fv_f_im, fv_f_im))) {
    free_ham(h);
    return rc;
  }
  *out = h;
  return NQS_OK;
}

int nqs_ham_free(nqs_ham* ham) {
  free_ham(ham);
  return NQS_OK;
}

int nqs_ham_info(const nqs_ham* h, int64_t info[8]) {
  if (!h || !info) return fail(NQS_ERR_ARG, "null argument");
  info[0] = h->n_qubits; info[1] = h->W; info[2] = h->n_terms; info[3] = h->n_xy;
  info[4] = h->has_diag; info[5] = h->max_group; info[6] = h->n_srch; info[7] = h->heavy_end;
  return NQS_OK;
}

int nqs_ham_is_complex(const nqs_ham* h) { return h ? h->cplx : 0; }

int nqs_ham_export_im(const nqs_ham* h, double* coef_im) {
  if (!h || !coef_im) return fail(NQS_ERR_ARG, "null argument");
  std::copy(h->h_coef_im.begin(), h->h_coef_im.end(), coef_im);
  return NQS_OK;
}

int nqs_ham_export(const nqs_ham* h, uint64_t* xy, int64_t* row_ptr, uint64_t* yz, double* coef) {
  if (!h) return fail(NQS_ERR_ARG, "null ham");
  if (xy) std::copy(h->h_xy.begin(), h->h_xy.end(), xy);
  if (row_ptr) std::copy(h->h_row_ptr.begin(), h->h_row_ptr.end(), row_ptr);
  if (yz) std::copy(h->h_yz.begin(), h->h_yz.end(), yz);
  if (coef) std::copy(h->h_coef.begin(), h->h_coef.end(), coef);
  return NQS_OK;
}

int64_t nqs_stage_bytes(const nqs_ham* ham, int64_t n_unq) {
  if (!ham || n_unq < 0) return fail(NQS_ERR_ARG, "bad argument to nqs_stage_bytes");
  return stage_layout(ham, n_unq).total_bytes;
}

static int status_to_code(int st) {
  if (st & kStatusDuplicate) return fail(NQS_ERR_DUPLICATE, "the sample batch repeats a basis vector");
  if (st & kStatusBadBits) return fail(NQS_ERR_ARG, "a sample has bits >= n_qubits");
  if (st & kStatusLimit)
    return fail(NQS_ERR_DEVICE_LIMIT, "a bounded device loop ran out or an index check skipped an access");
  if (st & kStatusRange)
    return fail(NQS_ERR_RANGE, "an amplitude ratio leaves the FP32 range or a local-energy term reaches 2^55");
  if (st & kStatusCapacity) return fail(NQS_ERR_CAPACITY, "a pair buffer sized at planning time was too small");
  if (st & kStatusNoTrie) return fail(NQS_ERR_ARG, "trie schedule without nqs_stage_trie after nqs_stage");
  return NQS_OK;
}

static int read_status(const void* work, cudaStream_t s, StageHeader* hdr_out = nullptr) {
  StageHeader hdr;
  cudaError_t e = cudaMemcpyAsync(&hdr, work, sizeof(hdr), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  if (hdr.magic != kStageMagic) return fail(NQS_ERR_ARG, "workspace was not staged");
  if (hdr_out) *hdr_out = hdr;
  return status_to_code(hdr.status);
}

static int check_work(const nqs_ham* ham, const uint64_t* U, int64_t n, const void* work, StageHeader* L) {
  if (!ham) return fail(NQS_ERR_ARG, "null ham");
  if (n < 0) return fail(NQS_ERR_ARG, "n_unq < 0");
  if (n > 0 && !U) return fail(NQS_ERR_ARG, "null U");
  if (n >= (int64_t(1) << 31)) return fail(NQS_ERR_UNSUPPORTED, "more than 2^31 samples");
  if (!work) return fail(NQS_ERR_ARG, "null workspace");
  if (((uintptr_t)work) & 255) return fail(NQS_ERR_ARG, "workspace not 256-byte aligned");
  *L = stage_layout(ham, n);
  return NQS_OK;
}

int nqs_stage(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, int64_t bytes,
              int check, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc) return rc;
  if (bytes < L.total_bytes) return fail(NQS_ERR_CAPACITY, "workspace smaller than nqs_stage_bytes");
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)work;
  // by a kernel, not a copy from this stack frame: a CUDA graph that captures
  // the call replays the write with the header's value
  cudaError_t e = launch_write_header(L, base, s);
  if (e != cudaSuccess) return cuda_fail(e, "header write");
  if ((e = cudaMemsetAsync(base + kRedOffset, 0, 256, s)) != cudaSuccess) return cuda_fail(e, "memset");
  if ((e = launch_stage(ham, U, n, base, L, s)) != cudaSuccess) return cuda_fail(e, "stage kernel");
  if (check) return read_status(work, s);
  return NQS_OK;
}

int nqs_stage_status(const void* work, void* stream) {
  if (!work) return fail(NQS_ERR_ARG, "null workspace");
  return read_status(work, (cudaStream_t)stream);
}

static int check_rows(int64_t n, int64_t rb, int64_t re) {
  if (rb < 0 || re < rb || re > n) return fail(NQS_ERR_ARG, "bad row range");
  return NQS_OK;
}

static int check_schedule(const nqs_ham* ham, int64_t n, int schedule) {
  if (schedule == NQS_SCHED_AUTO || schedule == NQS_SCHED_TERMS || schedule == NQS_SCHED_BATCH)
    return NQS_OK;
  if (schedule == NQS_SCHED_TRIE) {
    if (ham->n_qubits > 255) return fail(NQS_ERR_UNSUPPORTED, "trie schedule needs n_qubits <= 255");
    if (n >= (int64_t(1) << 23)) return fail(NQS_ERR_UNSUPPORTED, "trie schedule needs n_unq < 2^23");
    return NQS_OK;
  }
  return fail(NQS_ERR_ARG, "unknown schedule");
}

int nqs_stage_trie(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc || (rc = check_schedule(ham, n, NQS_SCHED_TRIE))) return rc;
  cudaError_t e = launch_trie_build(ham, U, n, (char*)work, L, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "prefix tree build");
  return NQS_OK;
}

// AUTO: LoopOverBatch costs ~N_unq^2 / 2 cheap pair tests, LoopOverTerms
// N_unq * |XY| filter probes; take the batch loop when it has fewer.
static int pick_schedule(const nqs_ham* ham, int64_t n, int schedule) {
  if (schedule != NQS_SCHED_AUTO) return schedule;
  return (n < ham->n_xy) ? NQS_SCHED_BATCH : NQS_SCHED_TERMS;
}

// The schedule argument of the pair calls carries NQS_ROWS_UNSORTED as a flag
// bit; split it off.
static int split_schedule(int schedule, bool* sorted) {
  *sorted = (schedule & NQS_ROWS_UNSORTED) == 0;
  return schedule & ~NQS_ROWS_UNSORTED;
}

static cudaError_t launch_search(const nqs_ham* ham, const uint64_t* U, int64_t n, char* work,
                                 const StageHeader& L, int64_t rb, int64_t re, int schedule,
                                 int64_t* rp, uint32_t* pj, uint32_t* pk, int mode,
                                 const PairScratch* sc, cudaStream_t s, bool sorted = true) {
  const int sched = pick_schedule(ham, n, schedule);
  if (sched == NQS_SCHED_BATCH)
    return launch_pairs_batch(ham, U, n, work, L, rb, re, rp, pj, pk, mode == kFill ? kFill : kCount, s);
  if (sched == NQS_SCHED_TRIE)
    return launch_pairs_trie(ham, U, n, work, L, rb, re, rp, pj, pk, mode == kFill ? kFill : kCount, s);
  SearchTune tune;
  tune.sort_rows = sorted;
  return launch_pairs_terms(ham, U, work, L, rb, re, rp, pj, pk, mode, sc, s, tune);
}

static int count_pass(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, const StageHeader& L,
                      int64_t rb, int64_t re, int schedule, int64_t* row_ptr, const PairScratch* sc,
                      cudaStream_t s) {
  const int64_t rows = re - rb;
  cudaError_t e = cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "memset row_ptr");
  if (rows > 0) {
    if ((e = launch_search(ham, U, n, (char*)work, L, rb, re, schedule, row_ptr + 1, nullptr, nullptr,
                           sc ? kEmit : kCount, sc, s)) != cudaSuccess)
      return cuda_fail(e, "pair search kernel");
    if ((e = launch_scan(row_ptr + 1, rows, (char*)work, L, s)) != cudaSuccess)
      return cuda_fail(e, "scan kernel");
  }
  return NQS_OK;
}

int nqs_count_coupled_pairs(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work,
                            int64_t rb, int64_t re, int schedule, int64_t* row_ptr,
                            int64_t* n_pairs, void* stream) {
  StageHeader L;
  bool sorted;
  schedule = split_schedule(schedule, &sorted);
  int rc = check_work(ham, U, n, work, &L);
  if (rc || (rc = check_rows(n, rb, re)) || (rc = check_schedule(ham, n, schedule))) return rc;
  if (!row_ptr || !n_pairs) return fail(NQS_ERR_ARG, "null row_ptr or n_pairs");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = count_pass(ham, U, n, work, L, rb, re, schedule, row_ptr, nullptr, s))) return rc;
  cudaError_t e = cudaMemcpyAsync(n_pairs, row_ptr + (re - rb), sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "count copy");
  return read_status(work, s);
}

int nqs_fill_coupled_pairs(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work,
                           int64_t rb, int64_t re, int schedule, const int64_t* row_ptr,
                           uint32_t* pair_j, uint32_t* pair_k, void* stream) {
  StageHeader L;
  bool sorted;
  schedule = split_schedule(schedule, &sorted);
  int rc = check_work(ham, U, n, work, &L);
  if (rc || (rc = check_rows(n, rb, re)) || (rc = check_schedule(ham, n, schedule))) return rc;
  if (!row_ptr || !pair_j || !pair_k) return fail(NQS_ERR_ARG, "null output");
  if (re == rb) return NQS_OK;
  cudaError_t e = launch_search(ham, U, n, (char*)work, L, rb, re, schedule, (int64_t*)row_ptr, pair_j,
                                pair_k, kFill, nullptr, (cudaStream_t)stream, sorted);
  if (e != cudaSuccess) return cuda_fail(e, "pair fill kernel");
  return NQS_OK;
}

int64_t nqs_pairs_scratch_bytes(int64_t rows, int64_t max_pairs) {
  if (rows < 0 || max_pairs < 0) return fail(NQS_ERR_ARG, "negative size");
  return pair_scratch_bytes(rows, max_pairs);
}

// Pinned host words that the one-pass search reads its count, overflow flag
// and header into.  Copies into pinned memory stay asynchronous, so the
// compaction is queued behind them before the host waits.  One block per host
// thread, kept for the thread's lifetime (portable across devices).
namespace {
struct CountWords {
  int64_t n_pairs;
  int64_t overflow;
  StageHeader hdr;
};
struct CountReadback {
  CountWords* w = nullptr;
  ~CountReadback() {
    if (w) cudaFreeHost(w);
  }
};
thread_local CountReadback g_readback;
}  // namespace

int nqs_find_coupled_pairs(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work,
                           int64_t rb, int64_t re, int schedule, void* scratch, int64_t scratch_bytes,
                           int64_t* row_ptr, uint32_t* pair_j, uint32_t* pair_k, int64_t capacity,
                           int64_t* n_pairs, void* stream) {
  StageHeader L;
  const int flags = schedule & NQS_ROWS_UNSORTED;
  bool sorted;
  schedule = split_schedule(schedule, &sorted);
  int rc = check_work(ham, U, n, work, &L);
  if (rc || (rc = check_rows(n, rb, re)) || (rc = check_schedule(ham, n, schedule))) return rc;
  if (!row_ptr || !n_pairs) return fail(NQS_ERR_ARG, "null row_ptr or n_pairs");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t rows = re - rb;
  const int sched = pick_schedule(ham, n, schedule);
  if (!scratch || sched == NQS_SCHED_BATCH || sched == NQS_SCHED_TRIE) {  // count, then fill
    rc = nqs_count_coupled_pairs(ham, U, n, work, rb, re, schedule, row_ptr, n_pairs, stream);
    if (rc) return rc;
    if (*n_pairs > capacity) return fail(NQS_ERR_CAPACITY, "pair capacity too small");
    if (*n_pairs > 0 && (!pair_j || !pair_k)) return fail(NQS_ERR_ARG, "null pair arrays");
    return nqs_fill_coupled_pairs(ham, U, n, work, rb, re, schedule | flags, row_ptr, pair_j, pair_k, stream);
  }
  if (((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  PairScratch sc = pair_scratch_view(scratch, rows, scratch_bytes);
  if (sc.max_pairs < 1) {  // no room at all: count only, so that row_ptr and *n_pairs are valid
    rc = nqs_count_coupled_pairs(ham, U, n, work, rb, re, schedule, row_ptr, n_pairs, stream);
    return rc ? rc : fail(NQS_ERR_CAPACITY, "scratch too small");
  }
  if ((rc = count_pass(ham, U, n, work, L, rb, re, schedule, row_ptr, &sc, s))) return rc;
  // The count, the overflow flag and the status reach the host while the
  // compaction (enqueued right behind them) runs; the compaction checks on the
  // device that the pairs fit and writes nothing otherwise.
  cudaError_t e = cudaSuccess;
  if (!g_readback.w) {
    void* h = nullptr;
    if ((e = cudaHostAlloc(&h, sizeof(CountWords), cudaHostAllocPortable)) != cudaSuccess)
      return cuda_fail(e, "pinned readback");
    g_readback.w = (CountWords*)h;
  }
  CountWords* cw = g_readback.w;
  e = cudaMemcpyAsync(&cw->n_pairs, row_ptr + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cw->overflow, sc.cursor + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cw->hdr, work, sizeof(StageHeader), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "count copy");
  cudaEvent_t counted;
  if ((e = cudaEventCreateWithFlags(&counted, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
  e = cudaEventRecord(counted, s);
  const bool arrays = pair_j && pair_k;
  if (e == cudaSuccess && rows > 0)
    e = launch_pairs_compact(ham, sc, (char*)work, L, rb, rows, row_ptr, pair_j, pair_k, arrays ? capacity : 0, s,
                             sorted);
  const cudaError_t es = cudaEventSynchronize(counted);
  cudaEventDestroy(counted);
  if (e != cudaSuccess) return cuda_fail(e, "compaction kernel");
  if (es != cudaSuccess) return cuda_fail(es, "stream synchronize");
  *n_pairs = cw->n_pairs;
  const int64_t overflow = cw->overflow;
  if (cw->hdr.magic != kStageMagic) return fail(NQS_ERR_ARG, "workspace was not staged");
  if ((rc = status_to_code(cw->hdr.status))) return rc;
  const bool fits = !overflow && *n_pairs <= sc.max_pairs && *n_pairs <= (arrays ? capacity : 0);
  if (!fits && rows > 0 && (e = launch_clear_capacity((char*)work, s)) != cudaSuccess)
    return cuda_fail(e, "status reset");
  if (overflow || *n_pairs > sc.max_pairs) return fail(NQS_ERR_CAPACITY, "scratch too small for the pairs found");
  if (*n_pairs > capacity) return fail(NQS_ERR_CAPACITY, "pair capacity too small");
  if (*n_pairs > 0 && !arrays) return fail(NQS_ERR_ARG, "null pair arrays");
  return NQS_OK;
}

int nqs_find_coupled_pairs_async(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work,
                                 int64_t rb, int64_t re, int schedule, void* scratch, int64_t scratch_bytes,
                                 int64_t* row_ptr, uint32_t* pair_j, uint32_t* pair_k, int64_t capacity,
                                 void* stream) {
  StageHeader L;
  bool sorted;
  schedule = split_schedule(schedule, &sorted);
  int rc = check_work(ham, U, n, work, &L);
  if (rc || (rc = check_rows(n, rb, re)) || (rc = check_schedule(ham, n, schedule))) return rc;
  const bool packed = pair_j && !pair_k;  // one 64-bit word per pair in pair_j (column << 32 | pattern)
  if (!row_ptr || capacity < 0 || (capacity > 0 && !pair_j)) return fail(NQS_ERR_ARG, "null row_ptr or pair arrays");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t rows = re - rb;
  const int sched = pick_schedule(ham, n, schedule);
  const bool one_pass = scratch && sched == NQS_SCHED_TERMS;
  if (packed && (sorted || !one_pass))
    return fail(NQS_ERR_UNSUPPORTED, "packed pairs need LoopOverTerms, a scratch and NQS_ROWS_UNSORTED");
  if (packed && (((uintptr_t)pair_j) & 7)) return fail(NQS_ERR_ARG, "packed pairs not 8-byte aligned");
  if (one_pass && (((uintptr_t)scratch) & 255)) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  PairScratch sc;
  if (one_pass) {
    sc = pair_scratch_view(scratch, rows, scratch_bytes);
    if (sc.max_pairs < 1) return fail(NQS_ERR_CAPACITY, "scratch too small");
  }
  // the capacity bit then tells about this call alone
  cudaError_t e = launch_clear_capacity((char*)work, s);
  if (e != cudaSuccess) return cuda_fail(e, "status reset");
  if ((rc = count_pass(ham, U, n, work, L, rb, re, schedule, row_ptr, one_pass ? &sc : nullptr, s))) return rc;
  if (rows == 0) return NQS_OK;
  if (one_pass) {
    // the compaction checks the total against min(capacity, scratch) and the scratch's
    // overflow flag, and writes nothing (capacity bit set) when the pairs do not fit
    e = launch_pairs_compact(ham, sc, (char*)work, L, rb, rows, row_ptr, pair_j, pair_k, capacity, s, sorted);
    if (e != cudaSuccess) return cuda_fail(e, "compaction kernel");
    return NQS_OK;
  }
  if ((e = launch_capacity_check(row_ptr, rows, capacity, (char*)work, s)) != cudaSuccess)
    return cuda_fail(e, "capacity check");
  e = launch_search(ham, U, n, (char*)work, L, rb, re, schedule, row_ptr, pair_j, pair_k, kFill, nullptr, s, sorted);
  if (e != cudaSuccess) return cuda_fail(e, "pair fill kernel");
  return NQS_OK;
}

int64_t nqs_candidates_scratch_bytes(const nqs_ham* ham, int64_t n_unq) {
  if (!ham || n_unq < 0) return fail(NQS_ERR_ARG, "bad argument to nqs_candidates_scratch_bytes");
  return cand_scratch_bytes(ham, n_unq);
}

int nqs_full_candidates(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, void* scratch,
                        int64_t scratch_bytes, uint32_t* cand_id, double* hval, uint64_t* cand,
                        int32_t* cand_in_u, int64_t capacity, int64_t* n_cand, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc) return rc;
  if (!n_cand) return fail(NQS_ERR_ARG, "null n_cand");
  *n_cand = 0;
  if (ham->cplx) return fail(NQS_ERR_UNSUPPORTED, "exact local energy of a complex Hamiltonian");
  if (n == 0 || ham->n_xy == 0) return NQS_OK;
  if (!scratch || !cand_id) return fail(NQS_ERR_ARG, "null scratch or cand_id");
  if (((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  if (n * ham->n_xy > (int64_t(1) << 29)) return fail(NQS_ERR_UNSUPPORTED, "more than 2^29 candidate entries");
  if (scratch_bytes < cand_scratch_bytes(ham, n)) return fail(NQS_ERR_CAPACITY, "scratch smaller than nqs_candidates_scratch_bytes");
  int limit = 0;
  cudaError_t e = launch_full_candidates(ham, U, n, (const char*)work, L, scratch, cand_id, hval, cand, cand_in_u,
                                         cand ? capacity : 0, n_cand, &limit, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "candidate kernels");
  if (limit) return fail(NQS_ERR_DEVICE_LIMIT, "candidate table or membership probe ran out");
  if (!cand || *n_cand > capacity) return fail(NQS_ERR_CAPACITY, "candidate capacity too small");
  return NQS_OK;
}

int nqs_local_energy_full(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, const double* a,
                          const double* b, const uint32_t* cand_id, const double* hval, int64_t n_cand,
                          const double* ca, const double* cb, void* scratch, int64_t scratch_bytes,
                          double* eloc_re, double* eloc_im, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc) return rc;
  if (ham->cplx) return fail(NQS_ERR_UNSUPPORTED, "exact local energy of a complex Hamiltonian");
  if (n == 0) return NQS_OK;
  if (!a || !eloc_re) return fail(NQS_ERR_ARG, "null logpsi_re or eloc_re");
  if ((b || cb) && !eloc_im) return fail(NQS_ERR_ARG, "complex amplitudes need eloc_im");
  if (ham->n_xy > 0 && (!cand_id || !hval || !ca || n_cand < 1)) return fail(NQS_ERR_ARG, "null candidate arrays");
  if (!scratch || scratch_bytes < 32 * std::max<int64_t>(n_cand, 1)) return fail(NQS_ERR_CAPACITY, "scratch too small");
  if (((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  cudaError_t e = launch_local_energy_full(n, ham->n_xy, (const char*)work, L, a, b, cand_id, hval, n_cand, ca, cb,
                                           scratch, eloc_re, eloc_im, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "full local energy kernels");
  return NQS_OK;
}

int64_t nqs_sr_scratch_bytes(int64_t n_unq, int64_t n_params) {
  if (n_unq < 0 || n_params < 0) return fail(NQS_ERR_ARG, "negative size");
  return std::max(sr_scratch_bytes(n_params), sr_top_scratch_bytes(n_unq));
}

int nqs_sr_top(int64_t n_unq, const double* logpsi_re, int64_t n_sr, int32_t* idx, void* scratch,
               int64_t scratch_bytes, void* stream) {
  if (n_unq < 1 || n_sr < 1 || !logpsi_re || !idx) return fail(NQS_ERR_ARG, "bad argument to nqs_sr_top");
  if (n_unq >= (int64_t(1) << 31)) return fail(NQS_ERR_UNSUPPORTED, "more than 2^31 samples");
  if (!scratch || scratch_bytes < sr_top_scratch_bytes(n_unq)) return fail(NQS_ERR_CAPACITY, "scratch too small");
  if (((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  cudaError_t e = launch_sr_top(n_unq, logpsi_re, n_sr, idx, scratch, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "top-probability selection");
  return NQS_OK;
}

int nqs_sr_step(int n_sr, int64_t n_params, const float* O, const double* logpsi_re, const double* eloc_re,
                const double* evar, double lambda, double* delta, double* T, void* scratch, int64_t scratch_bytes,
                void* stream) {
  if (n_sr < 1 || n_sr > 128) return fail(NQS_ERR_UNSUPPORTED, "n_sr must be in 1..128");
  if (n_params < 1 || !O || !logpsi_re || !eloc_re || !evar || !delta) return fail(NQS_ERR_ARG, "bad argument to nqs_sr_step");
  if (!(lambda >= 0.0)) return fail(NQS_ERR_ARG, "lambda must be >= 0");
  if (!scratch || scratch_bytes < sr_scratch_bytes(n_params)) return fail(NQS_ERR_CAPACITY, "scratch too small");
  if (((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  int32_t st = 0;
  cudaError_t e = launch_sr_step(n_sr, n_params, O, logpsi_re, eloc_re, evar, lambda, scratch, delta, T, &st,
                                 (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "SR kernels");
  if (st & kStatusLimit) return fail(NQS_ERR_DEVICE_LIMIT, "tensor-core pipeline wait ran out");
  if (st & kStatusRange) return fail(NQS_ERR_RANGE, "T + lambda I is not positive definite in FP64");
  return NQS_OK;
}

int64_t nqs_gumbel_scratch_bytes(int64_t n_parents) {
  if (n_parents < 0) return fail(NQS_ERR_ARG, "negative n_parents");
  return sample_scratch_bytes(n_parents);
}

int nqs_gumbel_topk_level(int n_qubits, int level, int64_t n_parents, const uint64_t* parent_x,
                          const double* parent_l, const double* parent_lt, const double* cond_logp,
                          const double* gumbel, int64_t K, void* scratch, int64_t scratch_bytes, uint64_t* child_x,
                          double* child_l, double* child_lt, int64_t* n_children, void* stream) {
  if (!n_children) return fail(NQS_ERR_ARG, "null n_children");
  *n_children = 0;
  if (n_qubits < 1 || n_qubits > 64 * kMaxWords) return fail(NQS_ERR_ARG, "n_qubits out of range");
  if (level < 0 || level >= n_qubits) return fail(NQS_ERR_ARG, "level out of range");
  if (n_parents < 1 || K < 1) return fail(NQS_ERR_ARG, "n_parents and K must be positive");
  if (n_parents >= (int64_t(1) << 30)) return fail(NQS_ERR_UNSUPPORTED, "more than 2^30 kept vectors");
  if ((level > 0 && !parent_x) || !parent_l || !parent_lt || !cond_logp || !gumbel || !child_x || !child_l || !child_lt)
    return fail(NQS_ERR_ARG, "null array");
  if (!scratch || scratch_bytes < sample_scratch_bytes(n_parents)) return fail(NQS_ERR_CAPACITY, "scratch too small");
  if (((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  cudaError_t e = launch_gumbel_level((n_qubits + 63) / 64, level, n_parents, parent_x, parent_l, parent_lt, cond_logp,
                                      gumbel, K, scratch, child_x, child_l, child_lt, n_children, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sampling kernels");
  return NQS_OK;
}

int nqs_gumbel_topk_level_async(int n_qubits, int level, int64_t max_parents, const int64_t* n_parents,
                                const uint64_t* parent_x, const double* parent_l, const double* parent_lt,
                                const double* cond_logp, const double* gumbel, int64_t K, void* scratch,
                                int64_t scratch_bytes, uint64_t* child_x, double* child_l, double* child_lt,
                                int64_t* counts, void* stream) {
  if (n_qubits < 1 || n_qubits > 64 * kMaxWords) return fail(NQS_ERR_ARG, "n_qubits out of range");
  if (level < 0 || level >= n_qubits) return fail(NQS_ERR_ARG, "level out of range");
  if (max_parents < 1 || K < 1) return fail(NQS_ERR_ARG, "max_parents and K must be positive");
  if (max_parents > sample_async_limit()) return fail(NQS_ERR_UNSUPPORTED, "max_parents above the device-count limit");
  if (!n_parents || !counts || (level > 0 && !parent_x) || !parent_l || !parent_lt || !cond_logp || !gumbel ||
      !child_x || !child_l || !child_lt)
    return fail(NQS_ERR_ARG, "null array");
  if (!scratch || scratch_bytes < sample_scratch_bytes(max_parents)) return fail(NQS_ERR_CAPACITY, "scratch too small");
  if (((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  cudaError_t e = launch_gumbel_level_async((n_qubits + 63) / 64, level, max_parents, (const long long*)n_parents,
                                            parent_x, parent_l, parent_lt, cond_logp, gumbel, K, scratch, child_x,
                                            child_l, child_lt, (long long*)counts, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sampling kernels");
  return NQS_OK;
}

int64_t nqs_gumbel_async_max_parents(void) { return sample_async_limit(); }

int nqs_find_pairs_half(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, uint32_t* rec_i,
                        uint32_t* rec_j, uint32_t* rec_k, int64_t capacity, int64_t* n_slots, void* stream) {
  return nqs_find_pairs_part(ham, U, n, work, 0, 1, rec_i, rec_j, rec_k, capacity, n_slots, stream);
}

int nqs_find_pairs_part(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, int part, int n_parts,
                        uint32_t* rec_i, uint32_t* rec_j, uint32_t* rec_k, int64_t capacity, int64_t* n_slots,
                        void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc) return rc;
  if (!n_slots) return fail(NQS_ERR_ARG, "null n_slots");
  *n_slots = 0;
  if (n_parts < 1 || part < 0 || part >= n_parts) return fail(NQS_ERR_ARG, "bad part");
  if (capacity < 0 || (capacity > 0 && (!rec_i || !rec_j || !rec_k))) return fail(NQS_ERR_ARG, "null record arrays");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_find_half(ham, U, (char*)work, L, rec_i, rec_j, rec_k, capacity, s, part, n_parts);
  if (e != cudaSuccess) return cuda_fail(e, "half-pair search kernel");
  int64_t cur[2] = {0, 0};
  e = cudaMemcpyAsync(cur, (char*)work + L.off_counters + 8 * kCtrHalf, sizeof(cur), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "slot count copy");
  if ((rc = read_status(work, s))) return rc;
  *n_slots = cur[0];
  if (cur[1] != 0) return fail(NQS_ERR_CAPACITY, "record capacity too small (n_slots: slots asked for)");
  return NQS_OK;
}

int64_t nqs_route_scratch_bytes(int n_parts) {
  if (n_parts < 1 || n_parts > 1024) return fail(NQS_ERR_ARG, "n_parts outside [1, 1024]");
  return 256 + 8 * (int64_t)(n_parts + 1) + 2 * 8 * (int64_t)n_parts + 256;
}

int nqs_route_records(int n_parts, const int64_t* bounds, const uint32_t* rec_i, const uint32_t* rec_j,
                      const uint32_t* rec_k, int64_t n_slots, uint32_t* out_i, uint32_t* out_j, uint32_t* out_k,
                      int64_t capacity, int64_t* counts, void* scratch, int64_t scratch_bytes, void* stream) {
  if (n_parts < 1 || n_parts > 1024) return fail(NQS_ERR_ARG, "n_parts outside [1, 1024]");
  if (!bounds || !counts) return fail(NQS_ERR_ARG, "null bounds or counts");
  if (n_slots < 0 || (n_slots > 0 && (!rec_i || !rec_j || !rec_k))) return fail(NQS_ERR_ARG, "null record arrays");
  if (!scratch || scratch_bytes < nqs_route_scratch_bytes(n_parts)) return fail(NQS_ERR_ARG, "scratch too small");
  if (((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch not 256-byte aligned");
  for (int p = 0; p < n_parts; ++p)
    if (bounds[p] < 0 || bounds[p + 1] < bounds[p]) return fail(NQS_ERR_ARG, "bounds not ascending");
  if (bounds[0] != 0) return fail(NQS_ERR_ARG, "bounds must start at row 0");
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)scratch;
  int64_t* d_bounds = (int64_t*)(base + 256);
  auto* d_counts = (unsigned long long*)(base + 256 + ((8 * (n_parts + 1) + 255) & ~255));
  unsigned long long* d_cur = d_counts + n_parts;
  cudaError_t e = cudaMemcpyAsync(d_bounds, bounds, 8 * (size_t)(n_parts + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_route_count(rec_i, rec_j, n_slots, d_bounds, n_parts, d_counts, s);
  std::vector<unsigned long long> c(n_parts, 0ull);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c.data(), d_counts, 8 * (size_t)n_parts, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "record routing count");
  std::vector<unsigned long long> off(n_parts, 0ull);
  unsigned long long total = 0;
  for (int p = 0; p < n_parts; ++p) {
    off[p] = total;
    total += c[p];
    counts[p] = (int64_t)c[p];
  }
  if ((int64_t)total > capacity) return fail(NQS_ERR_CAPACITY, "routed record capacity too small (counts: per part)");
  if (total > 0 && (!out_i || !out_j || !out_k)) return fail(NQS_ERR_ARG, "null output arrays");
  e = cudaMemcpyAsync(d_cur, off.data(), 8 * (size_t)n_parts, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_route_scatter(rec_i, rec_j, rec_k, n_slots, d_bounds, n_parts, d_cur, out_i, out_j, out_k, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // off lives on this stack frame
  if (e != cudaSuccess) return cuda_fail(e, "record routing scatter");
  return NQS_OK;
}

int nqs_pairs_from_records(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, const uint32_t* rec_i,
                           const uint32_t* rec_j, const uint32_t* rec_k, int64_t n_rec, int64_t rb, int64_t re,
                           void* scratch, int64_t scratch_bytes, int64_t* row_ptr, uint32_t* pair_j,
                           uint32_t* pair_k, int64_t capacity, int64_t* n_pairs, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc || (rc = check_rows(n, rb, re))) return rc;
  if (!row_ptr || !n_pairs) return fail(NQS_ERR_ARG, "null row_ptr or n_pairs");
  if (n_rec < 0 || (n_rec > 0 && (!rec_i || !rec_j || !rec_k))) return fail(NQS_ERR_ARG, "null record arrays");
  if (n_rec >= (int64_t(1) << 40)) return fail(NQS_ERR_ARG, "too many records");
  if (!scratch || ((uintptr_t)scratch) & 255) return fail(NQS_ERR_ARG, "scratch null or not 256-byte aligned");
  *n_pairs = 0;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t rows = re - rb;
  auto* status = (int32_t*)((char*)work + offsetof(StageHeader, status));
  cudaError_t e = cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) e = launch_records_count(rec_i, rec_j, n_rec, rb, rows, ham->has_diag, row_ptr + 1, status, s);
  if (e == cudaSuccess && rows > 0) e = launch_scan(row_ptr + 1, rows, (char*)work, L, s);
  if (e != cudaSuccess) return cuda_fail(e, "record count kernels");
  int64_t total = 0;
  if ((e = cudaMemcpyAsync(&total, row_ptr + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "count copy");
  if ((rc = read_status(work, s))) return rc;
  *n_pairs = total;
  if (total > capacity) return fail(NQS_ERR_CAPACITY, "pair capacity too small");
  if (total > 0 && (!pair_j || !pair_k)) return fail(NQS_ERR_ARG, "null pair arrays");
  // the records as a one-pass scratch: header (record count, overflow flag), then the sort keys
  if (scratch_bytes < 256 + 8 * total) return fail(NQS_ERR_CAPACITY, "scratch too small for the pairs (8 B each)");
  if (rows == 0) return NQS_OK;
  PairScratch sc;
  std::memset(&sc, 0, sizeof(sc));
  sc.cursor = (int64_t*)scratch;
  sc.rec_i = const_cast<uint32_t*>(rec_i);
  sc.rec_j = const_cast<uint32_t*>(rec_j);
  sc.rec_k = const_cast<uint32_t*>(rec_k);
  sc.max_rec = n_rec;
  sc.max_pairs = total;
  sc.keys = (uint64_t*)((char*)scratch + 256);
  const int64_t hdr[2] = {n_rec, 0};
  if ((e = cudaMemcpyAsync(sc.cursor, hdr, sizeof(hdr), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "record header");
  e = launch_pairs_compact(ham, sc, (char*)work, L, rb, rows, row_ptr, pair_j, pair_k, capacity, s);
  if (e != cudaSuccess) return cuda_fail(e, "record scatter and row sort");
  return read_status(work, s);   // synchronises: hdr is read before this frame returns
}

int nqs_local_energy_half(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, const double* a,
                          const double* b, const uint32_t* rec_i, const uint32_t* rec_j, const uint32_t* rec_k,
                          int64_t n_slots, int precision, double* eloc_re, double* eloc_im, double* hdiag,
                          void* hrec, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc) return rc;
  if (precision != NQS_PREC_FP64 && precision != NQS_PREC_FP32C) return fail(NQS_ERR_ARG, "bad precision");
  if (n > 0 && (!a || !eloc_re)) return fail(NQS_ERR_ARG, "null logpsi_re or eloc_re");
  if ((b || ham->cplx) && !eloc_im) return fail(NQS_ERR_ARG, "complex log psi or H needs eloc_im");
  if (n_slots < 0 || (n_slots > 0 && (!rec_i || !rec_j || !rec_k))) return fail(NQS_ERR_ARG, "null record arrays");
  if (n == 0) return NQS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_amplitudes(a, b, n, precision, (char*)work, L, s, U);
  if (e != cudaSuccess) return cuda_fail(e, "amplitude kernel");
  e = launch_local_energy_half(ham, U, n, (const char*)work, L, b != nullptr, rec_i, rec_j, rec_k, n_slots, precision,
                               eloc_re, eloc_im, hdiag, hrec, s);
  if (e != cudaSuccess) return cuda_fail(e, "half-pair energy kernels");
  return NQS_OK;
}

int nqs_local_energy_backward_half(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work, const double* a,
                                   const double* b, const uint32_t* rec_i, const uint32_t* rec_j,
                                   const uint32_t* rec_k, int64_t n_slots, const void* hrec, const double* eloc_re,
                                   const double* eloc_im, const double* hdiag, const double* evar,
                                   const double* g_re, const double* g_im, const double* g_evar, int precision,
                                   double* grad_re, double* grad_im, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc) return rc;
  if (precision != NQS_PREC_FP64 && precision != NQS_PREC_FP32C) return fail(NQS_ERR_ARG, "bad precision");
  if (n > 0 && (!a || !eloc_re || !evar || !grad_re)) return fail(NQS_ERR_ARG, "null forward input or grad_re");
  if (b && (!grad_im || !eloc_im)) return fail(NQS_ERR_ARG, "complex log psi needs grad_im and eloc_im");
  if (ham->cplx && !eloc_im) return fail(NQS_ERR_ARG, "a complex Hamiltonian needs eloc_im");
  const bool pairs_needed = g_re || g_im;
  if (pairs_needed && (!hdiag || n_slots < 0 || (n_slots > 0 && (!rec_i || !rec_j || !rec_k))))
    return fail(NQS_ERR_ARG, "upstream E_loc gradient needs the records and hdiag");
  if (n == 0) return NQS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (pairs_needed && (e = launch_amplitudes(a, b, n, precision, (char*)work, L, s, U)) != cudaSuccess)
    return cuda_fail(e, "amplitude kernel");
  e = launch_backward_half(ham, U, n, (char*)work, L, b != nullptr, a, rec_i, rec_j, rec_k, n_slots, hrec, eloc_re,
                           eloc_im, hdiag, evar, g_re, g_im, g_evar, precision, grad_re, grad_im, s);
  if (e != cudaSuccess) return cuda_fail(e, "half-pair adjoint kernels");
  return NQS_OK;
}

int nqs_local_energy(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work,
                     const double* a, const double* b, int64_t rb, int64_t re,
                     const int64_t* row_ptr, const uint32_t* pair_j, const uint32_t* pair_k,
                     int precision, double* eloc_re, double* eloc_im, double* hdiag,
                     void* hpair, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc || (rc = check_rows(n, rb, re))) return rc;
  if (precision != NQS_PREC_FP64 && precision != NQS_PREC_FP32C) return fail(NQS_ERR_ARG, "bad precision");
  if (n > 0 && !a) return fail(NQS_ERR_ARG, "null logpsi_re");
  if (!eloc_re) return fail(NQS_ERR_ARG, "null eloc_re");
  if (b && !eloc_im) return fail(NQS_ERR_ARG, "complex log psi needs eloc_im");
  if (ham->cplx && !eloc_im) return fail(NQS_ERR_ARG, "a complex Hamiltonian needs eloc_im");
  if (re > rb && (!row_ptr || !pair_j)) return fail(NQS_ERR_ARG, "null pair arrays");
  if (!pair_k && (((uintptr_t)pair_j) & 7)) return fail(NQS_ERR_ARG, "packed pairs not 8-byte aligned");
  if (re == rb) return NQS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_amplitudes(a, b, n, precision, (char*)work, L, s, U);
  if (e != cudaSuccess) return cuda_fail(e, "amplitude kernel");
  e = launch_local_energy(ham, U, n, (char*)work, L, b != nullptr, rb, re, row_ptr, pair_j, pair_k,
                          precision, eloc_re, eloc_im, hdiag, hpair, s);
  if (e != cudaSuccess) return cuda_fail(e, "local energy kernel");
  return NQS_OK;
}

int nqs_variational_energy(int64_t n, const double* a, const double* eloc_re, void* work, double* out,
                           void* stream) {
  if (n <= 0 || !a || !eloc_re || !out || !work) return fail(NQS_ERR_ARG, "bad argument");
  if (((uintptr_t)work) & 255) return fail(NQS_ERR_ARG, "workspace not 256-byte aligned");
  cudaError_t e = launch_variational_energy(n, a, eloc_re, (char*)work, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "variational energy kernel");
  return NQS_OK;
}

int nqs_evar_combine(const double* parts, int k, double* out, void* stream) {
  if (!parts || !out || k < 1) return fail(NQS_ERR_ARG, "bad argument to nqs_evar_combine");
  cudaError_t e = launch_evar_combine(parts, k, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "E^var combine kernel");
  return NQS_OK;
}

int nqs_evar_combine_host(const double* parts, int k, double* out) {
  if (!parts || !out || k < 1) return fail(NQS_ERR_ARG, "bad argument to nqs_evar_combine_host");
  double amax = -1.7976931348623157e308;
  for (int r = 0; r < k; ++r)
    if (parts[3 * r + 2] > 0.0) amax = std::max(amax, parts[3 * r + 1]);
  double S = 0.0, N = 0.0;
  for (int r = 0; r < k; ++r) {
    if (!(parts[3 * r + 2] > 0.0)) continue;
    const double f = std::exp(2.0 * (parts[3 * r + 1] - amax));
    S += parts[3 * r + 2] * f;
    N += parts[3 * r] * parts[3 * r + 2] * f;
  }
  out[0] = S > 0.0 ? N / S : 0.0;
  out[1] = amax;
  out[2] = S;
  return NQS_OK;
}

int nqs_local_energy_backward(const nqs_ham* ham, const uint64_t* U, int64_t n, void* work,
                              const double* a, const double* b, int64_t rb, int64_t re,
                              const int64_t* row_ptr, const uint32_t* pair_j, const uint32_t* pair_k,
                              const void* hpair,
                              const double* eloc_re, const double* eloc_im, const double* hdiag,
                              const double* evar, const double* g_re, const double* g_im,
                              const double* g_evar, int precision, double* grad_re,
                              double* grad_im, void* stream) {
  StageHeader L;
  int rc = check_work(ham, U, n, work, &L);
  if (rc || (rc = check_rows(n, rb, re))) return rc;
  if (precision != NQS_PREC_FP64 && precision != NQS_PREC_FP32C) return fail(NQS_ERR_ARG, "bad precision");
  if (n > 0 && (!a || !eloc_re || !evar)) return fail(NQS_ERR_ARG, "null forward input");
  if (!grad_re) return fail(NQS_ERR_ARG, "null grad_re");
  if (b && (!grad_im || !eloc_im)) return fail(NQS_ERR_ARG, "complex log psi needs grad_im and eloc_im");
  if (ham->cplx && !eloc_im) return fail(NQS_ERR_ARG, "a complex Hamiltonian needs eloc_im");
  const bool pairs_needed = g_re || g_im;
  if (pairs_needed && !pair_k && (((uintptr_t)pair_j) & 7))
    return fail(NQS_ERR_ARG, "packed pairs not 8-byte aligned");
  if (pairs_needed && re > rb && (!row_ptr || !pair_j || !hdiag))
    return fail(NQS_ERR_ARG, "upstream E_loc gradient needs pairs and hdiag");
  if (re == rb) return NQS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (pairs_needed) {
    e = launch_amplitudes(a, b, n, precision, (char*)work, L, s, U);
    if (e != cudaSuccess) return cuda_fail(e, "amplitude kernel");
  }
  e = launch_backward(ham, U, n, (char*)work, L, b != nullptr, a, b, rb, re, row_ptr, pair_j, pair_k,
                      eloc_re, eloc_im, hdiag, evar, g_re, g_im, g_evar, precision, hpair, grad_re, grad_im, s);
  if (e != cudaSuccess) return cuda_fail(e, "backward kernel");
  return NQS_OK;
}

}  // extern "C"
