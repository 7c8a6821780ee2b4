// Internal declarations of the GB300 local-energy library (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "nqs.h"

namespace nqs {

constexpr int kMaxWords = 4;                 // N <= 256 qubits
constexpr uint32_t kDummy = 0xFFFFFFFFu;     // padding slot of the search table
constexpr int kHeavyTerms = 24;              // |P_XY| above this: warp-cooperative term loop
namespace kForm { constexpr int Terms = 0, Local = 1; }
constexpr int kRowsPerWarp = 8;              // rows scanned together by one warp
constexpr int kSortWarpMax = 512;           // rows with up to this many pairs are sorted by one warp
constexpr int kSortBlockKeys = 16384;        // longer rows: one block, in shared memory up to this size

// counter slots (uint64) of the workspace's counter region
constexpr int kCtrItems = 0;                 // LoopOverTerms work items taken
constexpr int kCtrBigCount = 1;              // long rows queued for the block sort
constexpr int kCtrBigNext = 2;               // long rows taken by the block sort
constexpr int kCtrBatch = 3;                 // LoopOverBatch row batches taken
constexpr int kCtrTrie = 4;                  // LoopOverTrie rows taken
constexpr int kCtrHalf = 8;                  // half-stored records: slots taken (8), overflow flag (9)

// status bits (device status word)
constexpr int kStatusDuplicate = 1;
constexpr int kStatusBadBits = 2;
constexpr int kStatusLimit = 4;
constexpr int kStatusRange = 8;
constexpr int kStatusCapacity = 16;        // a pair buffer sized ahead of time was too small
constexpr int kStatusNoTrie = 32;          // trie search on a workspace whose prefix tree was not built

// ---------------------------------------------------------------------------
// Hamiltonian tables (device) -- Fig. ham_prep, regrouped:
//   pattern ids: [diag (XY = 0) if present][heavy patterns][light patterns],
//   each class sorted by XY value; terms grouped by pattern id, sorted by z.
// ---------------------------------------------------------------------------
struct nqs_ham_dev {
  int n_qubits = 0;
  int W = 0;
  int64_t n_terms = 0;
  int64_t n_xy = 0;
  int has_diag = 0;              // pattern 0 is XY = 0
  int64_t heavy_end = 0;         // ids < heavy_end (and >= has_diag) are heavy
  int64_t max_group = 0;
  int64_t n_srch = 0;            // search-table slots, multiple of 32
  int n_segs = 0;                // segments of the search table (one per orientation qubit)

  uint64_t* xy = nullptr;        // [n_xy][W]
  uint32_t* row_ptr = nullptr;   // [n_xy + 1]
  uint64_t* yz = nullptr;        // [n_terms][W]
  double* coef = nullptr;        // [n_terms]   h_l * (-1)^{|Y|/2}
  float2* coef_f = nullptr;      // [n_terms]   (hi, lo) split of coef
  uint32_t* srch_hash = nullptr; // [n_srch]    linear hash of each pattern
  uint32_t* srch_id = nullptr;   // [n_srch]    pattern id or kDummy
  uint64_t* srch_rec = nullptr;  // [n_srch][rec_words]: (hash | id << 32), XY words (0 for padding)
  int4* segs = nullptr;          // [n_segs] {t, first group, end group, 0}: the patterns whose highest
                                 // set qubit is t, in groups of 32 slots; largest segments first
  int rec_words = 0;             // 64-bit words per search record (16-byte multiple)
  uint32_t* hash_basis = nullptr;// [64 * W]    R[b]: h(v) = XOR of R[b] over set bits b
  unsigned long long* xy_table = nullptr;  // XY hash set: slots of W key words + (id | hash << 32), id = ~0: empty
  int64_t xy_cap = 0;            // slots (power of two)
  unsigned long long* wmask = nullptr;     // [5] bit w set if some pattern has Hamming weight w
  int4* xy_trie = nullptr;       // prefix tree of the patterns: {child0, child1, single pattern or -1, 0}
  int64_t n_xy_nodes = 0;
  uint32_t* xy_hash = nullptr;   // [n_xy] linear hash of each pattern

  // MatrixElement forms (exact regroupings of the sum of Eq. pauli_melem),
  // chosen per pattern at load; fm[k] = {kind | nb << 4, table offset, mask
  // offset, packed qubits}:
  //   kForm::Local  every YZ_l agrees with YZ_0 outside the pattern's own
  //     nb <= 4 qubits (packed 8 bits each): H = (-1)^{|x' & A|} T[u], A the
  //     common part, u = x' read at those qubits, T the 2^nb table;
  //   kForm::Terms  the term loop (heavy patterns: all lanes of a warp).
  // quadratic diagonal (every diagonal term a Z string on at most two qubits):
  //   H_xx = C + sum_{r in x} b_r + sum_{r < s in x} B_rs, stored as
  //   [C, b_0 .. b_{64W-1}, B (64W x 64W, row-major, r < s used)].
  int4* fm = nullptr;            // [n_xy]
  int4* fmx = nullptr;           // N <= 64: [n_xy][2] one 32-byte record per pattern: fm, then the
                                 //   local form's sign mask A (low, high 32 bits) -- one gather per pair
  double* fv_d = nullptr;        // value pool
  float2* fv_f = nullptr;        // same, (hi, lo) split
  uint64_t* fz = nullptr;        // mask pool [..][W]
  int64_t n_local = 0;
  int diag_quad = 0;             // the diagonal pattern uses the quadratic form
  double* quad_d = nullptr;      // [1 + 64W + (64W)^2]
  float2* quad_f = nullptr;
  // complex H: strings with an odd number of Y have imaginary coefficients
  // h i^{|Y|}; their parts live in the *_im arrays (zero for real terms) and
  // the local tables get imaginary parts too (the diagonal is always real)
  int cplx = 0;
  double* coef_im = nullptr;     // [n_terms]
  float2* coef_f_im = nullptr;
  double* fv_d_im = nullptr;     // same indexing as fv_d
  float2* fv_f_im = nullptr;

  // host copies (export, tests)
  std::vector<uint64_t> h_xy, h_yz;
  std::vector<int64_t> h_row_ptr;
  std::vector<double> h_coef, h_coef_im;
  std::vector<uint32_t> h_hash_basis;
  int device = 0;
};

}  // namespace nqs

struct nqs_ham : public nqs::nqs_ham_dev {};

namespace nqs {

// ---------------------------------------------------------------------------
// Batch workspace ("stage") layout: all offsets 256-byte aligned.
// ---------------------------------------------------------------------------
struct StageHeader {
  uint64_t magic;
  int64_t n_unq;
  int64_t cap;          // hash-table buckets of 4 slots (power of two)
  int64_t nwords;       // bloom words (power of two)
  int32_t W;
  int32_t status;       // device status word (kStatus* bits)
  int32_t trie_ok;      // nonzero once the prefix tree of U is built for this staging
  int32_t pad0;
  int64_t off_trie;     // prefix tree of U (LoopOverTrie)
  int64_t off_hx, off_table, off_bloom, off_scan, off_ampP, off_ampQ, off_geff, off_counters;
  int64_t off_own;      // adjoint: each row's own terms, double2 [n_unq]
  int64_t off_q;        // per-qubit sample counts and fill cursors: uint32 [2][64 W]
  int64_t off_qrows;    // per-qubit lists of the samples with that bit set: uint32 [n_unq * n_qubits]
  int64_t off_big;      // rows queued for the block sort: int32 [n_unq]
  int64_t off_rowcur;   // per-row fill cursors: uint64 [n_unq]
  int64_t off_sched, off_order;   // row schedule of the energy and adjoint kernels
  int64_t scan_blocks;
  int64_t total_bytes;
};
constexpr uint64_t kStageMagic = 0x6E71735F73746731ull;
constexpr int64_t kRedOffset = 256;        // E^var reduction scratch: fixed offset in the workspace
constexpr int kRedBlocks = 1024;           // at most this many partial sums
constexpr int64_t kRedBytes = 256 + 3 * 8 * kRedBlocks;

StageHeader stage_layout(const nqs_ham* ham, int64_t n_unq);

// error reporting
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// launchers (defined in the kernel translation units) -------------------------
// staging: clears the membership structures, then hashes, tables, filter and
// per-qubit lists of U (the header must already be in place)
cudaError_t launch_stage(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                         const StageHeader& L, cudaStream_t s);
// the header written into the workspace by a one-thread kernel (the header
// travels as a kernel argument, so the write can be captured in a CUDA graph)
cudaError_t launch_write_header(const StageHeader& L, char* stage, cudaStream_t s);

// launch parameters of the searches, chosen per instance by the batched plan's
// autotuner: LoopOverTerms work items per atomic and search-table groups per
// item; LoopOverTrie node pairs popped per step
struct SearchTune {
  int terms_grab = 4;
  int terms_groups = 16;
  int trie_pop = 32;
  int part = 0;      // LoopOverTerms: search only slice `part` of `n_parts` equal slices of the work items
  int n_parts = 1;
  bool sort_rows = true;  // LoopOverTerms FILL: sort each row by column (else the order the search placed them)
};

// search modes: COUNT writes per-row counts, FILL writes pairs at given CSR
// offsets, EMIT writes per-row counts and the pairs into scratch records,
// EMIT_HALF writes only the records (each unordered pair once, whole batch)
enum SearchMode { kCount = 0, kFill = 1, kEmit = 2, kEmitHalf = 3 };
constexpr uint32_t kNoRecordSlot = 0xFFFFFFFFu;   // i of an unused record slot

struct PairScratch {        // one-pass search scratch (caller memory): found pairs (i, j, k)
  int64_t max_rec;
  int64_t* cursor;          // [2]: records written, overflow flag
  uint32_t* rec_i;          // [max_rec] the sample that found the pair (has the pattern's top qubit)
  uint32_t* rec_j;          // [max_rec] the other sample
  uint32_t* rec_k;          // [max_rec] pattern index
  uint64_t* keys;           // [max_pairs] the range's pairs grouped by row: k << 32 | column
  int64_t max_pairs;
};
int64_t pair_scratch_bytes(int64_t rows, int64_t max_pairs);
PairScratch pair_scratch_view(void* base, int64_t rows, int64_t bytes);

// LoopOverTerms.  COUNT: counts_or_rowptr = per-row counts (rows entries).
// EMIT: the same counts, and the pairs into the scratch (compact afterwards).
// FILL: counts_or_rowptr = CSR offsets; writes and sorts the rows.
cudaError_t launch_pairs_terms(const nqs_ham* ham, const uint64_t* U, char* stage,
                               const StageHeader& L, int64_t row_begin, int64_t row_end,
                               int64_t* counts_or_rowptr, uint32_t* pair_j, uint32_t* pair_k,
                               int mode, const PairScratch* scratch, cudaStream_t s,
                               const SearchTune& tune = SearchTune());

// clear the capacity bit of the status word (stream-ordered)
cudaError_t launch_clear_capacity(char* stage, cudaStream_t s);
// set the capacity bit if rp[rows] - rp[0] > capacity (stream-ordered)
cudaError_t launch_capacity_check(const int64_t* rp, int64_t rows, int64_t capacity, char* stage, cudaStream_t s);

// EMIT records -> CSR rows of [row_begin, row_begin + rows), sorted.  If the
// pairs outgrow `capacity` or the scratch, sets kStatusCapacity and writes nothing.
cudaError_t launch_pairs_compact(const nqs_ham* ham, const PairScratch& sc, char* stage, const StageHeader& L,
                                 int64_t rb, int64_t rows, const int64_t* row_ptr, uint32_t* pair_j,
                                 uint32_t* pair_k, int64_t capacity, cudaStream_t s, bool sort_rows = true);

cudaError_t launch_pairs_batch(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, char* stage,
                               const StageHeader& L, int64_t row_begin, int64_t row_end,
                               int64_t* counts_or_rowptr, uint32_t* pair_j, uint32_t* pair_k,
                               int mode, cudaStream_t s);

// prefix trees (LoopOverTrie)
void build_xy_trie(const std::vector<uint64_t>& xy, int64_t n_xy, int W, std::vector<int32_t>& nodes);
int64_t trie_bytes(int W, int64_t n_unq);
cudaError_t launch_trie_build(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                              const StageHeader& L, cudaStream_t s);
cudaError_t launch_pairs_trie(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage,
                              const StageHeader& L, int64_t row_begin, int64_t row_end,
                              int64_t* counts_or_rowptr, uint32_t* pair_j, uint32_t* pair_k,
                              int mode, cudaStream_t s, const SearchTune& tune = SearchTune());

cudaError_t launch_scan(int64_t* data, int64_t n, char* stage, const StageHeader& L,
                        cudaStream_t s);

// LSD radix sort of W-word keys in numeric order with an int32 payload (k_trie.cu)
int64_t sort_blocks(int64_t n);
int64_t sort_scan_partials(int64_t n);   // ints of the tiled histogram scan for n keys
// exclusive scan of m int32 in place (partial: ceil(m / 2048) + 1 ints when m > 2^18)
cudaError_t launch_scan_i32(int32_t* d, int64_t m, int32_t* partial, cudaStream_t s);
cudaError_t launch_sort_words(const uint64_t* kin, const int32_t* iin, int64_t n, int W, int n_bytes,
                              uint64_t* kbuf[2], int32_t* ibuf[2], int32_t* hist, int32_t* partial, int* out,
                              cudaStream_t s);

// exact local energy over the coupled candidates (k_cand.cu)
int64_t cand_scratch_bytes(const nqs_ham* ham, int64_t n_unq);
cudaError_t launch_full_candidates(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage,
                                   const StageHeader& L, void* scratch, uint32_t* cand_id, double* hval,
                                   uint64_t* cand, int32_t* in_u, int64_t capacity, int64_t* n_cand,
                                   int* limit_hit, cudaStream_t s);
cudaError_t launch_local_energy_full(int64_t n, int64_t n_xy, const char* stage, const StageHeader& L,
                                     const double* a, const double* b, const uint32_t* cand_id, const double* hval,
                                     int64_t n_cand, const double* ca, const double* cb, void* scratch,
                                     double* er, double* ei, cudaStream_t s);

// benchmark timing of the LoopOverTerms search kernel (nqs_search_timing)
void search_timing(bool on);
cudaError_t search_time(double* total_ms, int64_t* launches);

// measured integer speed of light (nqs_probe_peaks): out[0] lane-ops/s of the
// probe's ALU mix, out[1] probes/s of the filter loop alone
cudaError_t probe_peaks(double* out, cudaStream_t s);

// per-sample amplitude records P (factor and exponent, and U's first word when U is given) and Q
cudaError_t launch_amplitudes(const double* a, const double* b, int64_t n, int precision,
                              char* stage, const StageHeader& L, cudaStream_t s, const uint64_t* U);

cudaError_t launch_local_energy(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                                const char* stage, const StageHeader& L, bool cplx,
                                int64_t row_begin, int64_t row_end, const int64_t* row_ptr,
                                const uint32_t* pair_j, const uint32_t* pair_k, int precision,
                                double* eloc_re, double* eloc_im, double* hdiag, void* hpair,
                                cudaStream_t s);

cudaError_t launch_variational_energy(int64_t n, const double* a, const double* eloc_re,
                                      char* work, double* out, cudaStream_t s);
cudaError_t launch_evar_combine(const double* parts, int k, double* out, cudaStream_t s);

// stochastic reconfiguration on the most probable samples (k_sr.cu)
int64_t sr_scratch_bytes(int64_t P);
int64_t sr_top_scratch_bytes(int64_t n);
cudaError_t launch_sr_top(int64_t n, const double* a, int64_t n_sr, int32_t* out, void* scratch, cudaStream_t s);
cudaError_t launch_sr_step(int n, int64_t P, const float* O, const double* a, const double* eloc,
                           const double* evar, double lambda, void* scratch, double* delta, double* T,
                           int32_t* status_out, cudaStream_t s);

// autoregressive sampling without replacement, one qubit (k_sample.cu)
int64_t sample_scratch_bytes(int64_t n_parents);
cudaError_t launch_gumbel_level(int W, int level, int64_t n, const uint64_t* px, const double* pl, const double* plt,
                                const double* logp, const double* G, int64_t K, void* scratch, uint64_t* cx,
                                double* cl, double* clt, int64_t* n_out, cudaStream_t s);
cudaError_t launch_gumbel_level_async(int W, int level, int64_t max_n, const long long* n_dev, const uint64_t* px,
                                      const double* pl, const double* plt, const double* logp, const double* G,
                                      int64_t K, void* scratch, uint64_t* cx, double* cl, double* clt,
                                      long long* counts, cudaStream_t s);
int64_t sample_async_limit();

// half-stored pairs: the records of one EMIT_HALF search (k_half section of k_energy.cu)
cudaError_t launch_find_half(const nqs_ham* ham, const uint64_t* U, char* stage, const StageHeader& L,
                             uint32_t* rec_i, uint32_t* rec_j, uint32_t* rec_k, int64_t capacity,
                             cudaStream_t s, int part = 0, int n_parts = 1);

// Sharded search support.  route: the live records (i != 0xFFFFFFFF) copied to
// the part(s) owning rows i and j (bounds: device [n_parts + 1] row bounds),
// grouped by part at the device offsets off[p] (exclusive prefix of the counts
// that route_count produced); counts are 64-bit.
cudaError_t launch_route_count(const uint32_t* rec_i, const uint32_t* rec_j, int64_t n_slots, const int64_t* bounds,
                               int n_parts, unsigned long long* counts, cudaStream_t s);
cudaError_t launch_route_scatter(const uint32_t* rec_i, const uint32_t* rec_j, const uint32_t* rec_k, int64_t n_slots,
                                 const int64_t* bounds, int n_parts, unsigned long long* cursors, uint32_t* out_i,
                                 uint32_t* out_j, uint32_t* out_k, cudaStream_t s);
// records -> per-row counts of rows [rb, rb + rows): has_diag, plus one for each record naming the row
cudaError_t launch_records_count(const uint32_t* rec_i, const uint32_t* rec_j, int64_t n_rec, int64_t rb,
                                 int64_t rows, int has_diag, int64_t* counts, int32_t* status, cudaStream_t s);
cudaError_t launch_local_energy_half(const nqs_ham* ham, const uint64_t* U, int64_t n, const char* stage,
                                     const StageHeader& L, bool cplx, const uint32_t* ri, const uint32_t* rj,
                                     const uint32_t* rk, int64_t n_slots, int precision, double* er, double* ei,
                                     double* hd, void* hrec, cudaStream_t s);
cudaError_t launch_backward_half(const nqs_ham* ham, const uint64_t* U, int64_t n, char* stage,
                                 const StageHeader& L, bool cplx, const double* a, const uint32_t* ri,
                                 const uint32_t* rj, const uint32_t* rk, int64_t n_slots, const void* hrec,
                                 const double* er, const double* ei, const double* hd, const double* evar,
                                 const double* g_re, const double* g_im, const double* g_evar, int precision,
                                 double* gre, double* gim, cudaStream_t s);

cudaError_t launch_backward(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                            char* stage, const StageHeader& L, bool cplx,
                            const double* a, const double* b,
                            int64_t row_begin, int64_t row_end, const int64_t* row_ptr,
                            const uint32_t* pair_j, const uint32_t* pair_k,
                            const double* eloc_re, const double* eloc_im, const double* hdiag,
                            const double* evar, const double* g_re, const double* g_im,
                            const double* g_evar, int precision, const void* hpair,
                            double* grad_re, double* grad_im, cudaStream_t s);

int num_sms();

}  // namespace nqs
