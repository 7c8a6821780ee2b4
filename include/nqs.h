/*
 * nqs.h -- C ABI of the GB300 (sm_103a) sampled-space local-energy library.
 *
 * The library evaluates, for a batch U of unique sampled basis vectors and a
 * Jordan-Wigner qubit Hamiltonian H = sum_l h_l P^(l) (Eq. jw_hamiltonian),
 *   - the coupled pairs (x, x') in U x U with x XOR x' equal to one of the
 *     Hamiltonian's unique XY patterns (FindCoupledPairs, Sec. "Unique XY"
 *     and Algs. 2A-2C),
 *   - the matrix elements H_xx' (Eq. pauli_melem and the supplementary
 *     algorithm "Calculating the Hamiltonian matrix element"),
 *   - the surrogate local energies E_loc^var(x) = sum_{x' in SC_x}
 *     H_xx' psi(x')/psi(x) (Eq. local_energy restricted to U, Fig.
 *     scatter_local_energies),
 *   - the variational energy E^var (Eq. variational_energy), and
 *   - the vector-Jacobian product of E_loc^var and E^var with respect to
 *     log psi (the adjoint; Eq. grad_def is its special case).
 *
 * Conventions shared by every call
 *   - Bit vectors: an N-qubit vector is W = ceil(N/64) uint64 words; qubit i
 *     is bit (i % 64) of word (i / 64).  A batch is row-major [n][W].
 *     Bits at positions >= N must be zero.
 *   - Pauli strings are given in the symplectic encoding (x, z): qubit i
 *     carries I (0,0), X (1,0), Y (1,1) or Z (0,1).  So the paper's
 *     XY^(l) = x, Y^(l) = x AND z, YZ^(l) = z.
 *   - Amplitudes enter as log psi = a + i b (two real FP64 arrays; b may be
 *     NULL for real, positive amplitudes).
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary host memory.  The caller owns
 *     every buffer it passes; the library never frees caller memory.
 *   - Every call that takes a stream enqueues its kernels on that stream
 *     (cudaStream_t passed as void*; NULL = legacy default stream).  Calls
 *     that return a count to the host synchronise that stream; all others
 *     are asynchronous and perform no host synchronisation.
 *   - Return value: NQS_OK (0) or a negative NQS_ERR_* code.  A failing call
 *     leaves caller buffers unspecified but valid; nqs_last_error() gives a
 *     thread-local message.  No call aborts the process or traps the GPU:
 *     device-side problems (repeated samples, bounded loops running out) are
 *     recorded in a status word and reported by the next synchronising call
 *     or by nqs_stage_status().
 *   - Scope: real coefficients h_l; strings with an odd number of Y make H
 *     complex Hermitian (coefficient h_l i^{|Y|} imaginary), and then the
 *     local energies are complex (eloc_im required); molecular Hamiltonians
 *     are real.  Complex log psi is supported; 1 <= N <= 256.  The batched
 *     plan and the exact local energy (nqs_full_candidates) take real
 *     Hamiltonians only.
 */
#ifndef NQS_H
#define NQS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NQS_VERSION 100

enum {
    NQS_OK = 0,
    NQS_ERR_ARG = -1,          /* bad argument (null pointer, size, range)          */
    NQS_ERR_UNSUPPORTED = -2,  /* outside the scope above (N > 256, ...)            */
    NQS_ERR_CUDA = -3,         /* a CUDA runtime call failed                        */
    NQS_ERR_CAPACITY = -4,     /* output buffer too small; required size returned  */
    NQS_ERR_DUPLICATE = -5,    /* the sample batch repeats a basis vector           */
    NQS_ERR_DEVICE_LIMIT = -6, /* a bounded device loop ran out, or a device index
                                  check failed and the access was skipped
                                  (corrupt input or pair list)                     */
    NQS_ERR_OOM = -7,          /* device allocation inside nqs_ham_load failed      */
    NQS_ERR_RANGE = -8         /* an amplitude ratio leaves the FP32 exponent range,
                                  or a term of a local-energy or adjoint row sum
                                  reaches 2^55 in magnitude                        */
};

enum {
    NQS_SCHED_AUTO = 0,   /* library's choice                                      */
    NQS_SCHED_TERMS = 1,  /* loop over unique XY per sample (Alg. 2A)               */
    NQS_SCHED_BATCH = 2,  /* loop over the batch per sample (Alg. 2B)               */
    NQS_SCHED_TRIE = 3,   /* joint prefix-tree traversal (Algs. 3 and 2C)          */
    /* Flag OR-ed into the schedule of nqs_find_coupled_pairs and
     * nqs_fill_coupled_pairs: leave each LoopOverTerms row (after its leading
     * diagonal pair) in the order the search placed its pairs, which depends
     * on thread timing, instead of ascending column order.  The set of pairs
     * of every row is the same; the row sort is skipped.  nqs_local_energy
     * and nqs_local_energy_backward sum every row exactly, so their results
     * are bitwise the same for either order.  Ignored by the other schedules
     * (their rows come out in column order). */
    NQS_ROWS_UNSORTED = 0x100
};

enum {
    NQS_PREC_FP64 = 0,    /* FP64 arithmetic throughout                             */
    NQS_PREC_FP32C = 1    /* FP32 with compensated (double-float) accumulation;     */
                          /* FP64 for the final energy reduction                    */
};

typedef struct nqs_ham nqs_ham;

/* ---------------------------------------------------------------------------
 * Hamiltonian (Sec. "Preparation", Fig. ham_prep; Eq. xy_to_yz_set)
 * ------------------------------------------------------------------------- */

/* Copy n_terms Pauli strings to the current device, grouped by XY pattern.
 *   x_mask, z_mask : host, [n_terms][W] uint64, symplectic encoding.
 *   coef           : host, [n_terms] FP64 real coefficients h_l.
 * Identical strings are merged (coefficients summed); terms whose merged
 * coefficient is exactly zero are dropped.  A string with an odd number of
 * Y gets the imaginary coefficient h_l i^{|Y|} (Eq. pauli_melem) and makes
 * the Hamiltonian complex (nqs_ham_is_complex).  Errors: NQS_ERR_ARG
 * (n_qubits out of range, bits >= N set, null pointer),
 * NQS_ERR_UNSUPPORTED (N > 256), NQS_ERR_OOM, NQS_ERR_CUDA.  On success
 * *out owns the device tables until nqs_ham_free. */
int nqs_ham_load(int n_qubits, int64_t n_terms, const uint64_t* x_mask,
                 const uint64_t* z_mask, const double* coef, nqs_ham** out);

/* Release the tables of nqs_ham_load (NULL is accepted). */
int nqs_ham_free(nqs_ham* ham);

/* Sizes after merging: info[0] = N, [1] = W, [2] = terms, [3] = unique XY
 * patterns, [4] = 1 if the XY = 0 (diagonal) pattern exists, [5] = size of
 * the largest P_XY, [6] = number of search-table slots (with padding). */
int nqs_ham_info(const nqs_ham* ham, int64_t info[8]);

/* Host copy of the grouped tables (any pointer may be NULL):
 *   xy      [n_xy][W]   unique XY patterns, in library order
 *   row_ptr [n_xy+1]    P_XY of pattern m = terms row_ptr[m] .. row_ptr[m+1]-1
 *   yz      [terms][W]  YZ^(l) (= z mask) per grouped term
 *   coef    [terms]     real part of h_l * i^{|Y^(l)|} (zero if |Y| is odd)   */
int nqs_ham_export(const nqs_ham* ham, uint64_t* xy, int64_t* row_ptr,
                   uint64_t* yz, double* coef);

/* 1 if some string has an odd number of Y (complex H), else 0 (also for NULL). */
int nqs_ham_is_complex(const nqs_ham* ham);

/* Imaginary parts of the grouped coefficients h_l * i^{|Y^(l)|}, host
 * [terms] in the order of nqs_ham_export (zero for even |Y|). */
int nqs_ham_export_im(const nqs_ham* ham, double* coef_im);

/* ---------------------------------------------------------------------------
 * Batch workspace and sample staging: the membership structure of U used by
 * the test "x' in U" of Algs. 2A-2C (Sec. "Unique XY"), plus per-sample
 * scratch used by the energy and adjoint calls.
 * ------------------------------------------------------------------------- */

/* Bytes of the batch workspace for n_unq samples (device memory, 256-byte
 * aligned, caller-owned; one workspace per batch and stream). */
int64_t nqs_stage_bytes(const nqs_ham* ham, int64_t n_unq);

/* Build the membership structure of U (device [n_unq][W]) in work.  U must
 * stay unchanged while the workspace is in use.  If check != 0 the call
 * synchronises the stream and returns NQS_ERR_DUPLICATE if U repeats a
 * vector, NQS_ERR_ARG if a sample has bits >= N.  With check == 0 it is
 * asynchronous and the same conditions are reported by nqs_stage_status(). */
int nqs_stage(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
              int64_t work_bytes, int check, void* stream);

/* Build the prefix tree of U (Alg. 3, Sec. "Prefix tree construction") in
 * the workspace of an nqs_stage call with the same U, for searches with
 * NQS_SCHED_TRIE.  Levels follow the qubit index; the tree is stored as U
 * sorted in qubit order with, per position, the levels where the run it
 * starts branches (see the implementation notes).  Needs n_qubits <= 255 and
 * n_unq < 2^23 (NQS_ERR_UNSUPPORTED otherwise).  Every nqs_stage call
 * invalidates the tree; a trie search on a workspace without one records
 * an error that the search call (or nqs_stage_status) returns as
 * NQS_ERR_ARG.  Asynchronous. */
int nqs_stage_trie(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                   void* stream);

/* Synchronise the stream and return the workspace's status: NQS_OK or the
 * first of NQS_ERR_DUPLICATE, NQS_ERR_ARG (bits >= N), NQS_ERR_DEVICE_LIMIT,
 * NQS_ERR_RANGE recorded by device code since nqs_stage. */
int nqs_stage_status(const void* work, void* stream);

/* ---------------------------------------------------------------------------
 * FindCoupledPairs (Sec. "FindCoupledPairs implementations")
 * Output: CSR over the rows [row_begin, row_end) of U:
 *   row_ptr[r - row_begin] .. row_ptr[r - row_begin + 1] - 1 index the pairs
 *   of row r; pair_j = column (index into U), pair_k = pattern index (into
 *   the library's unique-XY table).  Within a row the diagonal pair comes
 *   first (if the XY = 0 pattern exists), then the others in an order fixed
 *   by the schedule and the row alone: it depends neither on the row range
 *   nor on the call (count, fill and one-pass calls agree).  LoopOverTerms
 *   lists them by ascending column.  Both (i, j) and (j, i) are listed.
 *   NQS_SCHED_TRIE needs nqs_stage_trie after nqs_stage.
 * All calls need a workspace staged with the same U.  Readers of the CSR
 * (fill, energy, adjoint) take positions relative to row_ptr[0], so a slice
 * row_ptr + (r0 - row_begin) of a larger offset array can be passed for the
 * sub-range [r0, r1) together with pair arrays that start at that slice's
 * first pair.
 * ------------------------------------------------------------------------- */

/* Count pass: row_ptr (device int64 [row_end-row_begin+1]) receives the CSR
 * offsets, *n_pairs (host) the total.  Synchronises the stream; returns the
 * workspace status if device code recorded a problem. */
int nqs_count_coupled_pairs(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                            void* work, int64_t row_begin, int64_t row_end,
                            int schedule, int64_t* row_ptr, int64_t* n_pairs,
                            void* stream);

/* Fill pass for offsets from nqs_count_coupled_pairs with the same arguments:
 * pair_j, pair_k device uint32 [row_ptr[last]] (schedule may carry
 * NQS_ROWS_UNSORTED).  Asynchronous. */
int nqs_fill_coupled_pairs(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                           void* work, int64_t row_begin, int64_t row_end,
                           int schedule, const int64_t* row_ptr, uint32_t* pair_j,
                           uint32_t* pair_k, void* stream);

/* Bytes of the scratch that nqs_find_coupled_pairs needs to list up to
 * max_pairs pairs of `rows` rows in one pass. */
int64_t nqs_pairs_scratch_bytes(int64_t rows, int64_t max_pairs);

/* One search pass.  The pairs are written to scratch (device, 256-byte
 * aligned, scratch_bytes from nqs_pairs_scratch_bytes) while the rows are
 * counted, then copied in CSR order (each row sorted by column unless the
 * schedule carries NQS_ROWS_UNSORTED) to pair_j/pair_k (device uint32,
 * `capacity` entries).  The call waits until the count is known (the total
 * is returned in *n_pairs); the copy into pair_j/pair_k may still be running
 * on the stream when it returns (later work on the stream sees it done).
 * If the scratch or `capacity` is too small the call returns
 * NQS_ERR_CAPACITY with row_ptr and *n_pairs valid and pair_j/pair_k
 * unwritten; nqs_fill_coupled_pairs with the same row_ptr then completes the
 * list.  scratch == NULL selects the two-pass form (count, then fill). */
int nqs_find_coupled_pairs(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                           void* work, int64_t row_begin, int64_t row_end,
                           int schedule, void* scratch, int64_t scratch_bytes,
                           int64_t* row_ptr, uint32_t* pair_j, uint32_t* pair_k,
                           int64_t capacity, int64_t* n_pairs, void* stream);

/* The same search without any host wait (Sec. "FindCoupledPairs
 * implementations", Alg. 2A; Algs. 2B/2C through count + fill): every step is
 * enqueued on `stream` and the call returns at once, so a whole energy step
 * can be enqueued (or captured in a CUDA graph) without a round trip.  The
 * pair total stays on the device in row_ptr[row_end - row_begin].  pair_j,
 * pair_k: device uint32 [capacity], sized by the caller (for example from an
 * earlier batch's count).  With scratch (LoopOverTerms) the one-pass search is
 * used, else count, then fill.  If the pairs outgrow `capacity` or the
 * scratch, nothing is written to pair_j/pair_k, the workspace's capacity bit
 * is set, and later nqs_local_energy / nqs_local_energy_backward calls on the
 * workspace skip their rows; nqs_stage_status then returns NQS_ERR_CAPACITY
 * (row_ptr is valid: size the buffers from it and call again).  The capacity
 * bit is cleared at the start of every call.  Schedule flags as for
 * nqs_find_coupled_pairs.  Packed form: with pair_k == NULL, LoopOverTerms
 * with scratch and NQS_ROWS_UNSORTED, each pair is one 64-bit word
 * (column << 32 | pattern) in pair_j (8-byte aligned, `capacity` words), the
 * layout nqs_local_energy and nqs_local_energy_backward accept with
 * pair_k == NULL; it skips the pass that splits the words into two arrays.
 * Argument errors are returned at once. */
int nqs_find_coupled_pairs_async(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                                 void* work, int64_t row_begin, int64_t row_end,
                                 int schedule, void* scratch, int64_t scratch_bytes,
                                 int64_t* row_ptr, uint32_t* pair_j, uint32_t* pair_k,
                                 int64_t capacity, void* stream);

/* ---------------------------------------------------------------------------
 * Half-stored pairs (Sec. "FindCoupledPairs implementations", Alg. 2A; the
 * symmetry x XOR x' = XY of Eq. pauli_melem): each unordered coupled pair
 * {U_i, U_j}, i != j, found once by the oriented LoopOverTerms search and
 * written as one record (i, j, k), k the XY pattern index, instead of once
 * in each of its two rows.
 * ------------------------------------------------------------------------- */

/* Records of every unordered pair of the batch: rec_i/rec_j/rec_k device
 * uint32 [capacity].  *n_slots (host) = record slots used; a slot whose
 * rec_i is 0xFFFFFFFF is unused (the search hands out slots in chunks), and
 * the order of the records depends on thread timing.  NQS_ERR_CAPACITY if
 * `capacity` is too small (*n_slots then gives the slots asked for).
 * Synchronises the stream. */
int nqs_find_pairs_half(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                        uint32_t* rec_i, uint32_t* rec_j, uint32_t* rec_k, int64_t capacity,
                        int64_t* n_slots, void* stream);

/* The same search restricted to slice `part` of `n_parts` equal slices of
 * the oriented work items (sample-list batch x pattern groups): the slices
 * of parts 0 .. n_parts-1 together list every unordered pair exactly once,
 * so n_parts ranks (one GPU each, each holding the whole staged batch)
 * search disjoint slices.  part 0 of 1 is nqs_find_pairs_half. */
int nqs_find_pairs_part(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                        int part, int n_parts, uint32_t* rec_i, uint32_t* rec_j,
                        uint32_t* rec_k, int64_t capacity, int64_t* n_slots, void* stream);

/* Scratch bytes of nqs_route_records (n_parts in [1, 1024]). */
int64_t nqs_route_scratch_bytes(int n_parts);

/* The exchange step of the sharded search: part p owns rows
 * [bounds[p], bounds[p + 1]) (host int64 [n_parts + 1], bounds[0] = 0,
 * ascending).  Every used record slot of rec_i/rec_j/rec_k ([n_slots], from
 * nqs_find_pairs_part) is copied to out_i/out_j/out_k (device uint32
 * [capacity]) once for the part owning row i and once more for the part
 * owning row j if that is another part; the copies are grouped by part in
 * part order (order within a part unspecified), and counts[p] (host int64
 * [n_parts]) receives each part's number.  These groups are what an
 * all-to-all exchange sends to each rank.  scratch: device, 256-byte
 * aligned, nqs_route_scratch_bytes.  NQS_ERR_CAPACITY if the copies exceed
 * `capacity` (counts are then valid).  Synchronises the stream. */
int nqs_route_records(int n_parts, const int64_t* bounds, const uint32_t* rec_i,
                      const uint32_t* rec_j, const uint32_t* rec_k, int64_t n_slots,
                      uint32_t* out_i, uint32_t* out_j, uint32_t* out_k, int64_t capacity,
                      int64_t* counts, void* scratch, int64_t scratch_bytes, void* stream);

/* CSR pairs of rows [row_begin, row_end) from records (device uint32 [n_rec];
 * unused slots 0xFFFFFFFF allowed) that include every unordered pair with an
 * endpoint in the range, e.g. the records a rank received from the exchange:
 * row_ptr, pair_j, pair_k exactly as nqs_find_coupled_pairs writes them for
 * that range (diagonal pair first, then ascending column).  A pair listed
 * by several records is listed that often.  scratch: device, 256-byte
 * aligned, at least 256 + 8 * (pairs of the range) bytes.  *n_pairs (host)
 * = pairs of the range; NQS_ERR_CAPACITY if they exceed `capacity` or the
 * scratch (row_ptr and *n_pairs then valid).  Synchronises the stream. */
int nqs_pairs_from_records(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                           const uint32_t* rec_i, const uint32_t* rec_j, const uint32_t* rec_k,
                           int64_t n_rec, int64_t row_begin, int64_t row_end, void* scratch,
                           int64_t scratch_bytes, int64_t* row_ptr, uint32_t* pair_j,
                           uint32_t* pair_k, int64_t capacity, int64_t* n_pairs, void* stream);

/* E_loc^var of every sample from half-stored records (n_slots slots): the
 * diagonal term per row, then one MatrixElement per record, whose two terms
 * (row i with column j, row j with column i, the latter with
 * H_ji = conj(H_ij)) are added to eloc[i] and eloc[j] by FP64 atomic
 * addition (row sums equal the CSR path's to rounding, not bitwise).
 * Arguments as nqs_local_energy over the whole batch (eloc_re, eloc_im,
 * hdiag device FP64 [n_unq]); hrec: per-record H (layout of hpair, indexed
 * by slot) or NULL.  Asynchronous. */
int nqs_local_energy_half(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                          const double* logpsi_re, const double* logpsi_im, const uint32_t* rec_i,
                          const uint32_t* rec_j, const uint32_t* rec_k, int64_t n_slots,
                          int precision, double* eloc_re, double* eloc_im, double* hdiag,
                          void* hrec, void* stream);

/* Adjoint over half-stored records: the gradient of nqs_local_energy_backward
 * (same upstreams, closed form when both g_eloc arrays are NULL) for every
 * sample, each record's two terms added by FP64 atomic addition.  hrec: as
 * written by nqs_local_energy_half, or NULL to recompute.  Asynchronous. */
int nqs_local_energy_backward_half(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                                   void* work, const double* logpsi_re, const double* logpsi_im,
                                   const uint32_t* rec_i, const uint32_t* rec_j,
                                   const uint32_t* rec_k, int64_t n_slots, const void* hrec,
                                   const double* eloc_re, const double* eloc_im,
                                   const double* hdiag, const double* evar,
                                   const double* g_eloc_re, const double* g_eloc_im,
                                   const double* g_evar, int precision, double* grad_re,
                                   double* grad_im, void* stream);

/* ---------------------------------------------------------------------------
 * MatrixElement + ScatterAdd -> E_loc^var (Sec. "MatrixElement
 * implementation", Fig. scatter_local_energies)
 * ------------------------------------------------------------------------- */

/* For rows r in [row_begin, row_end), with their pairs from a fill pass over
 * the same range (pair_j/pair_k, or pair_k == NULL and pair_j holding the
 * packed 64-bit words of nqs_find_coupled_pairs_async), write
 *   eloc_re[r], eloc_im[r] = E_loc^var(U_r)  (eloc_im may be NULL only if
 *                                              logpsi_im is NULL and H is real),
 *   hdiag[r] = H_{U_r U_r} (may be NULL; real for any Hermitian H),
 *   hpair[q] = H of pair q, q indexing pair_j/pair_k (may be NULL): device
 *              float2 (hi, lo) per pair with NQS_PREC_FP32C, double with
 *              NQS_PREC_FP64; for a complex H both parts, float4 (re hi,
 *              re lo, im hi, im lo) or double2 per pair (16-byte aligned);
 *              nqs_local_energy_backward can read it instead of recomputing
 *              the matrix elements.
 * logpsi_re/_im: device FP64 [n_unq] for the whole batch.  Each row's terms
 * (H times the amplitude ratio, in the precision chosen) are cut to whole
 * units of 2^-64 (an error below 2^-64 per term), summed exactly as signed
 * 128-bit integers and rounded to FP64 once, so a row's result does not
 * depend on the order of its pairs (sorted
 * or NQS_ROWS_UNSORTED), on which thread took which pair, or on the order in
 * which rows are handed out; results are bitwise reproducible.  A term of
 * magnitude 2^55 or more is dropped and NQS_ERR_RANGE is recorded.
 * The call overwrites the per-sample scratch of work.  Asynchronous. */
int nqs_local_energy(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                     const double* logpsi_re, const double* logpsi_im,
                     int64_t row_begin, int64_t row_end, const int64_t* row_ptr,
                     const uint32_t* pair_j, const uint32_t* pair_k, int precision,
                     double* eloc_re, double* eloc_im, double* hdiag, void* hpair,
                     void* stream);

/* ---------------------------------------------------------------------------
 * Autoregressive sampling without replacement (Alg. 1, ARGumbelTopK; Sec.
 * "Autoregressive sampling without replacement"): the producer of the
 * unique batch U.  One call per qubit; the caller's ansatz supplies the
 * conditional log-probabilities between calls.
 * ------------------------------------------------------------------------- */

/* Bytes of the scratch of nqs_gumbel_topk_level for n_parents kept vectors. */
int64_t nqs_gumbel_scratch_bytes(int64_t n_parents);

/* Qubit `level` of Alg. 1.  The n_parents kept vectors x_<level (device
 * uint64 [n_parents][W], W = ceil(n_qubits / 64); may be NULL at level 0,
 * meaning the empty vector), their log-probabilities l and conditioned
 * perturbed log-probabilities L~ (device FP64 [n_parents]; 0 and 0 for the
 * empty vector), the conditional log-probabilities log p_level(x | x_<level)
 * for x = 0, 1 (device FP64 [n_parents][2]; -inf for an impossible outcome)
 * and the Gumbel(0) draws G (device FP64 [n_parents][2]) give the extensions
 * l' = l + log p, L' = l' + G, Z = max(L'_0, L'_1),
 * L~' = -log(exp(-L~) - exp(-Z) + exp(-L')) (evaluated as L~' = L~ for the
 * larger extension and L~ - softplus(L~ - Z + log(expm1(Z - L'))) for the
 * other: the same value without the cancellation).  The extensions with l' > -inf
 * are ordered by L~' descending (stable: ties keep the parent order, x = 0
 * first) and the first min(K, possible) are written to child_x [..][W],
 * child_l, child_lt (device, room for min(K, 2 n_parents)); *n_children
 * (host) is their number.  FP64 throughout.  Ordering: the extensions go to
 * buckets between splitters drawn from a sample of their keys and each bucket
 * is sorted by (L~', extension index) in one block's shared memory; when a
 * bucket would exceed 2048 extensions (many equal values) an LSD radix sort
 * of all keys is used instead.  The result is the same either way.
 * scratch: device, 256-byte aligned, nqs_gumbel_scratch_bytes(n_parents).
 * Synchronises the stream (to learn the count).  The paper's own
 * contribution is the use of this sampler (Ref. on ancestral Gumbel top-k
 * sampling); the kernel is this library's. */
int nqs_gumbel_topk_level(int n_qubits, int level, int64_t n_parents, const uint64_t* parent_x,
                          const double* parent_l, const double* parent_lt, const double* cond_logp,
                          const double* gumbel, int64_t K, void* scratch, int64_t scratch_bytes,
                          uint64_t* child_x, double* child_l, double* child_lt, int64_t* n_children,
                          void* stream);

/* Largest max_parents nqs_gumbel_topk_level_async takes (262144). */
int64_t nqs_gumbel_async_max_parents(void);

/* The same level with the parent count held on the device, for a run of
 * levels enqueued (or captured in a CUDA graph) without a host round trip:
 * *n_parents (device int64, at most max_parents) is the number of parents;
 * parent_l, parent_lt, cond_logp, gumbel and the child arrays are sized for
 * max_parents (room for min(K, 2 max_parents) children); counts (device
 * int64 [2]) receives the kept count and a status: 1 when done, 0 when a
 * bucket would exceed 2048 extensions (then nothing is kept, so later levels
 * that read this count start from no parents; repeat the run with
 * nqs_gumbel_topk_level).  Pass the previous level's counts as the next
 * level's n_parents.  scratch: nqs_gumbel_scratch_bytes(max_parents).  Does
 * not synchronise; errors of the arguments are returned at once. */
int nqs_gumbel_topk_level_async(int n_qubits, int level, int64_t max_parents, const int64_t* n_parents,
                                const uint64_t* parent_x, const double* parent_l, const double* parent_lt,
                                const double* cond_logp, const double* gumbel, int64_t K, void* scratch,
                                int64_t scratch_bytes, uint64_t* child_x, double* child_l, double* child_lt,
                                int64_t* counts, void* stream);

/* ---------------------------------------------------------------------------
 * Stochastic reconfiguration on the most probable samples (Sec. "ANQS-
 * tailored stochastic reconfiguration", Eq. qgt_definition), min-SR form.
 * ------------------------------------------------------------------------- */

/* Scratch bytes of nqs_sr_top (n_unq samples) and nqs_sr_step (n_params). */
int64_t nqs_sr_scratch_bytes(int64_t n_unq, int64_t n_params);

/* Indices (device int32 [n_sr]) of the n_sr samples of highest probability
 * p = |psi|^2, i.e. largest logpsi_re (device FP64 [n_unq]); equal values in
 * index order.  Asynchronous. */
int nqs_sr_top(int64_t n_unq, const double* logpsi_re, int64_t n_sr, int32_t* idx, void* scratch,
               int64_t scratch_bytes, void* stream);

/* The regularised SR step for n_sr <= 128 samples with real log-derivatives
 * O = d log psi(x) / d theta (device FP32 [n_sr][n_params], row-major):
 *   w = p / sum p over the n_sr samples (p = exp(2 logpsi_re)),
 *   m = sum_x w_x O_x,  Obar_x = sqrt(w_x) (O_x - m)   (so S = Obar^T Obar
 *   is the QGT estimate of Eq. qgt_definition with renormalised weights),
 *   T = Obar Obar^T, eps_x = sqrt(w_x) (eloc_re[x] - evar[0]),
 *   delta = Obar^T (T + lambda I)^{-1} eps   (device FP64 [n_params]),
 *   T (device FP64 [n_sr][n_sr], may be NULL) receives Obar Obar^T.
 * logpsi_re, eloc_re: device FP64 [n_sr]; evar: device FP64 [1].  T is
 * formed on the tensor cores (tcgen05, bf16 hi/lo split of Obar with FP32
 * accumulation: about 16 significant bits per element), summed in FP64 and
 * solved by an L D L^T factorisation in double-float arithmetic (about 48
 * significant bits).  The solve adds c sqrt(w) sqrt(w)^T (c = tr T / n_sr)
 * to T + lambda I: sqrt(w) is a null vector of the exact T and the step
 * annihilates it, so delta is unchanged while the factorisation no longer
 * sees an eigenvalue of lambda along it.  n_params a multiple of 4 (and O,
 * delta 16-byte aligned) takes the streamed kernels (tensor copies of O).
 * Synchronises the stream.  Errors: NQS_ERR_RANGE if a pivot of that matrix
 * is not positive (raise lambda),
 * NQS_ERR_DEVICE_LIMIT if a tensor-core pipeline wait ran out. */
int nqs_sr_step(int n_sr, int64_t n_params, const float* O, const double* logpsi_re, const double* eloc_re,
                const double* evar, double lambda, double* delta, double* T, void* scratch, int64_t scratch_bytes,
                void* stream);

/* ---------------------------------------------------------------------------
 * Exact local energy (Eq. local_energy): the sum over every x' with
 * H_xx' != 0, inside or outside the batch.  Term l couples x to x' exactly
 * when x XOR x' = XY^(l) (Eq. pauli_melem), so the candidates of x are
 * x XOR XY_k for the k = 0 .. n_xy-1 unique XY patterns of the loaded
 * Hamiltonian (library order, nqs_ham_export).  Every sample has exactly
 * n_xy candidate entries, e = i * n_xy + k, whose matrix element may be zero
 * (a pattern whose terms cancel on x).  The ansatz is evaluated once per
 * distinct candidate; the paper's surrogate E_loc^var (Sec. "Streamlined
 * local energy calculations") keeps only the candidates that lie in U.
 * ------------------------------------------------------------------------- */

/* Bytes of the scratch nqs_full_candidates needs for n_unq samples (about
 * 13 + 16 W bytes per entry and at least 32, n_unq * n_xy entries: the keys
 * and entry indices of a radix sort, its histograms, the candidate marks). */
int64_t nqs_candidates_scratch_bytes(const nqs_ham* ham, int64_t n_unq);

/* Candidates of every sample of U (device [n_unq][W]; staged in `work`):
 *   cand_id  device uint32 [n_unq][n_xy]: index of x_i XOR XY_k in `cand`;
 *   hval     device FP64 [n_unq][n_xy] or NULL: H_{x_i, x_i XOR XY_k} (the
 *            MatrixElement forms of nqs_local_energy, FP64);
 *   cand     device uint64 [capacity][W]: the distinct candidates of the
 *            whole batch in increasing numeric order (qubit 0 the least
 *            significant bit); *n_cand (host) their number;
 *   cand_in_u device int32 [capacity] or NULL: the candidate's index in U,
 *            or -1 if it is not a sample of the batch.
 * scratch: device, 256-byte aligned, scratch_bytes >= nqs_candidates_scratch_bytes.
 * Needs n_unq * n_xy <= 2^29.  The candidates are deduplicated by a radix
 * sort of all entries' keys.  Synchronises the stream (to learn *n_cand and
 * the membership probe's status).  NQS_ERR_CAPACITY (with *n_cand set, cand unwritten) if
 * capacity < *n_cand or cand is NULL; the call can be repeated with larger
 * buffers.  The candidate order and every index are independent of thread
 * timing. */
int nqs_full_candidates(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                        void* scratch, int64_t scratch_bytes, uint32_t* cand_id, double* hval,
                        uint64_t* cand, int32_t* cand_in_u, int64_t capacity, int64_t* n_cand,
                        void* stream);

/* E_loc(x_i) = sum_k H_{x_i, x_k} psi(x_k) / psi(x_i) over the candidate
 * entries of nqs_full_candidates (Eq. local_energy), FP64, one fixed-order
 * reduction per sample.  logpsi_re/_im: device [n_unq] for U (im may be
 * NULL); cand_logpsi_re/_im: device [n_cand] for the candidates in the
 * order of `cand` (im may be NULL; a candidate with psi = 0 may pass a very
 * negative log, its contributions underflow to zero).  scratch: device,
 * 256-byte aligned, >= 32 * n_cand bytes (the nqs_full_candidates scratch
 * qualifies).  eloc_im needed when either imaginary part is given.  The
 * per-sample amplitude records of `work` are overwritten.  A candidate index
 * out of range is skipped and reported by nqs_stage_status as
 * NQS_ERR_DEVICE_LIMIT.  Asynchronous. */
int nqs_local_energy_full(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                          const double* logpsi_re, const double* logpsi_im, const uint32_t* cand_id,
                          const double* hval, int64_t n_cand, const double* cand_logpsi_re,
                          const double* cand_logpsi_im, void* scratch, int64_t scratch_bytes,
                          double* eloc_re, double* eloc_im, void* stream);

/* E^var = sum_x p(x) Re E_loc^var(x) / sum_x p(x) with p = exp(2 a) over the
 * whole batch (Eq. variational_energy), FP64, deterministic (fixed block
 * partition and summation order).  work: a batch workspace that nqs_stage
 * has initialised (its reduction scratch is used; calls sharing one
 * workspace must not overlap).  Writes out[0] = E^var, out[1] = max a,
 * out[2] = sum_x exp(2 (a - max a)) (device FP64 [3]).  Asynchronous. */
int nqs_variational_energy(int64_t n_unq, const double* logpsi_re, const double* eloc_re,
                           void* work, double* out, void* stream);

/* Same result as nqs_variational_energy, for callers that cannot allocate
 * device memory: for instance code whose device memory is entirely owned by
 * another allocator, or that must not make the device-wide synchronising
 * allocation calls on its hot path.  It allocates nothing (no cudaMalloc,
 * cudaFree or library allocation) and needs no workspace: its partial sums
 * live in one fixed device array of the library (about 24 KB, kept by every
 * device that loads the library until the process exits).
 *   n_unq <= 2097152 (2048 samples for each of the array's 1024 slots);
 *   larger batches return NQS_ERR_CAPACITY and launch nothing.
 * The first call on a device looks up the array's device address (a
 * one-time set-up per device, cached by device index); make that first call
 * before any stream capture.  `stream` must belong to the current device
 * (the address is taken for the current device).  The cached addresses do
 * not survive cudaDeviceReset: a process that resets a device must not call
 * this entry point again afterwards.  Every call uses the same array: calls that overlap on the GPU
 * (different streams, or different host threads, at the same time) race and
 * corrupt each other's result, so serialise them.  The paper has no
 * counterpart to this entry point.  Asynchronous. */
int nqs_variational_energy_noalloc(int64_t n_unq, const double* logpsi_re,
                                   const double* eloc_re, double* out, void* stream);

/* E^var of a batch whose rows are split into k blocks (one per GPU when the
 * rows are sharded across ranks), from the k triples that
 * nqs_variational_energy wrote for the blocks (each called on its block's
 * slices of logpsi_re and eloc_re).  With m = max_r max_r and
 * f_r = exp(2 (max_r - m)) (Eq. variational_energy, weights |psi|^2):
 *   out[1] = m,  out[2] = sum_r sum_r f_r,  out[0] = sum_r E_r sum_r f_r / out[2].
 * Blocks with a zero weight sum (empty) are skipped.  The result can be
 * passed as `evar` to nqs_local_energy_backward for any block.
 * nqs_evar_combine: device parts [k][3] and out [3], asynchronous.
 * nqs_evar_combine_host: the same on host arrays (synchronous). */
int nqs_evar_combine(const double* parts, int k, double* out, void* stream);
int nqs_evar_combine_host(const double* parts, int k, double* out);

/* ---------------------------------------------------------------------------
 * Adjoint: gradient of L = sum_x [g_re(x) Re E_loc(x) + g_im(x) Im E_loc(x)]
 *          + g_evar E^var with respect to (Re log psi, Im log psi).
 * For rows y in [row_begin, row_end) (pairs of those rows, as two arrays or,
 * with pair_k == NULL, packed in pair_j as for nqs_local_energy) writes
 * grad_re[y], grad_im[y] (grad_im may be NULL if logpsi_im is NULL).
 *   eloc_re/_im, hdiag: the forward results for the WHOLE batch.
 *   evar: device FP64 [3] from nqs_variational_energy.
 *   g_eloc_re/_im: device FP64 [n_unq] or NULL (zero upstream).
 *   g_evar: device FP64 [1] or NULL (zero).
 *   hpair: the per-pair matrix elements stored by nqs_local_energy for the
 *          same pairs and precision, or NULL to recompute them (same bits).
 * With both g_eloc arrays NULL no pair data is read (row_ptr may be NULL)
 * and the result is the closed form 2 w_y (E_loc(y) - E) g_evar.  The sum
 * over x of each pair (x, y) is evaluated on row y, which lists the same
 * pairs because x XOR y is symmetric; it uses H_xy = conj(H_yx) (H
 * Hermitian; equal for a real H).  A complex H needs eloc_im.
 * Asynchronous. */
int nqs_local_energy_backward(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                              void* work, const double* logpsi_re, const double* logpsi_im,
                              int64_t row_begin, int64_t row_end, const int64_t* row_ptr,
                              const uint32_t* pair_j, const uint32_t* pair_k,
                              const void* hpair,
                              const double* eloc_re, const double* eloc_im,
                              const double* hdiag, const double* evar,
                              const double* g_eloc_re, const double* g_eloc_im,
                              const double* g_evar, int precision,
                              double* grad_re, double* grad_im, void* stream);

/* ---------------------------------------------------------------------------
 * Batched instances: many independent (Hamiltonian, sample batch) problems
 * of uneven size evaluated by one CUDA-graph launch (forward path: staging,
 * FindCoupledPairs, E_loc^var, E^var for every instance).  The paper runs one
 * instance at a time; its schedule comparison (Sec. "FindCoupledPairs
 * implementations", LoopOverTerms vs LoopOverBatch) motivates choosing the
 * schedule per instance.
 * ------------------------------------------------------------------------- */
typedef struct nqs_plan nqs_plan;

typedef struct {
    const nqs_ham* ham;       /* loaded Hamiltonian (its device)                    */
    const uint64_t* U;        /* device [n_unq][W]; contents may change between runs */
    int64_t n_unq;            /* fixed for the plan's lifetime                        */
    const double* logpsi_re;  /* device [n_unq] (real amplitudes)                    */
    double* eloc_re;          /* device [n_unq] output E_loc^var                      */
    double* evar;             /* device [3] output as nqs_variational_energy          */
    double* grad;             /* device [n_unq] output dE^var / d Re log psi, or NULL */
} nqs_instance;

/* Plan n_inst instances (arrays are read during the call; the pointers inside
 * must stay valid for the plan's lifetime).  Planning stages every instance,
 * counts its pairs, picks its schedule and launch parameters (flags bit 0:
 * time the count pass of LoopOverTerms with 2/4/8 work items per atomic and
 * 8/16/32 table groups per item, LoopOverBatch, and LoopOverTrie (with its
 * prefix-tree build) popping 8/16/32 node pairs per step, and keep the
 * fastest; otherwise the cost model of NQS_SCHED_AUTO with the default
 * parameters), allocates its buffers with 25% headroom over the planned
 * pair count, and captures all instances into one CUDA graph on forked
 * streams.  An instance with `grad` set also gets the gradient of its E^var
 * (the adjoint's closed form) in the graph.  Synchronises `stream`.  The
 * plan owns its device memory.  Real Hamiltonians only. */
int nqs_batch_plan(const nqs_instance* instances, int n_inst, int precision, int flags,
                   nqs_plan** out, void* stream);

/* One graph launch evaluating every instance: no host synchronisation, no
 * allocation.  If new sample contents need more pairs than planned, that
 * instance's outputs are left unwritten and nqs_batch_status reports it. */
int nqs_batch_run(nqs_plan* plan, void* stream);

/* Synchronise and return NQS_OK or the first instance's error
 * (NQS_ERR_CAPACITY when its pairs outgrew the planned buffers; re-plan). */
int nqs_batch_status(const nqs_plan* plan, int* failed_instance, void* stream);

/* info[0] schedule, [1] pair capacity, [2] planned pairs, [3] graph nodes,
 * [4] LoopOverTerms count time (us), [5] LoopOverBatch count time (us),
 * [6] LoopOverTrie tree build + count time (us) of instance i (-1: not
 * timed), [7] kernel nodes of the graph. */
int nqs_batch_info(const nqs_plan* plan, int i, int64_t info[8]);

/* Launch parameters chosen for instance i: tune[0] LoopOverTerms work items
 * per atomic, tune[1] its table groups per work item, tune[2] LoopOverTrie
 * node pairs popped per step (defaults 4, 16, 32 when not tuned). */
int nqs_batch_tune(const nqs_plan* plan, int i, int32_t tune[3]);

int nqs_batch_free(nqs_plan* plan);

/* ---------------------------------------------------------------------------
 * Misc
 * ------------------------------------------------------------------------- */
const char* nqs_last_error(void);   /* thread-local message of the last error */
int nqs_version(void);              /* NQS_VERSION                               */

/* Timing of the LoopOverTerms search kernel, for benchmarks.  While enabled
 * (on != 0), every launch of that kernel is bracketed by two CUDA events
 * recorded on its stream (no synchronisation, no effect on results).
 * nqs_search_time waits for the recorded events, returns the summed kernel
 * time (ms, host) and the number of launches (host), and forgets them.
 * Process-wide state; leave it disabled while capturing a CUDA graph (the
 * events would be captured, not recorded).  The paper has no counterpart. */
int nqs_search_timing(int on);
int nqs_search_time(double* total_ms, int64_t* launches);

/* Measured integer speed of light of the current device, for benchmark
 * rooflines of the LoopOverTerms search (the paper has no counterpart).
 * Runs two short kernels at the search kernel's launch shape (one 512-thread
 * block per SM), each timed with CUDA events on `stream` after a warm-up
 * launch, and synchronises the stream:
 *   out[0] = integer lane operations per second of a register-only mix of
 *            the operations of one filter probe (XOR, AND, 32-bit funnel
 *            shift, shift-or; counted as source-level operations, sixteen
 *            independent chains per thread);
 *   out[1] = probes per second of the search's filter loop by itself: eight
 *            samples per lane against a stream of pattern hashes, one word
 *            of a 128 KB shared-memory filter read and three bits tested per
 *            probe, no survivor handling.
 * out: host double[2].  Allocates and frees a small device buffer. */
int nqs_probe_peaks(double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NQS_H */
