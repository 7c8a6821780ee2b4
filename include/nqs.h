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
 *   - Scope of version 1: real Hamiltonians (every string has an even number
 *     of Y, real h_l; molecular Hamiltonians are of this kind); complex log
 *     psi is supported; 1 <= N <= 256.
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
    NQS_ERR_UNSUPPORTED = -2,  /* outside the scope above (odd |Y|, N > 256)        */
    NQS_ERR_CUDA = -3,         /* a CUDA runtime call failed                        */
    NQS_ERR_CAPACITY = -4,     /* output buffer too small; required size returned  */
    NQS_ERR_DUPLICATE = -5,    /* the sample batch repeats a basis vector           */
    NQS_ERR_DEVICE_LIMIT = -6, /* a bounded device loop ran out, or a device index
                                  check failed and the access was skipped
                                  (corrupt input or pair list)                     */
    NQS_ERR_OOM = -7,          /* device allocation inside nqs_ham_load failed      */
    NQS_ERR_RANGE = -8         /* an amplitude ratio leaves the FP32 exponent range */
};

enum {
    NQS_SCHED_AUTO = 0,   /* library's choice                                      */
    NQS_SCHED_TERMS = 1,  /* loop over unique XY per sample (Alg. 2A)               */
    NQS_SCHED_BATCH = 2,  /* loop over the batch per sample (Alg. 2B)               */
    NQS_SCHED_TRIE = 3    /* joint prefix-tree traversal (Algs. 3 and 2C)          */
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
 * coefficient is exactly zero are dropped.  Errors: NQS_ERR_ARG (n_qubits
 * out of range, bits >= N set, null pointer), NQS_ERR_UNSUPPORTED (a term
 * with an odd number of Y), NQS_ERR_OOM, NQS_ERR_CUDA.  On success *out
 * owns the device tables until nqs_ham_free. */
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
 *   coef    [terms]     h_l * i^{|Y^(l)|} (real, since |Y| is even)           */
int nqs_ham_export(const nqs_ham* ham, uint64_t* xy, int64_t* row_ptr,
                   uint64_t* yz, double* coef);

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
 * pair_j, pair_k device uint32 [row_ptr[last]].  Asynchronous. */
int nqs_fill_coupled_pairs(const nqs_ham* ham, const uint64_t* U, int64_t n_unq,
                           void* work, int64_t row_begin, int64_t row_end,
                           int schedule, const int64_t* row_ptr, uint32_t* pair_j,
                           uint32_t* pair_k, void* stream);

/* Bytes of the scratch that nqs_find_coupled_pairs needs to list up to
 * max_pairs pairs of `rows` rows in one pass. */
int64_t nqs_pairs_scratch_bytes(int64_t rows, int64_t max_pairs);

/* One search pass.  The pairs are written to scratch (device, 256-byte
 * aligned, scratch_bytes from nqs_pairs_scratch_bytes) while the rows are
 * counted, then copied in CSR order to pair_j/pair_k (device uint32,
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

/* ---------------------------------------------------------------------------
 * MatrixElement + ScatterAdd -> E_loc^var (Sec. "MatrixElement
 * implementation", Fig. scatter_local_energies)
 * ------------------------------------------------------------------------- */

/* For rows r in [row_begin, row_end), with their pairs from a fill pass over
 * the same range, write
 *   eloc_re[r], eloc_im[r] = E_loc^var(U_r)  (eloc_im may be NULL only if
 *                                              logpsi_im is NULL),
 *   hdiag[r] = H_{U_r U_r} (may be NULL),
 *   hpair[q] = H of pair q, q indexing pair_j/pair_k (may be NULL): device
 *              float2 (hi, lo) per pair with NQS_PREC_FP32C, double with
 *              NQS_PREC_FP64; nqs_local_energy_backward can read it instead
 *              of recomputing the matrix elements.
 * logpsi_re/_im: device FP64 [n_unq] for the whole batch.  Each row is a
 * fixed-order reduction by one warp, so results are bitwise reproducible
 * (rows are handed out heaviest first; the order does not affect any row).
 * The call overwrites the per-sample scratch of work.  Asynchronous. */
int nqs_local_energy(const nqs_ham* ham, const uint64_t* U, int64_t n_unq, void* work,
                     const double* logpsi_re, const double* logpsi_im,
                     int64_t row_begin, int64_t row_end, const int64_t* row_ptr,
                     const uint32_t* pair_j, const uint32_t* pair_k, int precision,
                     double* eloc_re, double* eloc_im, double* hdiag, void* hpair,
                     void* stream);

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
 * For rows y in [row_begin, row_end) (pairs of those rows) writes
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
 * pairs because x XOR y is symmetric and H is real symmetric.
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
} nqs_instance;

/* Plan n_inst instances (arrays are read during the call; the pointers inside
 * must stay valid for the plan's lifetime).  Planning stages every instance,
 * counts its pairs, picks its schedule (flags bit 0: time the count pass of
 * LoopOverTerms, LoopOverBatch and LoopOverTrie (with its prefix-tree build)
 * and keep the fastest; otherwise the cost model of NQS_SCHED_AUTO), allocates its buffers with 25% headroom over the planned
 * pair count, and captures all instances into one CUDA graph on forked
 * streams.  Synchronises `stream`.  The plan owns its device memory. */
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
