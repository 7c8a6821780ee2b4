// Batched evaluation of many independent (Hamiltonian, sample batch) instances
// as one CUDA graph: planning stages every instance, picks its FindCoupledPairs
// schedule and that schedule's launch parameters by timing the candidates
// (LoopOverTerms, Alg. 2A, with 2/4/8 work items per atomic and 8/16/32
// table groups per item; LoopOverBatch, Alg. 2B; LoopOverTrie, Alg. 2C with
// the prefix-tree build of Alg. 3, popping 8/16/32 node pairs per step),
// sizes its buffers, and captures all instances' kernels on forked streams
// into a single graph; each run is one graph launch with no host
// synchronisation and no allocation.  An instance with a gradient output also
// gets dE^var / d log psi (the closed form of the adjoint) in the graph.  Buffers sized at planning time are
// checked on the device: an overflow sets the instance's status word and the
// later kernels of that instance skip their work.
#include <algorithm>
#include <cstring>
#include <vector>

#include "nqs_internal.cuh"

namespace nqs {

struct PlanInstance {
  nqs_instance in;
  int schedule = NQS_SCHED_TERMS;
  StageHeader L;
  char* work = nullptr;
  int64_t* row_ptr = nullptr;
  uint32_t* pair_j = nullptr;
  uint32_t* pair_k = nullptr;
  void* scratch = nullptr;
  int64_t scratch_bytes = 0;
  double* hdiag = nullptr;
  int64_t capacity = 0;
  int64_t planned_pairs = 0;
  float t_terms_ms = -1.f, t_batch_ms = -1.f, t_trie_ms = -1.f;
  SearchTune tune;
};

}  // namespace nqs

struct nqs_plan {
  std::vector<nqs::PlanInstance> inst;
  int precision = NQS_PREC_FP32C;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  size_t n_nodes = 0;
  size_t n_kernels = 0;
  double* one = nullptr;   // device 1.0: the upstream of E^var for the gradients
};

namespace nqs {

__global__ void capacity_check_kernel(const int64_t* rp, int64_t rows, int64_t capacity, int32_t* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && rp[rows] - rp[0] > capacity) atomicOr(status, kStatusCapacity);
}

static void free_plan(nqs_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (auto& i : p->inst) {
    cudaFree(i.work); cudaFree(i.row_ptr); cudaFree(i.pair_j); cudaFree(i.pair_k);
    cudaFree(i.scratch); cudaFree(i.hdiag);
  }
  for (auto s : p->streams) cudaStreamDestroy(s);
  for (auto e : p->events) cudaEventDestroy(e);
  cudaFree(p->one);
  delete p;
}

// the kernels of one instance's forward pass, enqueued without host synchronisation
static cudaError_t enqueue_instance(PlanInstance& I, int precision, const double* one, cudaStream_t s) {
  const nqs_ham* ham = I.in.ham;
  const int64_t n = I.in.n_unq;
  char* w = I.work;
  cudaError_t e;
  int32_t* status = (int32_t*)(w + offsetof(StageHeader, status));
  if ((e = cudaMemsetAsync(status, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
  if ((e = launch_stage(ham, I.in.U, n, w, I.L, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(I.row_ptr, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
  if (I.schedule == NQS_SCHED_BATCH) {
    if ((e = launch_pairs_batch(ham, I.in.U, n, w, I.L, 0, n, I.row_ptr + 1, nullptr, nullptr, kCount, s)))
      return e;
    if ((e = launch_scan(I.row_ptr + 1, n, w, I.L, s)) != cudaSuccess) return e;
    capacity_check_kernel<<<1, 32, 0, s>>>(I.row_ptr, n, I.capacity, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_pairs_batch(ham, I.in.U, n, w, I.L, 0, n, I.row_ptr, I.pair_j, I.pair_k, kFill, s)))
      return e;
  } else if (I.schedule == NQS_SCHED_TRIE) {
    if ((e = launch_trie_build(ham, I.in.U, n, w, I.L, s)) != cudaSuccess) return e;
    if ((e = launch_pairs_trie(ham, I.in.U, n, w, I.L, 0, n, I.row_ptr + 1, nullptr, nullptr, kCount, s, I.tune)))
      return e;
    if ((e = launch_scan(I.row_ptr + 1, n, w, I.L, s)) != cudaSuccess) return e;
    capacity_check_kernel<<<1, 32, 0, s>>>(I.row_ptr, n, I.capacity, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_pairs_trie(ham, I.in.U, n, w, I.L, 0, n, I.row_ptr, I.pair_j, I.pair_k, kFill, s, I.tune)))
      return e;
  } else {
    PairScratch sc = pair_scratch_view(I.scratch, n, I.scratch_bytes);
    if ((e = launch_pairs_terms(ham, I.in.U, w, I.L, 0, n, I.row_ptr + 1, nullptr, nullptr, kEmit, &sc, s, I.tune)))
      return e;
    if ((e = launch_scan(I.row_ptr + 1, n, w, I.L, s)) != cudaSuccess) return e;
    // rows as the search placed them: the row sums are exact, so their order does not matter
    if ((e = launch_pairs_compact(ham, sc, w, I.L, 0, n, I.row_ptr, I.pair_j, I.pair_k, I.capacity, s, false)))
      return e;
  }
  if ((e = launch_amplitudes(I.in.logpsi_re, nullptr, n, precision, w, I.L, s, I.in.U)) != cudaSuccess) return e;
  if ((e = launch_local_energy(ham, I.in.U, n, w, I.L, false, 0, n, I.row_ptr, I.pair_j, I.pair_k, precision,
                               I.in.eloc_re, nullptr, I.hdiag, nullptr, s)) != cudaSuccess)
    return e;
  if ((e = launch_variational_energy(n, I.in.logpsi_re, I.in.eloc_re, w, I.in.evar, s)) != cudaSuccess) return e;
  if (!I.in.grad) return cudaSuccess;
  // dE^var / d Re log psi: the adjoint with no upstream on E_loc (closed form)
  return launch_backward(ham, I.in.U, n, w, I.L, false, I.in.logpsi_re, nullptr, 0, n, I.row_ptr, I.pair_j, I.pair_k,
                         I.in.eloc_re, nullptr, I.hdiag, I.in.evar, nullptr, nullptr, one, precision, nullptr,
                         I.in.grad, nullptr, s);
}

// one count pass of LoopOverTerms or LoopOverTrie with the given launch
// parameters, timed with events on the stream; *n_pairs receives the total
static cudaError_t time_count(PlanInstance& I, int sched, const SearchTune& t, cudaStream_t s, float* ms,
                              int64_t* n_pairs) {
  const nqs_ham* ham = I.in.ham;
  const int64_t n = I.in.n_unq;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  cudaEventRecord(e0, s);
  e = cudaMemsetAsync(I.row_ptr, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) {
    if (sched == NQS_SCHED_TRIE)
      e = launch_pairs_trie(ham, I.in.U, n, I.work, I.L, 0, n, I.row_ptr + 1, nullptr, nullptr, kCount, s, t);
    else
      e = launch_pairs_terms(ham, I.in.U, I.work, I.L, 0, n, I.row_ptr + 1, nullptr, nullptr, kCount, nullptr, s, t);
  }
  if (e == cudaSuccess) e = launch_scan(I.row_ptr + 1, n, I.work, I.L, s);
  cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n_pairs, I.row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace nqs

using namespace nqs;

extern "C" {

int nqs_batch_plan(const nqs_instance* insts, int n_inst, int precision, int flags, nqs_plan** out,
                   void* stream) {
  if (!out || !insts || n_inst <= 0) return fail(NQS_ERR_ARG, "bad argument");
  *out = nullptr;
  if (precision != NQS_PREC_FP64 && precision != NQS_PREC_FP32C) return fail(NQS_ERR_ARG, "bad precision");
  cudaStream_t s = (cudaStream_t)stream;
  nqs_plan* p = new nqs_plan();
  p->precision = precision;
  p->inst.resize(n_inst);
  cudaError_t e;
  int rc = NQS_OK;
  for (int i = 0; i < n_inst && !rc; ++i) {
    PlanInstance& I = p->inst[i];
    I.in = insts[i];
    const int64_t n = I.in.n_unq;
    if (!I.in.ham || !I.in.U || !I.in.logpsi_re || !I.in.eloc_re || !I.in.evar || n <= 0) {
      rc = fail(NQS_ERR_ARG, "instance " + std::to_string(i) + ": null pointer or empty batch");
      break;
    }
    if (I.in.ham->cplx) {  // the plan's outputs are real E_loc^var
      rc = fail(NQS_ERR_UNSUPPORTED, "instance " + std::to_string(i) + ": complex Hamiltonian in a batched plan");
      break;
    }
    I.L = stage_layout(I.in.ham, n);
    if ((e = cudaMalloc((void**)&I.work, I.L.total_bytes)) != cudaSuccess ||
        (e = cudaMalloc((void**)&I.row_ptr, 8 * (n + 1))) != cudaSuccess ||
        (e = cudaMalloc((void**)&I.hdiag, 8 * n)) != cudaSuccess) {
      rc = fail(NQS_ERR_OOM, "cudaMalloc in nqs_batch_plan");
      break;
    }
    if ((rc = nqs_stage(I.in.ham, I.in.U, n, I.work, I.L.total_bytes, 1, stream))) break;
    // schedule: time both count passes (autotune) or use the cost model
    int64_t np_terms = 0, np_batch = -1;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, s);
    rc = nqs_count_coupled_pairs(I.in.ham, I.in.U, n, I.work, 0, n, NQS_SCHED_TERMS, I.row_ptr, &np_terms, stream);
    cudaEventRecord(t1, s);
    cudaEventSynchronize(t1);
    cudaEventElapsedTime(&I.t_terms_ms, t0, t1);
    const bool try_batch = (flags & 1) && n <= 8 * I.in.ham->n_xy;
    if (!rc && try_batch) {
      cudaEventRecord(t0, s);
      rc = nqs_count_coupled_pairs(I.in.ham, I.in.U, n, I.work, 0, n, NQS_SCHED_BATCH, I.row_ptr, &np_batch,
                                   stream);
      cudaEventRecord(t1, s);
      cudaEventSynchronize(t1);
      cudaEventElapsedTime(&I.t_batch_ms, t0, t1);
      if (!rc && np_batch != np_terms) rc = fail(NQS_ERR_DEVICE_LIMIT, "schedules disagree on the pair count");
    }
    const bool try_trie = (flags & 1) && I.in.ham->n_qubits <= 255 && n < (int64_t(1) << 23);
    if (!rc && try_trie) {
      int64_t np_trie = -1;
      cudaEventRecord(t0, s);
      rc = nqs_stage_trie(I.in.ham, I.in.U, n, I.work, stream);
      if (!rc)
        rc = nqs_count_coupled_pairs(I.in.ham, I.in.U, n, I.work, 0, n, NQS_SCHED_TRIE, I.row_ptr, &np_trie,
                                     stream);
      cudaEventRecord(t1, s);
      cudaEventSynchronize(t1);
      cudaEventElapsedTime(&I.t_trie_ms, t0, t1);
      if (!rc && np_trie != np_terms) rc = fail(NQS_ERR_DEVICE_LIMIT, "schedules disagree on the pair count");
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc) break;
    if (flags & 1) {
      // launch parameters of the two tunable schedules: best of two timings per setting
      // (the trie's tree build, timed above, is shared by its settings)
      SearchTune best_terms, best_trie;
      float t_terms = 1e30f, t_trie = 1e30f;
      for (int grab : {2, 4, 8})
        for (int groups : {8, 16, 32}) {
          SearchTune t;
          t.terms_grab = grab;
          t.terms_groups = groups;
          for (int rep = 0; rep < 2 && !rc; ++rep) {
            float ms = 0.f;
            int64_t np = -1;
            if ((e = time_count(I, NQS_SCHED_TERMS, t, s, &ms, &np)) != cudaSuccess) rc = cuda_fail(e, "tuning");
            else if (np != np_terms) rc = fail(NQS_ERR_DEVICE_LIMIT, "launch settings disagree on the pair count");
            if (!rc && ms < t_terms) { t_terms = ms; best_terms = t; }
          }
        }
      if (!rc && try_trie) {
        const float build_ms = std::max(0.f, I.t_trie_ms);
        float count_default = 0.f;
        int64_t np = -1;
        if ((e = time_count(I, NQS_SCHED_TRIE, SearchTune(), s, &count_default, &np)) != cudaSuccess)
          rc = cuda_fail(e, "tuning");
        const float build_only = std::max(0.f, build_ms - count_default);
        for (int pop : {8, 16, 32}) {
          SearchTune t;
          t.trie_pop = pop;
          for (int rep = 0; rep < 2 && !rc; ++rep) {
            float ms = 0.f;
            if ((e = time_count(I, NQS_SCHED_TRIE, t, s, &ms, &np)) != cudaSuccess) rc = cuda_fail(e, "tuning");
            else if (np != np_terms) rc = fail(NQS_ERR_DEVICE_LIMIT, "launch settings disagree on the pair count");
            if (!rc && build_only + ms < t_trie) { t_trie = build_only + ms; best_trie = t; }
          }
        }
      }
      if (rc) break;
      I.t_terms_ms = t_terms;
      if (try_trie) I.t_trie_ms = t_trie;
      I.schedule = NQS_SCHED_TERMS;
      I.tune = best_terms;
      float best = t_terms;
      if (try_batch && I.t_batch_ms < best) { I.schedule = NQS_SCHED_BATCH; best = I.t_batch_ms; I.tune = SearchTune(); }
      if (try_trie && t_trie < best) { I.schedule = NQS_SCHED_TRIE; best = t_trie; I.tune = best_trie; }
    } else
      I.schedule = (n < I.in.ham->n_xy) ? NQS_SCHED_BATCH : NQS_SCHED_TERMS;
    I.planned_pairs = np_terms;
    I.capacity = np_terms + np_terms / 4 + 4096;
    I.scratch_bytes = pair_scratch_bytes(n, I.capacity);
    // LoopOverTerms instances keep their pairs packed (one 64-bit word each, pair_k unused):
    // the compaction writes them as the energy and adjoint kernels read them
    const bool packed = I.schedule == NQS_SCHED_TERMS;
    if ((e = cudaMalloc((void**)&I.pair_j, (packed ? 8 : 4) * I.capacity)) != cudaSuccess ||
        (!packed && (e = cudaMalloc((void**)&I.pair_k, 4 * I.capacity)) != cudaSuccess) ||
        (e = cudaMalloc(&I.scratch, I.scratch_bytes)) != cudaSuccess) {
      rc = fail(NQS_ERR_OOM, "cudaMalloc in nqs_batch_plan");
      break;
    }
  }
  if (rc) {
    free_plan(p);
    return rc;
  }
  // the upstream 1.0 of E^var for the instances' gradients (a device constant of the plan)
  {
    const double one = 1.0;
    if ((e = cudaMalloc((void**)&p->one, sizeof(double))) != cudaSuccess ||
        (e = cudaMemcpy(p->one, &one, sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
      free_plan(p);
      return fail(NQS_ERR_OOM, "cudaMalloc in nqs_batch_plan");
    }
  }
  // capture: fork over streams, one instance per stream round-robin, join
  const int K = std::min(8, n_inst);
  p->streams.resize(K);
  p->events.resize(K + 1);
  for (int k = 0; k < K; ++k) cudaStreamCreateWithFlags(&p->streams[k], cudaStreamNonBlocking);
  for (auto& ev : p->events) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaStream_t cs = p->streams[0];
  if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
    free_plan(p);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  cudaEventRecord(p->events[K], cs);
  for (int k = 1; k < K; ++k) cudaStreamWaitEvent(p->streams[k], p->events[K], 0);
  cudaError_t ce = cudaSuccess;
  for (int i = 0; i < n_inst && ce == cudaSuccess; ++i)
    ce = enqueue_instance(p->inst[i], precision, p->one, p->streams[i % K]);
  for (int k = 1; k < K; ++k) {
    cudaEventRecord(p->events[k], p->streams[k]);
    cudaStreamWaitEvent(cs, p->events[k], 0);
  }
  e = cudaStreamEndCapture(cs, &p->graph);
  if (ce != cudaSuccess || e != cudaSuccess) {
    free_plan(p);
    return cuda_fail(ce != cudaSuccess ? ce : e, "graph capture");
  }
  cudaGraphGetNodes(p->graph, nullptr, &p->n_nodes);
  {
    std::vector<cudaGraphNode_t> nodes(p->n_nodes);
    size_t nn = p->n_nodes;
    if (nn) cudaGraphGetNodes(p->graph, nodes.data(), &nn);
    for (size_t k = 0; k < nn; ++k) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++p->n_kernels;
    }
  }
  if ((e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess) {
    free_plan(p);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  *out = p;
  return NQS_OK;
}

int nqs_batch_run(nqs_plan* p, void* stream) {
  if (!p || !p->exec) return fail(NQS_ERR_ARG, "null plan");
  cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return NQS_OK;
}

int nqs_batch_status(const nqs_plan* p, int* failed_instance, void* stream) {
  if (!p) return fail(NQS_ERR_ARG, "null plan");
  if (failed_instance) *failed_instance = -1;
  for (size_t i = 0; i < p->inst.size(); ++i) {
    int rc = nqs_stage_status(p->inst[i].work, stream);
    if (rc) {
      if (failed_instance) *failed_instance = (int)i;
      return rc;
    }
  }
  return NQS_OK;
}

int nqs_batch_info(const nqs_plan* p, int i, int64_t info[8]) {
  if (!p || !info || i < 0 || i >= (int)p->inst.size()) return fail(NQS_ERR_ARG, "bad argument");
  const PlanInstance& I = p->inst[i];
  info[0] = I.schedule;
  info[1] = I.capacity;
  info[2] = I.planned_pairs;
  info[3] = (int64_t)p->n_nodes;
  info[4] = (int64_t)(1000.0f * I.t_terms_ms);
  info[5] = (int64_t)(1000.0f * I.t_batch_ms);
  info[6] = (int64_t)(1000.0f * I.t_trie_ms);
  info[7] = (int64_t)p->n_kernels;
  return NQS_OK;
}

int nqs_batch_tune(const nqs_plan* p, int i, int32_t tune[3]) {
  if (!p || !tune || i < 0 || i >= (int)p->inst.size()) return fail(NQS_ERR_ARG, "bad argument");
  const SearchTune& t = p->inst[i].tune;
  tune[0] = t.terms_grab;
  tune[1] = t.terms_groups;
  tune[2] = t.trie_pop;
  return NQS_OK;
}

int nqs_batch_free(nqs_plan* p) {
  free_plan(p);
  return NQS_OK;
}

}  // extern "C"
