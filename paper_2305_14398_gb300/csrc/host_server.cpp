// The serving loop (tqs_server_*): requests compiled at submit, admitted
// against an HBM budget, launched as batches of the fused kernels on stream
// slots and reaped by CUDA event.
#include "host_common.h"

// ------------------------------------------------------------------ server
//
// Continuous batching of simulate requests.  The caller submits requests as
// they arrive and calls tqs_server_poll often; each poll reaps finished
// batches (CUDA events), releases their device memory from the budget, then
// admits queued requests in arrival order while they fit the budget and
// launches them as one batch on a free stream, so that new work starts while
// earlier batches are still running.  Every request's result is the same as
// tqs_simulate's (same program, same team kind): batching never changes it.

namespace {

struct SrvReq {
  int64_t tag;
  Program prog;
  size_t bytes;  // device bytes while in flight
};

struct SrvSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<SrvReq> reqs;
  std::vector<int64_t> offsets;
  size_t bytes = 0;
  // pinned host staging of the batch's outputs
  float2* h_states = nullptr;
  double* h_norms = nullptr;
  size_t h_cap_amps = 0, h_cap_norms = 0;
  // pinned host copy of the batch program
  char* h_prog = nullptr;
  size_t h_prog_cap = 0;
};

struct SrvResult {
  std::vector<float2> state;
  double norm;
};

size_t request_bytes(const Program& P) {
  const size_t amps = size_t(1) << P.n;
  size_t b = P.passes.size() * sizeof(FusedPass) + P.ops.size() * sizeof(FusedOp) +
             sizeof(FusedCirc) + 3 * sizeof(int32_t) + amps * sizeof(float2) + sizeof(double) + 1024;
  if (team_for(P.nint) == TEAM_GLOBAL) b += (size_t(1) << kGlobalSlotQ) * sizeof(float2);
  return b;
}

cudaError_t grow_pinned(void** p, size_t* cap, size_t want) {
  if (want <= *cap && *p) return cudaSuccess;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  const size_t n = std::max(want, size_t(1) << 20);
  cudaError_t e = cudaMallocHost(p, n);
  if (e == cudaSuccess) *cap = n;
  return e;
}

}  // namespace

struct tqs_server {
  size_t budget = 0;
  size_t in_use = 0;
  size_t peak_in_use = 0;
  int max_batch = 256;
  std::vector<SrvSlot> slots;
  std::deque<SrvReq> queue;
  std::unordered_map<int64_t, SrvResult> results;
  int64_t done_count = 0;
  ~tqs_server() {
    for (SrvSlot& s : slots) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      if (s.done) cudaEventDestroy(s.done);
      if (s.stream) cudaStreamDestroy(s.stream);
      if (s.h_states) cudaFreeHost(s.h_states);
      if (s.h_norms) cudaFreeHost(s.h_norms);
      if (s.h_prog) cudaFreeHost(s.h_prog);
    }
  }
};

// Launch the requests of a slot as one batch on the slot's stream.
static tqs_status server_launch(tqs_server* sv, SrvSlot& sl) {
  Image img;
  sl.offsets.assign(sl.reqs.size() + 1, 0);
  int n_team[3] = {0, 0, 0};
  int max_nint[3] = {4, 4, 4};
  std::vector<int32_t> idx[3];
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    const Program& P = sl.reqs[i].prog;
    sl.offsets[i + 1] = sl.offsets[i] + (int64_t(1) << P.n);
    img.add(P, sl.offsets[i]);
    const int t = team_for(P.nint);
    idx[t].push_back(static_cast<int32_t>(i));
    max_nint[t] = std::max(max_nint[t], P.nint);
  }
  std::vector<int32_t> order;
  for (int t = 0; t < 3; ++t) {
    std::stable_sort(idx[t].begin(), idx[t].end(), [&](int a, int b) {
      return sl.reqs[a].prog.cost > sl.reqs[b].prog.cost;
    });
    n_team[t] = static_cast<int>(idx[t].size());
    order.insert(order.end(), idx[t].begin(), idx[t].end());
  }
  const size_t amps = static_cast<size_t>(sl.offsets.back());
  LaunchPlan plans[3];
  for (int t = 0; t < 3; ++t) plans[t] = plan_for(t, max_nint[t], n_team[t], 0);
  // Few global-class requests: K cooperating CTAs each (TEAM_MULTI),
  // bitwise the same results as one CTA each.  The J K CTAs take at most an
  // equal share of the SMs per slot in flight, so the cooperative grids of all
  // slots fit the GPU together (one such CTA per SM) and none waits at a
  // barrier for SMs held by another waiting grid.
  int multi_k = 0;
  const int J = n_team[TEAM_GLOBAL];
  if (J > 0 && J <= kMaxMultiJobs) {
    int k = 64;
    for (int32_t i : idx[TEAM_GLOBAL]) k = std::min(k, multi_ctas_for(sl.reqs[i].prog));
    const int share = device_sms() / std::max<int>(1, static_cast<int>(sv->slots.size()));
    if (k >= 2 && J * k <= share) multi_k = k;
  }
  const size_t order_off = (img.bytes() + 255) & ~size_t(255);
  const size_t counter_off = (order_off + order.size() * sizeof(int32_t) + 255) & ~size_t(255);
  const size_t states_off = counter_off + 256;
  const size_t norms_off = (states_off + amps * sizeof(float2) + 255) & ~size_t(255);
  const size_t gscr_off = (norms_off + sl.reqs.size() * sizeof(double) + 255) & ~size_t(255);
  const size_t gscr_bytes =
      J ? size_t(std::max(plans[TEAM_GLOBAL].grid, J)) << kGlobalSlotQ : size_t(0);
  const size_t total = gscr_off + gscr_bytes * sizeof(float2);
  // the program goes through pinned memory so the copy is truly asynchronous
  const size_t prog_bytes = order_off + order.size() * sizeof(int32_t);
  {
    void* p = sl.h_prog;
    TQS_CUDA(grow_pinned(&p, &sl.h_prog_cap, prog_bytes), "tqs_server: cudaMallocHost");
    sl.h_prog = static_cast<char*>(p);
  }
  img.copy_to(sl.h_prog);
  std::memcpy(sl.h_prog + order_off, order.data(), order.size() * sizeof(int32_t));
  {
    void* p = sl.h_states;
    TQS_CUDA(grow_pinned(&p, &sl.h_cap_amps, amps * sizeof(float2)), "tqs_server: cudaMallocHost");
    sl.h_states = static_cast<float2*>(p);
    p = sl.h_norms;
    TQS_CUDA(grow_pinned(&p, &sl.h_cap_norms, sl.reqs.size() * sizeof(double)),
             "tqs_server: cudaMallocHost");
    sl.h_norms = static_cast<double*>(p);
  }
  cudaStream_t s = sl.stream;
  char* base = nullptr;
  const Allocator A = current_allocator();
  if (A.alloc) {
    void* q = nullptr;
    TQS_CUDA(dev_alloc(A, &q, total, s), "tqs_server: allocator");
    base = static_cast<char*>(q);
  } else {
    TQS_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&base), total, s), "tqs_server: cudaMallocAsync");
  }
  TQS_CUDA(cudaMemcpyAsync(base, sl.h_prog, prog_bytes, cudaMemcpyHostToDevice, s), "tqs_server: H2D");
  int32_t* counters = reinterpret_cast<int32_t*>(base + counter_off);
  // team counters [0, 3), the TEAM_MULTI time-out word [3] and its per-job
  // barrier counters [4, 4 + J)
  TQS_CUDA(cudaMemsetAsync(counters, 0, (4 + (multi_k ? J : 0)) * sizeof(int32_t), s),
           "tqs_server: memset");
  float2* d_states = reinterpret_cast<float2*>(base + states_off);
  double* d_norms = reinterpret_cast<double*>(base + norms_off);
  int first = 0;
  for (int t = 0; t < 3; ++t) {
    if (n_team[t] == 0) continue;
    FusedLaunch L{};
    img.point(L, base);
    L.order = reinterpret_cast<const int32_t*>(base + order_off) + first;
    L.n_jobs = n_team[t];
    L.counter = counters + t;
    L.out = d_states;
    L.probs = nullptr;
    L.norms = d_norms;
    L.gscratch = reinterpret_cast<float2*>(base + gscr_off);
    L.team = plans[t].team;
    L.warps_per_cta = plans[t].warps;
    L.slice_q = plans[t].slice_q;
    L.grid = plans[t].grid;
    if (t == TEAM_GLOBAL && multi_k) {
      L.team = TEAM_MULTI;
      L.ctas_per_job = multi_k;
      L.grid = J * multi_k;
      L.counter = counters + 4;
      L.err = counters + 3;
    }
    TQS_CUDA(launch_fused(L, s), "tqs_server: launch");
    first += n_team[t];
  }
  TQS_CUDA(cudaMemcpyAsync(sl.h_states, d_states, amps * sizeof(float2), cudaMemcpyDeviceToHost, s),
           "tqs_server: D2H states");
  TQS_CUDA(cudaMemcpyAsync(sl.h_norms, d_norms, sl.reqs.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, s),
           "tqs_server: D2H norms");
  if (A.alloc) dev_free(A, base, s);
  else TQS_CUDA(cudaFreeAsync(base, s), "tqs_server: cudaFreeAsync");
  TQS_CUDA(cudaEventRecord(sl.done, s), "tqs_server: event");
  sl.busy = true;
  return TQS_OK;
}

extern "C" {

tqs_status tqs_server_create(size_t hbm_budget_bytes, int max_inflight, int max_batch,
                             tqs_server** out) {
  if (!out) return fail(TQS_ERR_ARG, "tqs_server_create: out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0 || max_inflight < 1 || max_inflight > 64 || max_batch < 1)
    return fail(TQS_ERR_ARG, "tqs_server_create: bad budget / max_inflight / max_batch");
  std::unique_ptr<tqs_server> sv(new (std::nothrow) tqs_server());
  if (!sv) return fail(TQS_ERR_NOMEM, "tqs_server_create: out of host memory");
  sv->budget = hbm_budget_bytes;
  sv->max_batch = max_batch;
  // keep freed batch memory in this process's default pool (up to the budget)
  // so that per-batch stream-ordered allocations do not go back to the driver
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = hbm_budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  sv->slots.resize(max_inflight);
  *out = sv.release();
  return TQS_OK;
}

tqs_status tqs_server_submit_packed(tqs_server* sv, int64_t tag, int n_qubits, int n_gates,
                                    const int32_t* h_kind, const int32_t* h_qubits,
                                    const double* h_params) {
  if (!sv) return fail(TQS_ERR_ARG, "tqs_server_submit_packed: server is NULL");
  if (n_qubits < 1 || n_qubits > TQS_MAX_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_server_submit_packed: n %d outside [1, %d]", n_qubits,
                TQS_MAX_QUBITS);
  if (n_gates < 0 || (n_gates > 0 && (!h_kind || !h_qubits || !h_params)))
    return fail(TQS_ERR_ARG, "tqs_server_submit_packed: bad gate arrays");
  if (sv->results.count(tag))
    return fail(TQS_ERR_ARG, "tqs_server_submit_packed: tag %lld has an untaken result",
                static_cast<long long>(tag));
  std::vector<Gate> gates(static_cast<size_t>(n_gates));
  std::vector<int> last(n_qubits, -1);
  for (int k = 0; k < n_gates; ++k) {
    const int kind = h_kind[k];
    const int nq = (kind >= 0 && kind < TQS_GATE_COUNT && is_two_qubit(kind)) ? 2 : 1;
    Gate& g = gates[k];
    tqs_status st = check_gate(n_qubits, kind, h_qubits + 2 * k, nq, h_params + 8 * k, 8, g);
    if (st != TQS_OK) return st;
    if (is_instruction(kind))
      return fail(TQS_ERR_UNSUPPORTED,
                  "tqs_server_submit_packed: measure/reset instructions are not served");
    assign_step(last, g);
  }
  SrvReq r;
  r.tag = tag;
  compile_program(n_qubits, step_order(gates), r.prog);
  r.bytes = request_bytes(r.prog);
  if (r.bytes > sv->budget)
    return fail(TQS_ERR_BUDGET, "tqs_server_submit_packed: request needs %zu bytes > budget %zu",
                r.bytes, sv->budget);
  sv->queue.push_back(std::move(r));
  return TQS_OK;
}

tqs_status tqs_server_poll(tqs_server* sv, int64_t* h_done_tags, int max_done, int* n_done) {
  if (!sv || (max_done > 0 && !h_done_tags)) return fail(TQS_ERR_ARG, "tqs_server_poll: bad arguments");
  int nd = 0;
  // 1. reap finished batches
  for (SrvSlot& sl : sv->slots) {
    if (!sl.busy) continue;
    if (static_cast<int>(sl.reqs.size()) > max_done - nd) continue;  // no room to report: later
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return cuda_fail(q, "tqs_server_poll: batch failed");
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
      SrvResult res;
      res.state.assign(sl.h_states + sl.offsets[i], sl.h_states + sl.offsets[i + 1]);
      res.norm = sl.h_norms[i];
      sv->results[sl.reqs[i].tag] = std::move(res);
      h_done_tags[nd++] = sl.reqs[i].tag;
    }
    sv->in_use -= sl.bytes;
    sv->done_count += static_cast<int64_t>(sl.reqs.size());
    sl.reqs.clear();
    sl.bytes = 0;
    sl.busy = false;
  }
  // 2. admit queued requests in arrival order into free slots
  for (SrvSlot& sl : sv->slots) {
    if (sv->queue.empty()) break;
    if (sl.busy) continue;
    if (!sl.stream) {
      TQS_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking), "tqs_server: stream");
      TQS_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "tqs_server: event");
      // Reserve pinned staging up front (cudaMallocHost is slow and
      // synchronising): room for a batch of 16 MiB of states and its program.
      void* p = nullptr;
      TQS_CUDA(grow_pinned(&p, &sl.h_cap_amps, size_t(16) << 20), "tqs_server: cudaMallocHost");
      sl.h_states = static_cast<float2*>(p);
      p = nullptr;
      TQS_CUDA(grow_pinned(&p, &sl.h_cap_norms, size_t(sv->max_batch) * sizeof(double)),
               "tqs_server: cudaMallocHost");
      sl.h_norms = static_cast<double*>(p);
      p = nullptr;
      TQS_CUDA(grow_pinned(&p, &sl.h_prog_cap, size_t(4) << 20), "tqs_server: cudaMallocHost");
      sl.h_prog = static_cast<char*>(p);
    }
    size_t bytes = 0;
    while (!sv->queue.empty() && static_cast<int>(sl.reqs.size()) < sv->max_batch &&
           sv->in_use + bytes + sv->queue.front().bytes <= sv->budget) {
      bytes += sv->queue.front().bytes;
      sl.reqs.push_back(std::move(sv->queue.front()));
      sv->queue.pop_front();
    }
    if (sl.reqs.empty()) break;  // the head does not fit yet: wait for memory
    sl.bytes = bytes;
    sv->in_use += bytes;
    sv->peak_in_use = std::max(sv->peak_in_use, sv->in_use);
    tqs_status st = server_launch(sv, sl);
    if (st != TQS_OK) return st;
  }
  if (n_done) *n_done = nd;
  return TQS_OK;
}

tqs_status tqs_server_take(tqs_server* sv, int64_t tag, tqs_c64* h_state, double* h_norm) {
  if (!sv) return fail(TQS_ERR_ARG, "tqs_server_take: server is NULL");
  auto it = sv->results.find(tag);
  if (it == sv->results.end())
    return fail(TQS_ERR_STATE, "tqs_server_take: no finished result for tag %lld",
                static_cast<long long>(tag));
  if (h_state) std::memcpy(h_state, it->second.state.data(), it->second.state.size() * sizeof(float2));
  if (h_norm) *h_norm = it->second.norm;
  sv->results.erase(it);
  return TQS_OK;
}

tqs_status tqs_server_cancel(tqs_server* sv, int64_t tag) {
  if (!sv) return fail(TQS_ERR_ARG, "tqs_server_cancel: server is NULL");
  for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
    if (it->tag == tag) {
      sv->queue.erase(it);
      return TQS_OK;
    }
  }
  for (const SrvSlot& sl : sv->slots)
    for (const SrvReq& r : sl.reqs)
      if (sl.busy && r.tag == tag)
        return fail(TQS_ERR_STATE, "tqs_server_cancel: request %lld is running",
                    static_cast<long long>(tag));
  if (sv->results.count(tag))
    return fail(TQS_ERR_STATE, "tqs_server_cancel: request %lld has finished",
                static_cast<long long>(tag));
  return fail(TQS_ERR_ARG, "tqs_server_cancel: no request %lld", static_cast<long long>(tag));
}

tqs_status tqs_server_stats(const tqs_server* sv, int64_t* queued, int64_t* inflight, int64_t* done,
                            int64_t* bytes_in_use, int64_t* peak_bytes) {
  if (!sv) return fail(TQS_ERR_ARG, "tqs_server_stats: server is NULL");
  int64_t fl = 0;
  for (const SrvSlot& sl : sv->slots) fl += sl.busy ? static_cast<int64_t>(sl.reqs.size()) : 0;
  if (queued) *queued = static_cast<int64_t>(sv->queue.size());
  if (inflight) *inflight = fl;
  if (done) *done = sv->done_count;
  if (bytes_in_use) *bytes_in_use = static_cast<int64_t>(sv->in_use);
  if (peak_bytes) *peak_bytes = static_cast<int64_t>(sv->peak_in_use);
  return TQS_OK;
}

tqs_status tqs_server_destroy(tqs_server* sv) {
  delete sv;
  return TQS_OK;
}

}  // extern "C"
