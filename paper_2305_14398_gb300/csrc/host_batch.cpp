// Batches (tqs_batch_*): packed creation on the host thread pool, the image
// assembly, the CUDA-graph run, the host-buffer run, and the circuit-unitary chain
// entry point.
#include "host_common.h"

// ------------------------------------------------------------------ batch





// Assemble the batch image from compiled programs held in segments: the
// device arrays are the segments concatenated in order, so a program's global
// offsets are its segment's base plus its local offsets.  Headers are written
// and passes renumbered in parallel, in place.
// Number of team kinds (warp, CTA, global) that have circuits in the batch.
static int team_kinds(const tqs_batch* b) {
  int k = 0;
  for (int t = 0; t < 3; ++t) k += b->n_team[t] > 0;
  return k;
}

static tqs_status batch_finish(tqs_batch* b, const std::vector<CircMeta>& progs,
                               std::vector<ImageSeg>&& segs) {
  b->count = static_cast<int>(progs.size());
  b->offsets.assign(b->count + 1, 0);
  b->instr_off.assign(b->count + 1, 0);
  for (int i = 0; i < b->count; ++i) {
    b->offsets[i + 1] = b->offsets[i] + (int64_t(1) << progs[i].n);
    b->instr_off[i + 1] = b->instr_off[i] + progs[i].n_instr;
  }
  const size_t nseg = segs.size();
  std::vector<int64_t> pbase(nseg + 1, 0), obase(nseg + 1, 0), cbase(nseg + 1, 0);
  for (size_t w = 0; w < nseg; ++w) {
    pbase[w + 1] = pbase[w] + static_cast<int64_t>(segs[w].passes.size());
    obase[w + 1] = obase[w] + static_cast<int64_t>(segs[w].ops.size());
    cbase[w + 1] = cbase[w] + static_cast<int64_t>(segs[w].coef.size());
  }
  if (b->instr_off.back() > 0xFFFFFFFFll || obase.back() > 0xFFFFFFFFll || cbase.back() > 0xFFFFFFFFll ||
      pbase.back() > 0x7FFFFFFFll)
    return fail(TQS_ERR_ARG, "tqs_batch: program too large for 32-bit offsets");
  b->img.circs = take_circs(static_cast<size_t>(b->count));
  b->img.segs = std::move(segs);
  b->img.npass = static_cast<size_t>(pbase.back());
  b->img.nop = static_cast<size_t>(obase.back());
  b->img.ncoef = static_cast<size_t>(cbase.back());
  parallel_for(b->count, 256, [&](int i) {
    const CircMeta& m = progs[i];
    ImageSeg& sg = b->img.segs[static_cast<size_t>(m.seg)];
    const int64_t p0 = pbase[m.seg] + static_cast<int64_t>(m.lp);
    const int64_t o0 = obase[m.seg] + static_cast<int64_t>(m.lo);
    const int64_t c0 = cbase[m.seg] + static_cast<int64_t>(m.lc);
    FusedCirc fc{};
    fc.n = static_cast<int16_t>(m.n);
    fc.nint = static_cast<int16_t>(m.nint);
    fc.pass_begin = static_cast<int32_t>(p0);
    fc.pass_count = static_cast<int32_t>(m.np);
    fc.out_off = b->offsets[i];
    fc.op_begin = static_cast<int32_t>(o0);
    fc.op_count = static_cast<int32_t>(m.no);
    fc.col_off = m.col_off;
    std::memcpy(fc.col, m.col, sizeof(fc.col));
    fc.init = nullptr;
    fc.out_scale = m.out_scale;
    fc.gen_index = m.gen_index;
    b->img.circs[i] = fc;
    for (size_t k = 0; k < m.np; ++k)
      sg.passes[m.lp + k] = Image::rebase(sg.passes[m.lp + k], o0, b->instr_off[i], c0);
  });
  // Job order per team kind, costliest first (load balance only: every
  // circuit's results are the same in any order).  A counting sort on the
  // cost's log2 in steps of 1/16 (about 4 % apart), batch order within a step.
  constexpr int kBuckets = 1024;
  static thread_local std::vector<int> key, start;
  key.resize(static_cast<size_t>(b->count));
  start.assign(3 * (kBuckets + 1), 0);
  for (int i = 0; i < b->count; ++i) {
    const int t = team_for(progs[i].nint);
    const double c = std::max(progs[i].cost, 1.0);
    const int k = std::min(kBuckets - 1, static_cast<int>(std::log2(c) * 16.0));
    key[static_cast<size_t>(i)] = t * kBuckets + (kBuckets - 1 - k);  // descending cost
    ++start[static_cast<size_t>(t * (kBuckets + 1) + (kBuckets - 1 - k) + 1)];
    ++b->n_team[t];
    b->max_nint[t] = std::max(b->max_nint[t], progs[i].nint);
  }
  b->order.resize(static_cast<size_t>(b->count));
  int base = 0;
  for (int t = 0; t < 3; ++t) {
    int* st = &start[static_cast<size_t>(t * (kBuckets + 1))];
    st[0] = base;
    for (int k = 0; k < kBuckets; ++k) st[k + 1] += st[k];
    base += b->n_team[t];
  }
  for (int i = 0; i < b->count; ++i) {
    const int kk = key[static_cast<size_t>(i)], t = kk / kBuckets, k = kk % kBuckets;
    b->order[static_cast<size_t>(start[static_cast<size_t>(t * (kBuckets + 1) + k)]++)] = i;
  }
  return TQS_OK;
}

extern "C" {

tqs_status tqs_batch_create(tqs_circuit* const* cs, int count, tqs_batch** out) {
  if (!out || !cs || count < 1) return fail(TQS_ERR_ARG, "tqs_batch_create: bad arguments");
  *out = nullptr;
  std::unique_ptr<tqs_batch> b(new (std::nothrow) tqs_batch());
  if (!b) return fail(TQS_ERR_NOMEM, "tqs_batch_create: out of host memory");
  std::vector<Program> progs(count);
  for (int i = 0; i < count; ++i) {
    if (!cs[i]) return fail(TQS_ERR_ARG, "tqs_batch_create: circuit %d is NULL", i);
    if (cs[i]->n > TQS_MAX_QUBITS)
      return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_batch_create: circuit %d has n %d > %d", i,
                  cs[i]->n, TQS_MAX_QUBITS);
    compile_program(cs[i]->n, step_order(cs[i]->gates), progs[i]);
    b->total_steps += cs[i]->nsteps;
  }
  std::vector<ImageSeg> segs;
  segs.push_back(take_seg());
  std::vector<CircMeta> metas(count);
  for (int i = 0; i < count; ++i) metas[i] = append_program(progs[i], segs[0], 0);
  tqs_status s = batch_finish(b.get(), metas, std::move(segs));
  if (s != TQS_OK) return s;
  *out = b.release();
  return TQS_OK;
}

tqs_status tqs_batch_create_packed(int count, const int32_t* h_nq, const int64_t* h_gate_off,
                                   const int32_t* h_kind, const int32_t* h_qubits,
                                   const double* h_params, tqs_batch** out) {
  if (!out || count < 1 || !h_nq || !h_gate_off || !h_kind || !h_qubits || !h_params)
    return fail(TQS_ERR_ARG, "tqs_batch_create_packed: bad arguments");
  *out = nullptr;
  std::unique_ptr<tqs_batch> b(new (std::nothrow) tqs_batch());
  if (!b) return fail(TQS_ERR_NOMEM, "tqs_batch_create_packed: out of host memory");
  std::vector<CircMeta> metas(count);
  std::vector<int> nsteps(count, 0);
  // Circuits are independent: compile them on all host cores.  Worker w takes
  // the contiguous range [w C / W, (w + 1) C / W) and compiles into one reused
  // Program, appending the result to its own segment, reserved up front from
  // the gate counts of its range (about one op and at most one pass per gate;
  // a program rarely needs more, and then the segment grows).
  // Each worker records its first failure; the lowest failing circuit index
  // is reported.
  int width = static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
  if (const char* env = std::getenv("TQS_HOST_THREADS")) width = std::max(1, std::atoi(env));
  const int nworkers = std::max(1, std::min({count / 64, 32, width}));
  std::vector<ImageSeg> segs(static_cast<size_t>(nworkers));
  struct Failure {
    int index = -1;
    tqs_status status = TQS_OK;
    std::string message;
  };
  std::mutex fail_mu;
  Failure first;
  for (int w = 0; w < nworkers; ++w) segs[static_cast<size_t>(w)] = take_seg();
  parallel_for(nworkers, 1, [&](int w) {
    const int lo = static_cast<int>(int64_t(count) * w / nworkers);
    const int hi = static_cast<int>(int64_t(count) * (w + 1) / nworkers);
    ImageSeg& sg = segs[static_cast<size_t>(w)];
    const int64_t span = h_gate_off[hi] - h_gate_off[lo];
    if (span >= 0) {
      sg.passes.reserve(static_cast<size_t>(span) + static_cast<size_t>(hi - lo));
      sg.ops.reserve(static_cast<size_t>(span) + 4 * static_cast<size_t>(hi - lo));
    }
    static thread_local std::vector<Gate> gates;
    static thread_local std::vector<int> last;
    static thread_local Program tp;
    for (int i = lo; i < hi; ++i) {
      auto record = [&](tqs_status st) {
        std::lock_guard<std::mutex> lock(fail_mu);
        if (first.index < 0 || i < first.index) {
          first.index = i;
          first.status = st;
          first.message = g_last_error;  // this worker thread's message
        }
      };
      const int n = h_nq[i];
      if (n < 1 || n > TQS_MAX_QUBITS) {
        record(fail(TQS_ERR_TOO_MANY_QUBITS, "circuit %d: n %d outside [1, %d]", i, n, TQS_MAX_QUBITS));
        continue;
      }
      const int64_t g0 = h_gate_off[i], g1 = h_gate_off[i + 1];
      if (g1 < g0) {
        record(fail(TQS_ERR_ARG, "circuit %d: gate offsets decrease", i));
        continue;
      }
      // the buffer only grows (check_gate sets every field of the gates used)
      const size_t ng = static_cast<size_t>(g1 - g0);
      if (gates.size() < ng) gates.resize(ng);
      last.assign(n, -1);
      tqs_status st = TQS_OK;
      for (int64_t k = g0; k < g1 && st == TQS_OK; ++k) {
        const int kind = h_kind[k];
        const int nq = (kind >= 0 && kind < TQS_GATE_COUNT && is_two_qubit(kind)) ? 2 : 1;
        Gate& g = gates[static_cast<size_t>(k - g0)];
        st = check_gate(n, kind, h_qubits + 2 * k, nq, h_params + 8 * k, 8, g);
        if (st != TQS_OK) break;
        assign_step(last, g);
      }
      if (st != TQS_OK) {
        record(st);
        continue;
      }
      for (int q = 0; q < n; ++q) nsteps[i] = std::max(nsteps[i], last[q] + 1);
      tp.reset();
      compile_program(n, step_order(gates.data(), ng), tp);
      metas[i] = append_program(tp, sg, w);
    }
  });
  if (first.index >= 0) {
    give_segs(segs);
    return fail(first.status, "%s", first.message.c_str());
  }
  for (int i = 0; i < count; ++i) b->total_steps += nsteps[i];
  tqs_status s = batch_finish(b.get(), metas, std::move(segs));
  if (s != TQS_OK) return s;
  *out = b.release();
  return TQS_OK;
}

tqs_status tqs_batch_info(const tqs_batch* b, int* count, int64_t* total_amps, int64_t* total_steps,
                          int64_t* program_bytes, int64_t* h_offsets) {
  if (!b) return fail(TQS_ERR_ARG, "tqs_batch_info: batch is NULL");
  if (count) *count = b->count;
  if (total_amps) *total_amps = b->offsets.back();
  if (total_steps) *total_steps = b->total_steps;
  if (program_bytes)
    *program_bytes = static_cast<int64_t>(b->img.bytes() + b->order.size() * sizeof(int32_t));
  if (h_offsets) std::memcpy(h_offsets, b->offsets.data(), b->offsets.size() * sizeof(int64_t));
  return TQS_OK;
}

}  // extern "C"

static tqs_status batch_upload(tqs_batch* b, cudaStream_t s) {
  b->order_off = (b->img.bytes() + 255) & ~size_t(255);
  b->counter_off = (b->order_off + b->order.size() * sizeof(int32_t) + 255) & ~size_t(255);
  TQS_CUDA(b->d_img.ensure(b->counter_off + 256), "tqs_batch: cudaMalloc program");
  TQS_CUDA(b->img.upload(b->d_img.p, s), "tqs_batch: upload program");
  TQS_CUDA(cudaMemcpyAsync(b->d_img.as<char>() + b->order_off, b->order.data(),
                           b->order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s),
           "tqs_batch: upload order");
  for (int t = 0; t < 3; ++t)
    b->plans[t] = plan_for(t, b->max_nint[t], b->n_team[t], 0);
  if (b->n_team[TEAM_GLOBAL] > 0)
    TQS_CUDA(b->d_gscratch.ensure(size_t(b->plans[TEAM_GLOBAL].grid) *
                                  (size_t(1) << kGlobalSlotQ) * sizeof(float2)),
             "tqs_batch: cudaMalloc scratch");
  if (team_kinds(b) > 1) TQS_CUDA(b->ensure_side(), "tqs_batch: side streams");
  b->uploaded = true;
  return TQS_OK;
}

// Enqueue the batch's kernels (memset of the job counters + one launch per
// team kind present) for a program image at `base`.
static tqs_status batch_enqueue_at(tqs_batch* b, char* base, size_t order_off, size_t counter_off,
                                   float2* gscratch, float2* states, double* probs, double* norms,
                                   cudaStream_t s, int* kernels = nullptr,
                                   const double* u = nullptr, int32_t* outcomes = nullptr) {
  int32_t* counters = reinterpret_cast<int32_t*>(base + counter_off);
  TQS_CUDA(cudaMemsetAsync(counters, 0, 3 * sizeof(int32_t), s), "tqs_batch: memset counters");
  int k = 0;
  int first = 0;
  const bool fork = team_kinds(b) > 1;  // (the side streams exist: ensure_side before any capture)
  if (fork) {
    if (!b->ev_fork) return fail(TQS_ERR_STATE, "tqs_batch: side streams missing");
    TQS_CUDA(cudaEventRecord(b->ev_fork, s), "tqs_batch: fork");
  }
  for (int t = 0; t < 3; ++t) {
    if (b->n_team[t] == 0) continue;
    FusedLaunch L{};
    b->img.point(L, base);
    L.order = reinterpret_cast<const int32_t*>(base + order_off) + first;
    L.n_jobs = b->n_team[t];
    L.counter = counters + t;
    L.out = states;
    L.probs = probs;
    L.exact_probs = b->exact_probs;
    L.norms = norms;
    L.gscratch = gscratch;
    L.uniforms = u;
    L.outcomes = outcomes;
    L.team = b->plans[t].team;
    L.warps_per_cta = b->plans[t].warps;
    L.slice_q = b->plans[t].slice_q;
    L.grid = b->plans[t].grid;
    if (fork) {
      TQS_CUDA(cudaStreamWaitEvent(b->side[t], b->ev_fork, 0), "tqs_batch: fork");
      TQS_CUDA(launch_fused(L, b->side[t]), "tqs_batch: launch");
      TQS_CUDA(cudaEventRecord(b->ev_join[t], b->side[t]), "tqs_batch: join");
    } else {
      TQS_CUDA(launch_fused(L, s), "tqs_batch: launch");
    }
    first += b->n_team[t];
    ++k;
  }
  if (fork)
    for (int t = 0; t < 3; ++t)
      if (b->n_team[t] > 0) TQS_CUDA(cudaStreamWaitEvent(s, b->ev_join[t], 0), "tqs_batch: join");
  if (kernels) *kernels = k;
  return TQS_OK;
}

static tqs_status batch_enqueue(tqs_batch* b, float2* states, double* probs, double* norms,
                                cudaStream_t s, int* kernels, const double* u = nullptr,
                                int32_t* outcomes = nullptr) {
  return batch_enqueue_at(b, b->d_img.as<char>(), b->order_off, b->counter_off,
                          b->d_gscratch.as<float2>(), states, probs, norms, s, kernels, u, outcomes);
}


static tqs_status batch_run_impl(tqs_batch* b, tqs_c64* d_states, double* d_probs, double* d_norms,
                                 const double* d_u, int32_t* d_outcomes, int use_graph,
                                 void* stream) {
  if (!b || !d_states) return fail(TQS_ERR_ARG, "tqs_batch_run: NULL batch or states");
  if (!aligned16(d_states) || (d_probs && !aligned16(d_probs)))
    return fail(TQS_ERR_ARG, "tqs_batch_run: device buffers must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!b->uploaded) {
    tqs_status st = batch_upload(b, s);
    if (st != TQS_OK) return st;
  }
  float2* states = reinterpret_cast<float2*>(d_states);
  if (!use_graph) {
    b->exact_probs = g_exact_probs.load();
    return batch_enqueue(b, states, d_probs, d_norms, s, nullptr, d_u, d_outcomes);
  }
  b->exact_probs = g_exact_probs.load();
  if (!b->exec || b->g_states != d_states || b->g_probs != d_probs || b->g_norms != d_norms ||
      b->g_u != d_u || b->g_outcomes != d_outcomes || b->g_exact != b->exact_probs) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (!b->cap_stream)
      TQS_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "tqs_batch: stream");
    // the upload must be complete before the captured work can run on another stream
    TQS_CUDA(cudaStreamSynchronize(s), "tqs_batch: sync before capture");
    TQS_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal),
             "tqs_batch: begin capture");
    const int64_t before = tqs_launch_count();
    int kernels = 0;
    tqs_status st = batch_enqueue(b, states, d_probs, d_norms, b->cap_stream, &kernels, d_u,
                                  d_outcomes);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    count_launches(before - tqs_launch_count());  // captured launches did not run yet
    if (st != TQS_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "tqs_batch: end capture");
    b->graph = g;
    TQS_CUDA(cudaGraphInstantiate(&b->exec, g, 0), "tqs_batch: instantiate");
    b->g_states = d_states;
    b->g_probs = d_probs;
    b->g_norms = d_norms;
    b->g_u = d_u;
    b->g_outcomes = d_outcomes;
    b->g_exact = b->exact_probs;
    b->graph_kernels = kernels;
  }
  TQS_CUDA(cudaGraphLaunch(b->exec, s), "tqs_batch: graph launch");
  count_launches(b->graph_kernels);
  return TQS_OK;
}

extern "C" {

tqs_status tqs_batch_run(tqs_batch* b, tqs_c64* d_states, double* d_probs, double* d_norms,
                         int use_graph, void* stream) {
  if (b && b->instr_off.back() > 0)
    return fail(TQS_ERR_UNSUPPORTED,
                "tqs_batch_run: the batch holds measure/reset instructions: use tqs_batch_run_measured");
  return batch_run_impl(b, d_states, d_probs, d_norms, nullptr, nullptr, use_graph, stream);
}

tqs_status tqs_batch_run_measured(tqs_batch* b, tqs_c64* d_states, double* d_probs,
                                  double* d_norms, const double* d_u, int32_t* d_outcomes,
                                  int use_graph, void* stream) {
  if (b && b->instr_off.back() > 0 && !d_u)
    return fail(TQS_ERR_ARG, "tqs_batch_run_measured: the batch holds instructions: d_u is NULL");
  return batch_run_impl(b, d_states, d_probs, d_norms, d_u, d_outcomes, use_graph, stream);
}

tqs_status tqs_batch_instructions(const tqs_batch* b, int64_t* h_off) {
  if (!b || !h_off) return fail(TQS_ERR_ARG, "tqs_batch_instructions: NULL argument");
  std::memcpy(h_off, b->instr_off.data(), b->instr_off.size() * sizeof(int64_t));
  return TQS_OK;
}

tqs_status tqs_batch_launch_info(const tqs_batch* b, int size_class, int* jobs, int* grid,
                                 int* threads, int* teams) {
  if (!b || size_class < 0 || size_class > 2)
    return fail(TQS_ERR_ARG, "tqs_batch_launch_info: NULL batch or size class outside 0..2");
  if (!b->uploaded) return fail(TQS_ERR_STATE, "tqs_batch_launch_info: the batch has not run yet");
  const LaunchPlan& lp = b->plans[size_class];
  const int n_jobs = b->n_team[size_class];
  int per_cta = 1;
  if (lp.team == TEAM_WARP) per_cta = lp.warps;
  else if (lp.team == TEAM_PAIR) per_cta = lp.warps / 2;
  if (jobs) *jobs = n_jobs;
  if (grid) *grid = n_jobs ? lp.grid : 0;
  const int nthreads = (lp.team == TEAM_WARP || lp.team == TEAM_PAIR) ? 32 * lp.warps
                       : lp.team == TEAM_CTA ? 32 * lp.warps : kGlobalThreads;
  if (threads) *threads = n_jobs ? nthreads : 0;
  if (teams) *teams = n_jobs ? lp.grid * per_cta : 0;
  return TQS_OK;
}

}  // extern "C"


extern "C" {

tqs_status tqs_batch_run_host(tqs_batch* b, tqs_c64* h_states, double* h_probs, double* h_norms,
                              void* stream) {
  if (!b) return fail(TQS_ERR_ARG, "tqs_batch_run_host: batch is NULL");
  if (b->instr_off.back() > 0)
    return fail(TQS_ERR_UNSUPPORTED, "tqs_batch_run_host: the batch holds measure/reset instructions");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  keep_pool_memory();
  // Everything this call needs on the device (the program is its input) comes
  // stream-ordered from the device's memory pool and goes back to it at the end.
  const size_t amps = static_cast<size_t>(b->offsets.back());
  // outputs whose host buffers the GPU can write directly skip the device copy
  const bool direct = g_host_writes.load() != 0;
  float2* zs = direct ? static_cast<float2*>(mapped_alias(h_states, amps * sizeof(float2))) : nullptr;
  double* zp = direct ? static_cast<double*>(mapped_alias(h_probs, amps * sizeof(double))) : nullptr;
  double* zn = direct ? static_cast<double*>(mapped_alias(h_norms, size_t(b->count) * sizeof(double)))
                      : nullptr;
  const size_t order_off = (b->img.bytes() + 255) & ~size_t(255);
  const size_t counter_off = (order_off + b->order.size() * sizeof(int32_t) + 255) & ~size_t(255);
  const size_t states_off = counter_off + 256;
  const size_t probs_off = (states_off + (zs ? 0 : amps * sizeof(float2)) + 255) & ~size_t(255);
  const size_t norms_off = (probs_off + (h_probs && !zp ? amps * sizeof(double) : 0) + 255) & ~size_t(255);
  const size_t total = norms_off + (zn ? 0 : size_t(b->count) * sizeof(double));
  for (int t = 0; t < 3; ++t) b->plans[t] = plan_for(t, b->max_nint[t], b->n_team[t], 0);
  const size_t gscr = b->n_team[TEAM_GLOBAL]
                          ? size_t(b->plans[TEAM_GLOBAL].grid) * (size_t(1) << kGlobalSlotQ) * sizeof(float2)
                          : 0;
  char* base = nullptr;
  const Allocator A = current_allocator();
  if (A.alloc) {
    void* q = nullptr;
    TQS_CUDA(dev_alloc(A, &q, ((total + 255) & ~size_t(255)) + gscr, s), "tqs_batch_run_host: allocator");
    base = static_cast<char*>(q);
  } else {
    TQS_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&base), ((total + 255) & ~size_t(255)) + gscr, s),
             "tqs_batch_run_host: cudaMallocAsync");
  }
  TQS_CUDA(b->img.upload(base, s), "tqs_batch_run_host: upload program");
  TQS_CUDA(cudaMemcpyAsync(base + order_off, b->order.data(), b->order.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s),
           "tqs_batch_run_host: upload order");
  float2* ds = zs ? zs : reinterpret_cast<float2*>(base + states_off);
  double* dp = zp ? zp : (h_probs ? reinterpret_cast<double*>(base + probs_off) : nullptr);
  double* dn = zn ? zn : reinterpret_cast<double*>(base + norms_off);
  const size_t gscr_at = (total + 255) & ~size_t(255);
  b->exact_probs = g_exact_probs.load();
  if (team_kinds(b) > 1) TQS_CUDA(b->ensure_side(), "tqs_batch_run_host: side streams");
  tqs_status st = batch_enqueue_at(b, base, order_off, counter_off,
                                   reinterpret_cast<float2*>(base + gscr_at), ds, dp, dn, s);
  if (st != TQS_OK) return st;
  if (h_states && !zs)
    TQS_CUDA(cudaMemcpyAsync(h_states, ds, amps * sizeof(float2), cudaMemcpyDeviceToHost, s), "D2H states");
  if (h_probs && !zp)
    TQS_CUDA(cudaMemcpyAsync(h_probs, dp, amps * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H probs");
  if (h_norms && !zn)
    TQS_CUDA(cudaMemcpyAsync(h_norms, dn, size_t(b->count) * sizeof(double), cudaMemcpyDeviceToHost, s),
             "D2H norms");
  if (A.alloc) dev_free(A, base, s);
  else TQS_CUDA(cudaFreeAsync(base, s), "tqs_batch_run_host: cudaFreeAsync");
  // wait without spinning, so that host threads compiling other batches keep the cores
  cudaEvent_t done = nullptr;
  TQS_CUDA(cudaEventCreateWithFlags(&done, cudaEventBlockingSync | cudaEventDisableTiming),
           "tqs_batch_run_host: event");
  cudaError_t e = cudaEventRecord(done, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(done);
  cudaEventDestroy(done);
  TQS_CUDA(e, "tqs_batch_run_host: sync");
  return TQS_OK;
}

tqs_status tqs_batch_destroy(tqs_batch* b) {
  delete b;
  return TQS_OK;
}

}  // extern "C"

// Columns [col0, col0 + ncols) of the circuit unitary (Algorithm 1) into
// d_U[r * ldu + j] = U[r][col0 + j]; the whole unitary is the block col0 = 0,
// ncols = ldu = 2^n.
static tqs_status unitary_block(tqs_circuit* c, int prec, int col0, int ncols, tqs_c64* d_U,
                                int64_t ldu, void* stream, const char* who) {
  if (c && c->n_instr > 0)
    return fail(TQS_ERR_UNSUPPORTED, "%s: measure/reset instructions have no circuit unitary", who);
  if (!c || !d_U) return fail(TQS_ERR_ARG, "%s: NULL argument", who);
  if (!aligned16(d_U)) return fail(TQS_ERR_ARG, "%s: d_U must be 16-byte aligned", who);
  if (c->n > TQS_MAX_DENSE_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "%s: n %d > %d", who, c->n, TQS_MAX_DENSE_QUBITS);
  if (prec != TQS_PREC_FP32_SIMT && prec != TQS_PREC_TC_BF16X3 && prec != TQS_PREC_TC_TF32X3)
    return fail(TQS_ERR_ARG, "%s: unknown precision %d", who, prec);
  if (prec != TQS_PREC_FP32_SIMT && c->n < 7)
    return fail(TQS_ERR_ARG, "%s: the tensor-core chain needs n >= 7", who);
  const int N = 1 << c->n;
  if (col0 < 0 || ncols < 1 || col0 > N - ncols || ldu < ncols)
    return fail(TQS_ERR_ARG, "%s: column block [%d, %d + %d) or ldu %lld outside the %d columns", who,
                col0, col0, ncols, static_cast<long long>(ldu), N);
  if (c->n >= 7 && (col0 % 128 != 0 || ncols % 128 != 0))
    return fail(TQS_ERR_ARG, "%s: for n >= 7, col0 and ncols must be multiples of 128", who);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tqs_status st = upload_factors(c, s);
  if (st != TQS_OK) return st;
  float2* U = reinterpret_cast<float2*>(d_U);
  if (c->nsteps <= 1) {
    // Algorithm 1 with at most one step: U = S_1 (or the identity).
    StepDesc d = c->nsteps == 1 ? c->steps[0] : StepDesc{0, 0, (1u << c->n) - 1u, 0};
    if (col0 == 0 && ncols == N && ldu == N) {
      TQS_CUDA(launch_materialize(c->d_factors.as<StepFactor>(), d, c->n, U, s),
               "tqs_circuit_unitary: materialize");
      return TQS_OK;
    }
    TQS_CUDA(c->d_chain.ensure(size_t(N) * N * sizeof(float2)), "tqs_circuit_unitary: cudaMalloc");
    float2* S = c->d_chain.as<float2>();
    TQS_CUDA(launch_materialize(c->d_factors.as<StepFactor>(), d, c->n, S, s),
             "tqs_circuit_unitary: materialize");
    TQS_CUDA(cudaMemcpy2DAsync(U, size_t(ldu) * sizeof(float2), S + col0, size_t(N) * sizeof(float2),
                               size_t(ncols) * sizeof(float2), size_t(N), cudaMemcpyDeviceToDevice, s),
             "tqs_circuit_unitary: copy block");
    return TQS_OK;
  }
  if (prec == TQS_PREC_FP32_SIMT) {
    TQS_CUDA(c->d_chain.ensure(chain_simt_scratch_bytes(c->n, ncols)), "tqs_circuit_unitary: cudaMalloc");
    TQS_CUDA(chain_simt(c->d_factors.as<StepFactor>(), c->steps.data(), c->nsteps, c->n, col0, ncols,
                        U, ldu, c->d_chain.p, s),
             "tqs_circuit_unitary: SIMT chain");
    return TQS_OK;
  }
  TQS_CUDA(c->d_chain.ensure(chain_tc_scratch_bytes(c->n, prec, ncols)), "tqs_circuit_unitary: cudaMalloc");
  TQS_CUDA(c->d_err.ensure(sizeof(int)), "tqs_circuit_unitary: cudaMalloc");
  TQS_CUDA(cudaMemsetAsync(c->d_err.p, 0, sizeof(int), s), "tqs_circuit_unitary: memset");
  TQS_CUDA(chain_tc(c->d_factors.as<StepFactor>(), c->steps.data(), c->nsteps, c->n, prec, col0, ncols,
                    U, ldu, c->d_chain.p, c->d_err.as<int>(), g_chain_group.load(),
                    g_chain_kchunk.load(), g_chain_pair.load(), s),
           "tqs_circuit_unitary: tensor-core chain");
  int err = 0;
  TQS_CUDA(cudaMemcpyAsync(&err, c->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s),
           "tqs_circuit_unitary: read status");
  TQS_CUDA(cudaStreamSynchronize(s), "tqs_circuit_unitary: sync");
  if (err) return fail(TQS_ERR_TIMEOUT, "%s: a device wait ran out", who);
  return TQS_OK;
}

extern "C" {

tqs_status tqs_circuit_unitary(tqs_circuit* c, int prec, tqs_c64* d_U, void* stream) {
  if (c && c->n > TQS_MAX_DENSE_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_circuit_unitary: n %d > %d", c->n, TQS_MAX_DENSE_QUBITS);
  const int N = c ? 1 << c->n : 1;
  return unitary_block(c, prec, 0, N, d_U, N, stream, "tqs_circuit_unitary");
}

tqs_status tqs_circuit_unitary_cols(tqs_circuit* c, int prec, int col0, int ncols, tqs_c64* d_U,
                                    int64_t ldu, void* stream) {
  return unitary_block(c, prec, col0, ncols, d_U, ldu, stream, "tqs_circuit_unitary_cols");
}

}  // extern "C"

