// Host side of the C ABI (include/tqs.h): errors, the circuit model and its
// step packing (tqs_circuit_*, tqs_add_gate, custom unitaries), single-circuit
// simulation, the plain form, probabilities, options and the allocator hook.
// Batches, the server, sampling and the full-state-vector backend live in
// host_batch.cpp, host_server.cpp and host_fsv.cpp, the pass compiler in
// host_compile.cpp; their shared types are in host_common.h.
//
// Sec. 5.2: the circuit model records operations and creates steps as they
// are added; the data provider supplies each operation's matrix separately
// from the circuit structure.  Sec. 5.3: stages 1-3 (steps, operations per
// step, operation data) run here; stages 4-6 run in the kernels.
#include "host_common.h"

namespace tqs {

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_last_error(const char* msg) { g_last_error = msg; }

}  // namespace tqs

extern "C" {

const char* tqs_last_error(void) { return g_last_error.c_str(); }

const char* tqs_status_string(int s) {
  switch (s) {
    case TQS_OK: return "TQS_OK";
    case TQS_ERR_ARG: return "TQS_ERR_ARG";
    case TQS_ERR_QUBIT_RANGE: return "TQS_ERR_QUBIT_RANGE";
    case TQS_ERR_QUBIT_DUP: return "TQS_ERR_QUBIT_DUP";
    case TQS_ERR_TOO_MANY_QUBITS: return "TQS_ERR_TOO_MANY_QUBITS";
    case TQS_ERR_NOMEM: return "TQS_ERR_NOMEM";
    case TQS_ERR_BUDGET: return "TQS_ERR_BUDGET";
    case TQS_ERR_CUDA: return "TQS_ERR_CUDA";
    case TQS_ERR_TIMEOUT: return "TQS_ERR_TIMEOUT";
    case TQS_ERR_STATE: return "TQS_ERR_STATE";
    case TQS_ERR_UNSUPPORTED: return "TQS_ERR_UNSUPPORTED";
    default: return "TQS_ERR_UNKNOWN";
  }
}

int64_t tqs_launch_count(void) { return g_launches.load(); }

tqs_status tqs_circuit_create(int n_qubits, tqs_circuit** out) {
  if (!out) return fail(TQS_ERR_ARG, "tqs_circuit_create: out is NULL");
  *out = nullptr;
  if (n_qubits < 1) return fail(TQS_ERR_ARG, "tqs_circuit_create: n_qubits must be >= 1");
  if (n_qubits > TQS_MAX_FSV_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_circuit_create: n_qubits %d > %d", n_qubits,
                TQS_MAX_FSV_QUBITS);
  tqs_circuit* c = new (std::nothrow) tqs_circuit();
  if (!c) return fail(TQS_ERR_NOMEM, "tqs_circuit_create: out of host memory");
  c->n = n_qubits;
  c->last.assign(n_qubits, -1);
  *out = c;
  return TQS_OK;
}

tqs_status tqs_circuit_destroy(tqs_circuit* c) {
  delete c;
  return TQS_OK;
}


}  // extern "C"


extern "C" {

tqs_status tqs_add_gate(tqs_circuit* c, int gate, const int* qubits, int nq, const double* params,
                        int np) {
  if (!c) return fail(TQS_ERR_ARG, "tqs_add_gate: circuit is NULL");
  Gate g{};
  tqs_status s = check_gate(c->n, gate, qubits, nq, params, np, g);
  if (s != TQS_OK) return s;
  assign_step(c->last, g);
  if (is_instruction(gate)) ++c->n_instr;
  const int step = g.step;
  c->nsteps = std::max(c->nsteps, step + 1);
  c->gates.push_back(g);
  c->prog_valid = false;
  c->prog_init_valid = false;
  c->uploaded = false;
  c->steps_valid = false;
  c->fsv_valid = false;
  return TQS_OK;
}

}  // extern "C"

// Process-wide registry of custom unitaries (the operation data provider of
// Sec. 5.2): name -> matrix.  Circuits keep their own reference to the data
// they were built with.
static std::mutex g_registry_mu;
static std::unordered_map<std::string, std::shared_ptr<const CustomMat>> g_registry;

extern "C" {

tqs_status tqs_register_unitary(const char* name, int k, const double* m) {
  if (!name || !*name || !m) return fail(TQS_ERR_ARG, "tqs_register_unitary: NULL name or matrix");
  if (k < 1 || k > kMaxCustomQubits)
    return fail(TQS_ERR_ARG, "tqs_register_unitary: k %d outside [1, %d]", k, kMaxCustomQubits);
  auto cm = std::make_shared<CustomMat>();
  const int G = 1 << k;
  cm->k = k;
  cm->m.resize(size_t(G) * G);
  for (size_t i = 0; i < cm->m.size(); ++i) {
    if (!std::isfinite(m[2 * i]) || !std::isfinite(m[2 * i + 1]))
      return fail(TQS_ERR_ARG, "tqs_register_unitary: non-finite entry");
    cm->m[i] = cd(m[2 * i], m[2 * i + 1]);
  }
  // unitary to 1e-9: every entry of M^dagger M - I
  for (int a = 0; a < G; ++a)
    for (int b = 0; b < G; ++b) {
      cd acc = 0.0;
      for (int r = 0; r < G; ++r) acc += std::conj(cm->m[size_t(r) * G + a]) * cm->m[size_t(r) * G + b];
      if (std::abs(acc - (a == b ? 1.0 : 0.0)) > 1e-9)
        return fail(TQS_ERR_ARG, "tqs_register_unitary: '%s' is not unitary to 1e-9", name);
    }
  std::lock_guard<std::mutex> lock(g_registry_mu);
  g_registry[name] = std::move(cm);
  return TQS_OK;
}

tqs_status tqs_add_custom(tqs_circuit* c, const char* name, const int* qubits, int k) {
  if (!c || !name || !qubits) return fail(TQS_ERR_ARG, "tqs_add_custom: NULL argument");
  std::shared_ptr<const CustomMat> cm;
  {
    std::lock_guard<std::mutex> lock(g_registry_mu);
    auto it = g_registry.find(name);
    if (it == g_registry.end())
      return fail(TQS_ERR_ARG, "tqs_add_custom: no unitary registered as '%s'", name);
    cm = it->second;
  }
  if (k != cm->k)
    return fail(TQS_ERR_ARG, "tqs_add_custom: '%s' acts on %d qubit(s), got %d", name, cm->k, k);
  for (int i = 0; i < k; ++i) {
    if (qubits[i] < 0 || qubits[i] >= c->n)
      return fail(TQS_ERR_QUBIT_RANGE, "qubit %d outside [0, %d)", qubits[i], c->n);
    for (int j = 0; j < i; ++j)
      if (qubits[j] == qubits[i])
        return fail(TQS_ERR_QUBIT_DUP, "tqs_add_custom: qubit %d twice", qubits[i]);
  }
  Gate g{};
  g.kind = kCustomKind;
  g.nq = k;
  for (int i = 0; i < k; ++i) g.q[i] = qubits[i];
  for (int i = k; i < kMaxCustomQubits; ++i) g.q[i] = qubits[0];
  if (k == 1) {
    for (int i = 0; i < 4; ++i) g.u.m[i] = cm->m[i];  // a dense single-qubit factor
  } else {
    g.u = Mat2{{1.0, 0.0, 0.0, 1.0}};
    g.cm = cm;
  }
  assign_step(c->last, g);
  c->nsteps = std::max(c->nsteps, g.step + 1);
  c->gates.push_back(g);
  c->prog_valid = false;
  c->prog_init_valid = false;
  c->uploaded = false;
  c->steps_valid = false;
  c->fsv_valid = false;
  return TQS_OK;
}

tqs_status tqs_circuit_info(const tqs_circuit* c, int* n_qubits, int* n_gates, int* n_steps) {
  if (!c) return fail(TQS_ERR_ARG, "tqs_circuit_info: circuit is NULL");
  if (n_qubits) *n_qubits = c->n;
  if (n_gates) *n_gates = static_cast<int>(c->gates.size());
  if (n_steps) *n_steps = c->nsteps;
  return TQS_OK;
}

tqs_status tqs_circuit_steps(const tqs_circuit* c, int* h_step_of_gate) {
  if (!c || !h_step_of_gate) return fail(TQS_ERR_ARG, "tqs_circuit_steps: NULL argument");
  for (size_t i = 0; i < c->gates.size(); ++i) h_step_of_gate[i] = c->gates[i].step;
  return TQS_OK;
}

}  // extern "C"



extern "C" tqs_status tqs_circuit_program(tqs_circuit* c, int* n_passes, int* n_ops, void* h_passes,
                                          void* h_ops, uint16_t* h_map, float* h_out_scale,
                                          int* h_gen_index) {
  if (!c) return fail(TQS_ERR_ARG, "tqs_circuit_program: circuit is NULL");
  if (c->n > TQS_MAX_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_circuit_program: n %d > %d", c->n, TQS_MAX_QUBITS);
  ensure_program(c);
  if (h_gen_index) *h_gen_index = c->prog.gen_index;
  if (n_passes) *n_passes = static_cast<int>(c->prog.passes.size());
  if (n_ops) *n_ops = static_cast<int>(c->prog.ops.size());
  if (h_passes) std::memcpy(h_passes, c->prog.passes.data(), c->prog.passes.size() * sizeof(FusedPass));
  if (h_ops) std::memcpy(h_ops, c->prog.ops.data(), c->prog.ops.size() * sizeof(FusedOp));
  if (h_map) {
    std::memcpy(h_map, c->prog.col, sizeof(c->prog.col));
    h_map[16] = c->prog.col_off;
  }
  if (h_out_scale) *h_out_scale = c->prog.out_scale;
  return TQS_OK;
}






static tqs_status simulate_impl(tqs_circuit* c, const tqs_c64* d_init, tqs_c64* d_out,
                                double* d_probs, double* d_norm, const double* d_u,
                                int32_t* d_outcomes, void* stream) {
  if (c && c->n > TQS_MAX_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_simulate: n %d > %d (tqs_simulate_fsv takes up to %d)",
                c->n, TQS_MAX_QUBITS, TQS_MAX_FSV_QUBITS);
  if (!c || !d_out) return fail(TQS_ERR_ARG, "tqs_simulate: NULL circuit or output");
  if (c->n_instr > 0 && !d_u)
    return fail(TQS_ERR_ARG, "tqs_simulate_measured: the circuit has %d instruction(s): d_u is NULL",
                c->n_instr);
  if (!aligned16(d_out) || (d_probs && !aligned16(d_probs)) || (d_init && !aligned16(d_init)))
    return fail(TQS_ERR_ARG, "tqs_simulate: device buffers must be 16-byte aligned");
  if (d_init && reinterpret_cast<const void*>(d_init) == reinterpret_cast<const void*>(d_out))
    return fail(TQS_ERR_ARG, "tqs_simulate: d_init must not alias d_out");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Program& P = ensure_program(c, d_init != nullptr);
  const int team = team_for(P.nint);
  Image img;
  img.add(P, 0);
  img.circs[0].init = reinterpret_cast<const float2*>(d_init);
  const size_t order_off = (img.bytes() + 255) & ~size_t(255);
  // The device program is uploaded once per (program, initial-state pointer)
  // and reused by later calls on the circuit.
  if (!c->uploaded || c->uploaded_prog != &P || c->uploaded_init != d_init) {
    c->uploaded = false;
    TQS_CUDA(c->d_prog.ensure(order_off + 256), "tqs_simulate: cudaMalloc program");
    TQS_CUDA(img.upload(c->d_prog.p, s), "tqs_simulate: upload program");
    // order[0] = 0 lives right after the image
    static const int32_t zero_order[1] = {0};
    TQS_CUDA(cudaMemcpyAsync(c->d_prog.as<char>() + order_off, zero_order, sizeof(int32_t),
                             cudaMemcpyHostToDevice, s),
             "tqs_simulate: upload order");
    if (!c->upload_done)
      TQS_CUDA(cudaEventCreateWithFlags(&c->upload_done, cudaEventDisableTiming),
               "tqs_simulate: event");
    TQS_CUDA(cudaEventRecord(c->upload_done, s), "tqs_simulate: event");
    c->upload_stream = s;
    c->uploaded = true;
    c->uploaded_prog = &P;
    c->uploaded_init = d_init;
  } else if (s != c->upload_stream) {
    // another stream reuses the program: its kernels wait for the upload
    TQS_CUDA(cudaStreamWaitEvent(s, c->upload_done, 0), "tqs_simulate: wait upload");
  }
  TQS_CUDA(c->d_counter.ensure(2 * sizeof(int32_t)), "tqs_simulate: cudaMalloc counter");
  char* base = c->d_prog.as<char>();
  TQS_CUDA(cudaMemsetAsync(c->d_counter.p, 0, 2 * sizeof(int32_t), s), "tqs_simulate: memset");
  FusedLaunch L{};
  img.point(L, base);
  L.order = reinterpret_cast<const int32_t*>(base + order_off);
  L.n_jobs = 1;
  L.counter = c->d_counter.as<int32_t>();
  L.out = reinterpret_cast<float2*>(d_out);
  L.probs = d_probs;
  L.exact_probs = g_exact_probs.load();
  L.norms = d_norm;
  L.uniforms = d_u;
  L.outcomes = d_outcomes;
  LaunchPlan lp = plan_for(team, P.nint, 1, 1);
  if (team == TEAM_GLOBAL) {
    TQS_CUDA(c->d_gscratch.ensure((size_t(1) << kGlobalSlotQ) * sizeof(float2)),
             "tqs_simulate: cudaMalloc scratch");
    L.gscratch = c->d_gscratch.as<float2>();
  }
  L.team = lp.team;
  L.warps_per_cta = lp.warps;
  L.slice_q = lp.slice_q;
  L.grid = 1;
  // A single circuit of the global class runs on several CTAs (TEAM_MULTI,
  // bitwise the same results) when it has no instructions or custom unitaries.
  const int multi = multi_ctas_for(P);
  if (team == TEAM_GLOBAL && multi >= 2) {
    L.team = TEAM_MULTI;
    L.grid = multi;
    L.ctas_per_job = multi;
    L.err = c->d_counter.as<int32_t>() + 1;  // zeroed with the counter above
  }
  TQS_CUDA(launch_fused(L, s), "tqs_simulate: launch");
  return TQS_OK;
}

extern "C" {

tqs_status tqs_simulate(tqs_circuit* c, const tqs_c64* d_init, tqs_c64* d_out, double* d_probs,
                        double* d_norm, void* stream) {
  if (c && c->n_instr > 0)
    return fail(TQS_ERR_UNSUPPORTED,
                "tqs_simulate: the circuit holds measure/reset instructions: use tqs_simulate_measured");
  return simulate_impl(c, d_init, d_out, d_probs, d_norm, nullptr, nullptr, stream);
}

tqs_status tqs_simulate_measured(tqs_circuit* c, const tqs_c64* d_init, tqs_c64* d_out,
                                 double* d_probs, double* d_norm, const double* d_u,
                                 int32_t* d_outcomes, void* stream) {
  return simulate_impl(c, d_init, d_out, d_probs, d_norm, d_u, d_outcomes, stream);
}

}  // extern "C"

// ------------------------------------------------------ plain step table



extern "C" {

tqs_status tqs_materialize_step(tqs_circuit* c, int step, tqs_c64* d_S, void* stream) {
  if (c && c->n_instr > 0)
    return fail(TQS_ERR_UNSUPPORTED, "tqs_materialize_step: the circuit holds measure/reset instructions");
  if (!c || !d_S) return fail(TQS_ERR_ARG, "tqs_materialize_step: NULL argument");
  if (c->n > TQS_MAX_DENSE_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_materialize_step: n %d > %d", c->n,
                TQS_MAX_DENSE_QUBITS);
  if (step < 0 || step >= c->nsteps)
    return fail(TQS_ERR_ARG, "tqs_materialize_step: step %d outside [0, %d)", step, c->nsteps);
  if (!aligned16(d_S)) return fail(TQS_ERR_ARG, "tqs_materialize_step: d_S must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tqs_status st = upload_factors(c, s);
  if (st != TQS_OK) return st;
  TQS_CUDA(launch_materialize(c->d_factors.as<StepFactor>(), c->steps[step], c->n,
                              reinterpret_cast<float2*>(d_S), s),
           "tqs_materialize_step: launch");
  return TQS_OK;
}

tqs_status tqs_simulate_plain(tqs_circuit* c, const tqs_c64* d_init, tqs_c64* d_out, void* stream) {
  if (c && c->n_instr > 0)
    return fail(TQS_ERR_UNSUPPORTED, "tqs_simulate_plain: the circuit holds measure/reset instructions");
  if (!c || !d_out) return fail(TQS_ERR_ARG, "tqs_simulate_plain: NULL argument");
  if (c->n > TQS_MAX_DENSE_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_simulate_plain: n %d > %d", c->n,
                TQS_MAX_DENSE_QUBITS);
  if (!aligned16(d_out) || (d_init && !aligned16(d_init)))
    return fail(TQS_ERR_ARG, "tqs_simulate_plain: device buffers must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tqs_status st = upload_factors(c, s);
  if (st != TQS_OK) return st;
  const size_t N = size_t(1) << c->n;
  const size_t sbytes = N * N * sizeof(float2);
  TQS_CUDA(c->d_plain.ensure(sbytes + 2 * N * sizeof(float2)), "tqs_simulate_plain: cudaMalloc");
  float2* S = c->d_plain.as<float2>();
  float2* x = reinterpret_cast<float2*>(reinterpret_cast<char*>(c->d_plain.p) + sbytes);
  float2* y = x + N;
  if (d_init) {
    TQS_CUDA(cudaMemcpyAsync(x, d_init, N * sizeof(float2), cudaMemcpyDeviceToDevice, s), "copy init");
  } else {
    TQS_CUDA(cudaMemsetAsync(x, 0, N * sizeof(float2), s), "memset init");
    const float2 one = make_float2(1.f, 0.f);
    TQS_CUDA(cudaMemcpyAsync(x, &one, sizeof(float2), cudaMemcpyHostToDevice, s), "init |0>");
  }
  for (int k = 0; k < c->nsteps; ++k) {
    TQS_CUDA(launch_materialize(c->d_factors.as<StepFactor>(), c->steps[k], c->n, S, s),
             "tqs_simulate_plain: materialize");
    TQS_CUDA(launch_matvec(S, x, y, c->n, s), "tqs_simulate_plain: matvec");
    std::swap(x, y);
  }
  TQS_CUDA(cudaMemcpyAsync(d_out, x, N * sizeof(float2), cudaMemcpyDeviceToDevice, s), "copy out");
  return TQS_OK;
}

// ------------------------------------------------------------ probabilities

// Scratch for the partial sums: one per circuit-less call site, kept per thread.
static DevBuf& probs_scratch() {
  static thread_local DevBuf buf;
  return buf;
}

static tqs_status probs_common(const tqs_c64* d_state, int n, double* d_probs, uint64_t mask,
                               double* d_sum, cudaStream_t s, const char* who) {
  if (!d_state) return fail(TQS_ERR_ARG, "%s: d_state is NULL", who);
  if (n < 1 || n > 30) return fail(TQS_ERR_TOO_MANY_QUBITS, "%s: n %d outside [1, 30]", who, n);
  if (!aligned16(d_state) || (d_probs && !aligned16(d_probs)))
    return fail(TQS_ERR_ARG, "%s: device buffers must be 16-byte aligned", who);
  const int parts = probs_partial_count(n);
  DevBuf& buf = probs_scratch();
  TQS_CUDA(buf.ensure(size_t(parts) * sizeof(double)), "probabilities: cudaMalloc partials");
  TQS_CUDA(launch_probs(reinterpret_cast<const float2*>(d_state), n, d_probs, mask,
                        buf.as<double>(), parts, d_sum, s),
           "probabilities: launch");
  return TQS_OK;
}

tqs_status tqs_probabilities(const tqs_c64* d_state, int n, double* d_probs, double* d_sum,
                             void* stream) {
  return probs_common(d_state, n, d_probs, 0, d_sum, static_cast<cudaStream_t>(stream),
                      "tqs_probabilities");
}

tqs_status tqs_marginal_zero(const tqs_c64* d_state, int n, uint64_t mask, double* d_out,
                             void* stream) {
  if (!d_out) return fail(TQS_ERR_ARG, "tqs_marginal_zero: d_out is NULL");
  if (n >= 1 && n <= 30 && (mask >> n) != 0)
    return fail(TQS_ERR_QUBIT_RANGE, "tqs_marginal_zero: mask names qubits >= n");
  return probs_common(d_state, n, nullptr, mask, d_out, static_cast<cudaStream_t>(stream),
                      "tqs_marginal_zero");
}

}  // extern "C"



extern "C" {

tqs_status tqs_check_violations(uint32_t* count, int reset) {
  if (!count) return fail(TQS_ERR_ARG, "tqs_check_violations: count is NULL");
  using Counter = cudaError_t (*)(unsigned int*, bool);
  static const Counter counters[] = {violations_fused,  violations_plain,      violations_probs,
                                     violations_sample, violations_chain_simt, violations_chain_tc};
  uint32_t total = 0;
  for (Counter f : counters) {
    unsigned int v = 0;
    TQS_CUDA(f(&v, reset != 0), "tqs_check_violations");
    total += v;
  }
  *count = total;
  return TQS_OK;
}

tqs_status tqs_set_allocator(tqs_alloc_fn alloc, tqs_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(TQS_ERR_ARG, "tqs_set_allocator: give both callbacks or neither");
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.free = free_fn;
  g_alloc.ctx = ctx;
  return TQS_OK;
}

tqs_status tqs_set_option(int option, int key, int64_t value) {
  if (option == TQS_OPT_TEAM_WARPS) {
    if (key < 4 || key > kWarpMaxQ) return fail(TQS_ERR_ARG, "tqs_set_option: key %d outside [4, %d]", key, kWarpMaxQ);
    if (value != 1 && value != 2) return fail(TQS_ERR_ARG, "tqs_set_option: team warps %lld is not 1 or 2", static_cast<long long>(value));
    g_team_warps_for_q[key].store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_WARPS_PER_CTA) {
    if (key < 4 || key > kWarpMaxQ) return fail(TQS_ERR_ARG, "tqs_set_option: key %d outside [4, %d]", key, kWarpMaxQ);
    if (value < 1 || value > 16) return fail(TQS_ERR_ARG, "tqs_set_option: warps %lld outside [1, 16]", static_cast<long long>(value));
    g_warps_for_q[key].store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_EXACT_PROBS) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_EXACT_PROBS is not 0", key);
    if (value != 0 && value != 1) return fail(TQS_ERR_ARG, "tqs_set_option: exact probabilities %lld is not 0 or 1", static_cast<long long>(value));
    g_exact_probs.store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_HOST_WRITES) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_HOST_WRITES is not 0", key);
    if (value != 0 && value != 1) return fail(TQS_ERR_ARG, "tqs_set_option: host writes %lld is not 0 or 1", static_cast<long long>(value));
    g_host_writes.store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_MULTI_CTAS) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_MULTI_CTAS is not 0", key);
    if (value < 0 || value > 64) return fail(TQS_ERR_ARG, "tqs_set_option: CTAs %lld outside [0, 64]", static_cast<long long>(value));
    g_multi_ctas.store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_FSV_MAX_GATES) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_FSV_MAX_GATES is not 0", key);
    if (value < 0 || value > (int64_t(1) << 30)) return fail(TQS_ERR_ARG, "tqs_set_option: gates per pass %lld outside [0, 2^30]", static_cast<long long>(value));
    g_fsv_max_gates.store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_CTA_THREADS) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_CTA_THREADS is not 0", key);
    if (value != 256 && value != 512) return fail(TQS_ERR_ARG, "tqs_set_option: CTA threads %lld is not 256 or 512", static_cast<long long>(value));
    g_cta_threads.store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_FSV_TILE_Q) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_FSV_TILE_Q is not 0", key);
    if (value != 0 && (value < 10 || value > kFsvTileQ)) return fail(TQS_ERR_ARG, "tqs_set_option: tile bits %lld not 0 or in [10, %d]", static_cast<long long>(value), kFsvTileQ);
    g_fsv_tile_q.store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_CHAIN_GROUP) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_CHAIN_GROUP is not 0", key);
    if (value < 1 || value > 64) return fail(TQS_ERR_ARG, "tqs_set_option: raster band %lld outside [1, 64]", static_cast<long long>(value));
    g_chain_group.store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_CHAIN_KCHUNK) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_CHAIN_KCHUNK is not 0", key);
    if (value < 0 || value > (int64_t(1) << 20) || value % 64)
      return fail(TQS_ERR_ARG, "tqs_set_option: K chunk %lld is not 0 or a multiple of 64 up to 2^20",
                  static_cast<long long>(value));
    g_chain_kchunk.store(static_cast<int>(value));
    return TQS_OK;
  }
  if (option == TQS_OPT_CHAIN_PAIR) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_set_option: key %d of TQS_OPT_CHAIN_PAIR is not 0", key);
    if (value != 0 && value != 1)
      return fail(TQS_ERR_ARG, "tqs_set_option: TQS_OPT_CHAIN_PAIR %lld is not 0 or 1", static_cast<long long>(value));
    g_chain_pair.store(static_cast<int>(value));
    return TQS_OK;
  }
  return fail(TQS_ERR_ARG, "tqs_set_option: unknown option %d", option);
}

tqs_status tqs_get_option(int option, int key, int64_t* value) {
  if (!value) return fail(TQS_ERR_ARG, "tqs_get_option: value is NULL");
  if (option == TQS_OPT_TEAM_WARPS) {
    if (key < 4 || key > kWarpMaxQ) return fail(TQS_ERR_ARG, "tqs_get_option: key %d outside [4, %d]", key, kWarpMaxQ);
    *value = g_team_warps_for_q[key].load();
    return TQS_OK;
  }
  if (option == TQS_OPT_WARPS_PER_CTA) {
    if (key < 4 || key > kWarpMaxQ) return fail(TQS_ERR_ARG, "tqs_get_option: key %d outside [4, %d]", key, kWarpMaxQ);
    *value = g_warps_for_q[key].load();
    return TQS_OK;
  }
  if (option == TQS_OPT_EXACT_PROBS) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_get_option: key %d of TQS_OPT_EXACT_PROBS is not 0", key);
    *value = g_exact_probs.load();
    return TQS_OK;
  }
  if (option == TQS_OPT_HOST_WRITES) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_get_option: key %d of TQS_OPT_HOST_WRITES is not 0", key);
    *value = g_host_writes.load();
    return TQS_OK;
  }
  if (option == TQS_OPT_MULTI_CTAS) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_get_option: key %d of TQS_OPT_MULTI_CTAS is not 0", key);
    *value = g_multi_ctas.load();
    return TQS_OK;
  }
  if (option == TQS_OPT_FSV_MAX_GATES) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_get_option: key %d of TQS_OPT_FSV_MAX_GATES is not 0", key);
    *value = g_fsv_max_gates.load();
    return TQS_OK;
  }
  if (option == TQS_OPT_CHAIN_PAIR) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_get_option: key %d of option %d is not 0", key, option);
    *value = g_chain_pair.load();
    return TQS_OK;
  }
  if (option == TQS_OPT_CTA_THREADS || option == TQS_OPT_FSV_TILE_Q || option == TQS_OPT_CHAIN_GROUP ||
      option == TQS_OPT_CHAIN_KCHUNK) {
    if (key != 0) return fail(TQS_ERR_ARG, "tqs_get_option: key %d of option %d is not 0", key, option);
    *value = option == TQS_OPT_CTA_THREADS  ? g_cta_threads.load()
             : option == TQS_OPT_FSV_TILE_Q ? g_fsv_tile_q.load()
             : option == TQS_OPT_CHAIN_GROUP ? g_chain_group.load()
                                             : g_chain_kchunk.load();
    return TQS_OK;
  }
  return fail(TQS_ERR_ARG, "tqs_get_option: unknown option %d", option);
}

tqs_status tqs_selftest_wait_timeout(int64_t wait_cycles, void* stream) {
  if (wait_cycles < 1 || wait_cycles > (int64_t(1) << 31))
    return fail(TQS_ERR_ARG, "tqs_selftest_wait_timeout: wait_cycles outside [1, 2^31]");
  static thread_local DevBuf status;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TQS_CUDA(status.ensure(sizeof(int)), "tqs_selftest_wait_timeout: cudaMalloc");
  TQS_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), s), "tqs_selftest_wait_timeout: memset");
  TQS_CUDA(launch_wait_selftest(status.as<int>(), wait_cycles, s), "tqs_selftest_wait_timeout: launch");
  int h = 0;
  TQS_CUDA(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, s), "read status");
  TQS_CUDA(cudaStreamSynchronize(s), "tqs_selftest_wait_timeout: sync");
  if (h) return fail(TQS_ERR_TIMEOUT, "tqs_selftest_wait_timeout: the wait ran out (expected)");
  return TQS_OK;
}

}  // extern "C"
