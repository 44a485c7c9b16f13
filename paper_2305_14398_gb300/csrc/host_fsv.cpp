// Sampling and collapse (tqs_sample, tqs_simulate_and_collapse,
// tqs_batch_sample) and the full-state-vector backend (tqs_simulate_fsv).
#include "host_common.h"


// ---------------------------------------------------------------- collapse
// Inverse-CDF sampling (simulateAndCollapse, Sec. 5.2).  Scratch layout:
// [global-path segments][shared-memory-path segments][block totals]
// [block prefixes][chunk prefixes][segment totals].

namespace {

DevBuf& sample_scratch_tls() {
  static thread_local DevBuf buf;
  return buf;
}

}  // namespace

// One probability vector, global path (its shots spread over the whole GPU).
static tqs_status sample_one_state(DevBuf& buf, const double* d_probs, int n, int64_t shots,
                                   const double* d_u, int64_t* d_out, cudaStream_t s,
                                   const char* who) {
  SamplePlan plan;
  plan.add(0, 0, n, false);
  plan.layout();
  TQS_CUDA(buf.ensure(plan.bytes), "sample: cudaMalloc scratch");
  TQS_CUDA(plan.upload(buf.as<char>(), s), "sample: upload segment");
  TQS_CUDA(launch_sample(plan.launch(buf.as<char>(), d_probs, d_u, shots, d_out), s), who);
  return TQS_OK;
}

extern "C" {

tqs_status tqs_sample(const double* d_probs, int n, int64_t shots, const double* d_u,
                      int64_t* d_out, void* stream) {
  if (!d_probs) return fail(TQS_ERR_ARG, "tqs_sample: d_probs is NULL");
  if (n < 1 || n > 30) return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_sample: n %d outside [1, 30]", n);
  if (shots < 0) return fail(TQS_ERR_ARG, "tqs_sample: shots < 0");
  if (shots > 0 && (!d_u || !d_out)) return fail(TQS_ERR_ARG, "tqs_sample: NULL d_u or d_out");
  return sample_one_state(sample_scratch_tls(), d_probs, n, shots, d_u, d_out,
                          static_cast<cudaStream_t>(stream), "tqs_sample: launch");
}

tqs_status tqs_simulate_and_collapse(tqs_circuit* c, const double* d_u, int64_t* d_index,
                                     tqs_c64* d_state, void* stream) {
  if (!c || !d_u || !d_index)
    return fail(TQS_ERR_ARG, "tqs_simulate_and_collapse: NULL circuit, d_u or d_index");
  if (c->n > TQS_MAX_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_simulate_and_collapse: n %d > %d", c->n, TQS_MAX_QUBITS);
  if (d_state && !aligned16(d_state))
    return fail(TQS_ERR_ARG, "tqs_simulate_and_collapse: d_state must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t N = size_t(1) << c->n;
  const size_t state_bytes = d_state ? 0 : N * sizeof(float2);
  TQS_CUDA(c->d_collapse.ensure(state_bytes + N * sizeof(double)),
           "tqs_simulate_and_collapse: cudaMalloc scratch");
  tqs_c64* st = d_state ? d_state : c->d_collapse.as<tqs_c64>();
  double* probs = reinterpret_cast<double*>(c->d_collapse.as<char>() + state_bytes);
  tqs_status r = tqs_simulate(c, nullptr, st, probs, nullptr, stream);
  if (r != TQS_OK) return r;
  r = sample_one_state(c->d_sample, probs, c->n, 1, d_u, d_index, s,
                       "tqs_simulate_and_collapse: sample");
  if (r != TQS_OK) return r;
  if (d_state)
    TQS_CUDA(launch_set_basis(reinterpret_cast<float2*>(d_state), c->n, d_index, s),
             "tqs_simulate_and_collapse: collapsed state");
  return TQS_OK;
}

tqs_status tqs_batch_sample(tqs_batch* b, const double* d_probs, int shots, const double* d_u,
                            int64_t* d_out, void* stream) {
  if (!b || !d_probs) return fail(TQS_ERR_ARG, "tqs_batch_sample: NULL batch or d_probs");
  if (!aligned16(d_probs)) return fail(TQS_ERR_ARG, "tqs_batch_sample: d_probs must be 16-byte aligned");
  if (shots < 0) return fail(TQS_ERR_ARG, "tqs_batch_sample: shots < 0");
  if (shots > 0 && (!d_u || !d_out)) return fail(TQS_ERR_ARG, "tqs_batch_sample: NULL d_u or d_out");
  if (shots == 0) return TQS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!b->sample_plan) {
    auto plan = std::make_unique<SamplePlan>();
    for (int i = 0; i < b->count; ++i) plan->add(i, b->offsets[i], b->img.circs[i].n, true);
    plan->layout();
    TQS_CUDA(b->d_sample.ensure(plan->bytes), "tqs_batch_sample: cudaMalloc scratch");
    TQS_CUDA(plan->upload(b->d_sample.as<char>(), s), "tqs_batch_sample: upload segments");
    TQS_CUDA(cudaStreamSynchronize(s), "tqs_batch_sample: upload segments");
    b->sample_plan = std::move(plan);
  }
  TQS_CUDA(launch_sample(b->sample_plan->launch(b->d_sample.as<char>(), d_probs, d_u, shots, d_out),
                         s),
           "tqs_batch_sample: launch");
  return TQS_OK;
}

}  // extern "C"

// ------------------------------------------------------- full state vector
// Gates are grouped into passes: a pass's tile bits are the kFsvLowQ lowest
// bits plus the bits its gates act on non-diagonally (a target, a SWAP's two
// bits, a custom unitary's bits), at most T in all.  Controls and diagonal
// factors may sit on any bit.  Unused tile slots take the lowest free bits.

static tqs_status compile_fsv(int n, const std::vector<Gate>& gates, int max_gates, int tile_opt,
                              FsvProgram& P) {
  P = FsvProgram();
  P.max_gates = max_gates;
  P.tile_opt = tile_opt;
  // Automatic: 2^13-amplitude tiles from 24 qubits on (fewer passes); below
  // that 2^12, so that a state still spreads over enough tiles to fill the
  // GPU.  TQS_OPT_FSV_TILE_Q sets the tile bits instead.
  const int T = std::min(n, tile_opt > 0 ? tile_opt : (n >= 24 ? kFsvTileQ : kFsvTileQ - 1));
  const int nlow = std::min(T, kFsvLowQ);
  P.T = T;
  const uint64_t low = (uint64_t(1) << nlow) - 1;
  auto need_of = [&](const Gate& g) -> uint64_t {
    if (is_wide(g) || g.kind == TQS_SWAP) {
      uint64_t m = 0;
      for (int i = 0; i < g.nq; ++i) m |= uint64_t(1) << g.q[i];
      return m;
    }
    if (classify_mat(g.u) == G_DIAG) return 0;
    return uint64_t(1) << (is_controlled(g.kind) ? g.q[1] : g.q[0]);
  };
  for (const Gate& g : gates)
    if (is_instruction(g.kind))
      return fail(TQS_ERR_UNSUPPORTED, "tqs_simulate_fsv: measure/reset instructions are not supported");
  // One in-order scan per pass: a gate joins the pass if no earlier gate left
  // for a later pass shares a qubit with it (gates on disjoint qubits
  // commute), its non-diagonal bits fit the tile and its other bits fit the
  // far-bit budget; otherwise its qubits are blocked for the rest of the scan.
  std::vector<int> pending(gates.size()), still;
  std::iota(pending.begin(), pending.end(), 0);
  const uint64_t all = (n >= 64) ? ~uint64_t(0) : ((uint64_t(1) << n) - 1);
  std::vector<const Gate*> cur;
  std::vector<Gate> relabelled;
  while (!pending.empty()) {
    uint64_t mask = low, touched = 0, blocked = 0;
    still.clear();
    cur.clear();
    size_t i = 0;
    for (; i < pending.size() && blocked != all &&
           (max_gates == 0 || cur.size() < static_cast<size_t>(max_gates));
         ++i) {
      const Gate& g = gates[pending[i]];
      uint64_t qm = 0;
      for (int j = 0; j < g.nq; ++j) qm |= uint64_t(1) << g.q[j];
      const uint64_t need = need_of(g);
      const uint64_t m2 = mask | need;
      // far bits tested after adding g (the tile is filled to T bits from the
      // lowest free bits at the end, which can only shrink this count)
      const int far = __builtin_popcountll((touched | qm) & ~m2);
      if ((qm & blocked) || __builtin_popcountll(m2) > T || far > kFsvMaxFar) {
        blocked |= qm;
        still.push_back(pending[i]);
        continue;
      }
      mask = m2;
      touched |= qm;
      cur.push_back(&g);
    }
    for (; i < pending.size(); ++i) still.push_back(pending[i]);
    pending.swap(still);
    // fill the tile up to T bits with the lowest free bits
    for (int bit = 0; __builtin_popcountll(mask) < T && bit < n; ++bit) mask |= uint64_t(1) << bit;
    FsvPassInfo info;
    info.mask = mask;
    int map[64];
    for (int q = 0; q < 64; ++q) map[q] = -1;
    for (int q = 0, k = 0; q < n; ++q)
      if ((mask >> q) & 1) map[q] = k++;
    for (int q = 0; q < n; ++q)
      if (((touched >> q) & 1) && map[q] < 0) {
        map[q] = T + info.nfar;
        info.far[info.nfar++] = static_cast<uint8_t>(q);
      }
    relabelled.assign(cur.size(), Gate{});
    std::vector<const Gate*> ptrs(cur.size());
    for (size_t k = 0; k < cur.size(); ++k) {
      relabelled[k] = *cur[k];
      for (int j = 0; j < kMaxCustomQubits; ++j)
        relabelled[k].q[j] = (j < cur[k]->nq) ? map[cur[k]->q[j]] : map[cur[k]->q[0]];
      ptrs[k] = &relabelled[k];
    }
    Program tp;
    compile_program(T + info.nfar, ptrs, tp, false, false);
    P.passes.push_back(info);
    P.progs.push_back(std::move(tp));
  }
  return TQS_OK;
}

extern "C" {

tqs_status tqs_simulate_fsv(tqs_circuit* c, tqs_c64* d_state, void* stream) {
  if (!c || !d_state) return fail(TQS_ERR_ARG, "tqs_simulate_fsv: NULL circuit or state");
  if (!aligned16(d_state)) return fail(TQS_ERR_ARG, "tqs_simulate_fsv: d_state must be 16-byte aligned");
  if (c->n_instr > 0)
    return fail(TQS_ERR_UNSUPPORTED, "tqs_simulate_fsv: measure/reset instructions are not supported");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c->n < 4) {
    // smaller than any tile: the fused kernel, from a copy of the state
    const size_t bytes = (size_t(1) << c->n) * sizeof(float2);
    TQS_CUDA(c->d_collapse.ensure(bytes), "tqs_simulate_fsv: cudaMalloc");
    TQS_CUDA(cudaMemcpyAsync(c->d_collapse.p, d_state, bytes, cudaMemcpyDeviceToDevice, s),
             "tqs_simulate_fsv: copy");
    return tqs_simulate(c, c->d_collapse.as<tqs_c64>(), d_state, nullptr, nullptr, stream);
  }
  const int max_gates = g_fsv_max_gates.load();
  const int tile_opt = g_fsv_tile_q.load();
  if (!c->fsv_valid || c->fsv.max_gates != max_gates || c->fsv.tile_opt != tile_opt) {
    tqs_status st = compile_fsv(c->n, c->gates, max_gates, tile_opt, c->fsv);
    if (st != TQS_OK) return st;
    c->fsv_img = Image();
    for (const Program& tp : c->fsv.progs) c->fsv_img.add(tp, 0);
    TQS_CUDA(c->d_fsv.ensure(c->fsv_img.bytes()), "tqs_simulate_fsv: cudaMalloc");
    TQS_CUDA(c->fsv_img.upload(c->d_fsv.p, s), "tqs_simulate_fsv: upload");
    c->fsv_valid = true;
  }
  FusedLaunch L{};
  c->fsv_img.point(L, c->d_fsv.as<char>());
  const FusedCirc* circs = L.circs;
  for (size_t k = 0; k < c->fsv.passes.size(); ++k) {
    const FsvPassInfo& info = c->fsv.passes[k];
    FsvTile F{};
    F.state = reinterpret_cast<float2*>(d_state);
    F.mask = info.mask;
    F.n = c->n;
    F.T = c->fsv.T;
    F.nfar = info.nfar;
    std::memcpy(F.far, info.far, sizeof(F.far));
    L.circs = circs + k;
    TQS_CUDA(launch_fsv_tile(L, F, s), "tqs_simulate_fsv: launch");
  }
  return TQS_OK;
}

tqs_status tqs_fsv_passes(tqs_circuit* c, int* n_passes, int* tile_bits) {
  if (!c) return fail(TQS_ERR_ARG, "tqs_fsv_passes: circuit is NULL");
  FsvProgram local;
  const FsvProgram* P = &c->fsv;
  const int max_gates = g_fsv_max_gates.load();
  const int tile_opt = g_fsv_tile_q.load();
  if (!c->fsv_valid || c->fsv.max_gates != max_gates || c->fsv.tile_opt != tile_opt) {
    tqs_status st = compile_fsv(c->n, c->gates, max_gates, tile_opt, local);
    if (st != TQS_OK) return st;
    P = &local;
  }
  if (n_passes) *n_passes = static_cast<int>(P->passes.size());
  if (tile_bits) *tile_bits = P->T;
  return TQS_OK;
}

}  // extern "C"

