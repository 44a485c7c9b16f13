// The fused-pass compiler (compile_program): a circuit's steps into passes of 4
// local qubit bits with their ops (declared, with its description, in
// host_common.h).
#include "host_common.h"

namespace tqs {

void compile_program(int n, const std::vector<const Gate*>& gs_in, Program& P,
                      bool fold_x) {
  P.n = n;
  P.nint = std::max(n, 4);
  // Leading uncontrolled X factors on a qubit that nothing has touched yet act
  // on the basis input |0...0> only by flipping that qubit: fold them into the
  // start index instead of spending butterflies (input |0...0> only).
  // scratch reused across calls on this thread (no allocation per circuit)
  static thread_local std::vector<const Gate*> gs_tls;
  static thread_local std::vector<int> pending_tls, still_tls, order_tls;
  static thread_local std::vector<CompileRaw> raw_tls;
  static thread_local std::vector<uint32_t> qmask_tls;  // per entry of gs: its qubit mask
  static thread_local std::vector<GClass> cls_tls;      // per entry of gs: its class
  std::vector<const Gate*>& gs = gs_tls;
  gs.clear();
  P.gen_index = 0;
  {
    uint32_t touched = 0;
    for (const Gate* g : gs_in) {
      if (fold_x && g->kind == TQS_X && !((touched >> g->q[0]) & 1)) {
        P.gen_index ^= 1 << g->q[0];
        continue;
      }
      touched |= qubit_mask(*g);
      gs.push_back(g);
    }
  }
  std::vector<uint32_t>& qmask = qmask_tls;
  std::vector<GClass>& gcls = cls_tls;
  qmask.resize(gs.size());
  gcls.resize(gs.size());
  for (size_t i = 0; i < gs.size(); ++i) {
    qmask[i] = qubit_mask(*gs[i]);
    gcls[i] = (is_instruction(gs[i]->kind) || is_wide(*gs[i])) ? G_DENSE : classify(*gs[i]);
  }
  const int nint = P.nint;
  int phys[32];
  for (int q = 0; q < 32; ++q) phys[q] = q;
  const uint32_t all = (n >= 32) ? 0xffffffffu : ((1u << n) - 1u);
  std::vector<int>& pending = pending_tls;
  std::vector<int>& still = still_tls;
  pending.clear();
  still.clear();
  using Raw = CompileRaw;
  std::vector<Raw>& raw = raw_tls;
  raw.clear();
  int last_touch[32];
  int h_in_pass = 0;
  int h_carry = 0;  // Hadamard factors 2^-1/2 not yet applied
  auto push_raw = [&](const Gate& g, GClass cls, int t, int c) {
    const bool single = (c < 0);
    if (single) {
      const int last = last_touch[t];
      if (last >= 0 && raw[last].single && raw[last].t == t) {
        Raw& r = raw[last];
        if (r.is_h) --h_in_pass;
        r.u = mat_mul(g.u, r.u);
        r.is_h = false;
        r.cls = classify_mat(r.u);
        return;
      }
    }
    const bool is_h = single && g.kind == TQS_H && h_in_pass < kMaxHPerPass;
    if (is_h) ++h_in_pass;
    raw.push_back({g.u, cls, is_h, single, t, c});
    last_touch[t] = static_cast<int>(raw.size()) - 1;
    if (c >= 0) last_touch[c] = static_cast<int>(raw.size()) - 1;
  };
  auto emit_pass = [&](uint32_t Lmask, int nL, bool last) {
    (void)last;
    for (int b = 0; nL < 4 && b < nint; ++b)  // padding: the lowest free bits
      if (!((Lmask >> b) & 1)) { Lmask |= 1u << b; ++nL; }
    FusedPass ps{};
    int loc[32];
    for (int b = 0; b < 32; ++b) loc[b] = -1;
    int k = 0;
    for (int b = 0; b < nint; ++b)
      if ((Lmask >> b) & 1) { ps.L[k] = static_cast<uint8_t>(b); loc[b] = k++; }
    ps.op_begin = static_cast<uint32_t>(P.ops.size());
    double pass_cost = 6.0;
    int h_count = 0;
    static const uint16_t kBitMask[4] = {0xAAAA, 0xCCCC, 0xF0F0, 0xFF00};
    for (const Raw& r : raw) {
      // a factor that fused to the identity (H H, X X, ...) does nothing
      if (!r.is_h && std::abs(r.u.m[0] - 1.0) <= 1e-15 && std::abs(r.u.m[3] - 1.0) <= 1e-15 &&
          std::abs(r.u.m[1]) <= 1e-15 && std::abs(r.u.m[2]) <= 1e-15)
        continue;
      FusedOp op{};
      const Mat2& u = r.u;
      op.fbit = 0xFF;
      op.act = 0xFFFF;
      op.tbit = 0xFF;
      const int tl = loc[r.t];                    // local target position or -1
      const int cl = r.c >= 0 ? loc[r.c] : -1;    // local control position or -1
      const bool far_c = r.c >= 0 && cl < 0;
      if (far_c) op.fbit = static_cast<uint8_t>(r.c);
      if (r.cls != G_DIAG || r.is_h) {
        // non-diagonal: the target is local
        if (cl >= 0) op.act = kBitMask[cl];
        if (r.is_h) {
          op.code = static_cast<uint8_t>(OPC_H + tl);
          ++h_count;
          pass_cost += 0.5;
        } else if (r.cls == G_ANTI && u.m[1] == cd(1.0) && u.m[2] == cd(1.0)) {
          if (r.c < 0) op.code = static_cast<uint8_t>(OPC_X + tl);
          else if (far_c) op.code = static_cast<uint8_t>(OPC_XF + tl);
          else op.code = static_cast<uint8_t>(OPC_XL + 4 * tl + cl);
          pass_cost += 0.5;
        } else {  // dense, or anti-diagonal other than X (as a dense factor)
          op.code = static_cast<uint8_t>((r.c < 0 ? OPC_DENSE : OPC_CDENSE) + tl);
          for (int i = 0; i < 4; ++i) {
            op.m[i] = to_f2(u.m[i]);
            const cd hi(op.m[i].x, op.m[i].y);
            op.lo[i] = to_f2(u.m[i] - hi);
          }
          pass_cost += 3.0;
        }
      } else {
        op.m[0] = to_f2(u.m[0]);
        op.m[1] = to_f2(u.m[3]);
        op.m[2] = to_f2(u.m[3] / u.m[0]);
        op.d0one = (u.m[0] == cd(1.0)) ? 1 : 0;
        op.hc = (tl >= 0 && cl < 0) ? op.m[2] : op.m[1];
        pass_cost += 0.25;
        if (tl >= 0) {
          if (cl >= 0) {
            op.code = OPC_DLL;
            op.t = static_cast<uint8_t>(tl);
            op.c = static_cast<uint8_t>(cl);
          } else {
            op.code = static_cast<uint8_t>((far_c ? OPC_DLF : OPC_DLN) + tl);
          }
        } else {
          op.tbit = static_cast<uint8_t>(r.t);
          op.code = cl >= 0 ? static_cast<uint8_t>(OPC_DFL + cl) : static_cast<uint8_t>(OPC_DFF);
        }
      }
      P.ops.push_back(op);
    }
    ps.op_count = static_cast<uint32_t>(P.ops.size() - ps.op_begin);
    // exact power-of-two rescale for this pass's unscaled Hadamards
    const int tot = h_carry + h_count;
    ps.scale = std::ldexp(1.0f, -(tot / 2));
    h_carry = tot % 2;
    P.passes.push_back(ps);
    P.cost += pass_cost * static_cast<double>(1u << nint);
    raw.clear();
    h_in_pass = 0;
  };
  // An instruction is a barrier: the gates before it are scheduled (pending),
  // then it becomes a pass of its own, then scheduling resumes after it.
  std::vector<int>& order = order_tls;
  order.resize(gs.size());
  std::iota(order.begin(), order.end(), 0);
  pending.clear();
  size_t next = 0;
  auto take_segment = [&]() {
    pending.clear();
    while (next < order.size() && !is_instruction(gs[order[next]]->kind) && !is_wide(*gs[order[next]]))
      pending.push_back(order[next++]);
  };
  take_segment();
  for (;;) {
  while (!pending.empty()) {
    uint32_t Lmask = 0, blocked = 0;
    int nL = 0;
    for (int b = 0; b < 32; ++b) last_touch[b] = -1;
    still.clear();
    size_t idx = 0;
    for (; idx < pending.size(); ++idx) {
      if (blocked == all) break;
      const Gate& g = *gs[pending[idx]];
      const uint32_t qm = qmask[pending[idx]];
      if (qm & blocked) {  // an earlier gate on one of its qubits waits: so must it,
        blocked |= qm;     // and every later gate on any of its qubits
        still.push_back(pending[idx]);
        continue;
      }
      const GClass cls = gcls[pending[idx]];
      if (cls == G_SWAP) { std::swap(phys[g.q[0]], phys[g.q[1]]); continue; }
      const int tq = is_controlled(g.kind) ? g.q[1] : g.q[0];
      const int cq = is_controlled(g.kind) ? g.q[0] : -1;
      const int t = phys[tq];
      const int c = cq >= 0 ? phys[cq] : -1;
      if (cls != G_DIAG && !((Lmask >> t) & 1)) {
        if (nL == 4) { blocked |= qm; still.push_back(pending[idx]); continue; }
        Lmask |= 1u << t;
        ++nL;
      }
      push_raw(g, cls, t, c);
    }
    for (; idx < pending.size(); ++idx) still.push_back(pending[idx]);
    emit_pass(Lmask, nL, still.empty());
    pending.swap(still);
  }
  if (next >= order.size()) break;
  {
    const Gate& g = *gs[order[next++]];
    if (P.passes.empty()) emit_pass(0u, 0, false);  // the first pass generates the start state
    FusedPass ps{};
    if (is_wide(g)) {
      // custom k-qubit unitary: FP32 hi + lo coefficients, transposed
      const int k = g.nq, G = 1 << k;
      ps.L[0] = kWidePass;
      ps.L[1] = static_cast<uint8_t>(k);
      ps.op_begin = static_cast<uint32_t>(P.coef.size());
      uint32_t bits = 0, mask = 0;
      for (int t = 0; t < k; ++t) {
        bits |= static_cast<uint32_t>(phys[g.q[t]]) << (5 * t);
        mask |= 1u << phys[g.q[t]];
      }
      ps.op_count = bits;
      std::memcpy(&ps.scale, &mask, sizeof(mask));
      const size_t c0 = P.coef.size();
      P.coef.resize(c0 + 2 * size_t(G) * G);
      for (int r = 0; r < G; ++r)
        for (int c = 0; c < G; ++c) {
          const cd v = g.cm->m[size_t(r) * G + c];
          const float2 hi = to_f2(v);
          P.coef[c0 + size_t(c) * G + r] = hi;
          P.coef[c0 + size_t(G) * G + size_t(c) * G + r] = to_f2(v - cd(hi.x, hi.y));
        }
      P.cost += 8.0 * G * static_cast<double>(1u << nint);
    } else {
      ps.L[0] = kInstrPass;
      ps.L[1] = static_cast<uint8_t>(phys[g.q[0]]);
      ps.L[2] = g.kind == TQS_RESET ? 1 : 0;
      ps.op_begin = static_cast<uint32_t>(P.n_instr++);
      ps.op_count = 0;
      ps.scale = 1.0f;
      P.cost += 2.0 * static_cast<double>(1u << nint);
    }
    P.passes.push_back(ps);
  }
  take_segment();
  }
  if (P.passes.empty()) emit_pass(0u, 0, true);
  // Drop passes left with nothing to do (every factor fused to the identity).
  // The first pass kept generates the start state, so it must be a register
  // pass: an empty one stays in front of a leading instruction or custom
  // unitary, and one stays when nothing else is left.
  {
    auto normal = [](const FusedPass& ps) { return ps.L[0] != kInstrPass && ps.L[0] != kWidePass; };
    const FusedPass first = P.passes[0];
    size_t k = 0;
    for (size_t i = 0; i < P.passes.size(); ++i) {
      const FusedPass ps = P.passes[i];
      if (normal(ps) && ps.op_count == 0 && ps.scale == 1.0f) continue;
      if (k == 0 && !normal(ps)) P.passes[k++] = first;
      P.passes[k++] = ps;
    }
    if (k == 0) P.passes[k++] = first;
    P.passes.resize(k);
  }
  P.out_scale = h_carry ? static_cast<float>(1.0 / std::sqrt(2.0)) : 1.0f;
  P.identity = 1;
  for (int q = 0; q < 16; ++q) {
    P.pos[q] = static_cast<uint8_t>(q < n ? phys[q] : q);
    if (q < n && phys[q] != q) P.identity = 0;
  }
  P.cost += 2.0 * static_cast<double>(1u << n);
}

}  // namespace tqs
