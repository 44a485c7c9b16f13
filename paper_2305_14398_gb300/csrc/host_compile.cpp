// The fused-pass compiler (compile_program): a circuit's steps into passes of 4
// local qubit bits with their ops (declared, with its description, in
// host_common.h).
#include <deque>

#include "host_common.h"

namespace tqs {

namespace {

// The FP32 neighbour of a finite float x one ulp up (up) or down.
float fstep(float x, bool up) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  if ((b & 0x7fffffffu) == 0) b = up ? 1u : 0x80000001u;       // +-0: the smallest denormal
  else if ((b >> 31) == 0) b = up ? b + 1 : b - 1;             // positive
  else b = up ? b - 1 : b + 1;                                 // negative
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

// A unit-modulus phase z in FP32: of the four pairs that round z's parts
// down or up, the one whose squared modulus is nearest 1 (ties: nearest z).
// Every amplitude a phase multiplies shares its modulus error, so this error,
// unlike the rounding of the products, adds up over a circuit's phases in the
// norm; choosing the pair keeps it to about a quarter of plain rounding.
// Other values (not of modulus 1 to 1e-12) round to nearest.
float2 to_unit_f2(cd z) {
  // Circuits of a batch share most of their phases (the controlled phases of
  // a QFT, S, T, ...): a small direct-mapped cache per host thread, keyed by
  // the bits of z, answers repeats.
  struct Entry {
    uint64_t re = 0, im = 0;
    float2 r;
    bool used = false;
  };
  static thread_local Entry cache[1024];
  uint64_t kre, kim;
  const double zre = z.real(), zim = z.imag();
  // parts FP32 holds exactly (1, -1, i, 0.5, ...): nothing to choose
  if (static_cast<double>(static_cast<float>(zre)) == zre &&
      static_cast<double>(static_cast<float>(zim)) == zim)
    return make_float2(static_cast<float>(zre), static_cast<float>(zim));
  std::memcpy(&kre, &zre, 8);
  std::memcpy(&kim, &zim, 8);
  Entry& ent = cache[((kre * 0x9E3779B97F4A7C15ull) ^ (kim * 0xC2B2AE3D27D4EB4Full)) >> 54];
  if (ent.used && ent.re == kre && ent.im == kim) return ent.r;
  const float2 rn = to_f2(z);
  const double zr = z.real(), zi = z.imag();
  float2 best = rn;
  if (std::abs(zr * zr + zi * zi - 1.0) <= 2e-12) {
    // the FP32 values just below and just above each part (equal when exact)
    float xs[2] = {rn.x, rn.x}, ys[2] = {rn.y, rn.y};
    if (double(rn.x) < zr) xs[1] = fstep(rn.x, true);
    if (double(rn.x) > zr) xs[0] = fstep(rn.x, false);
    if (double(rn.y) < zi) ys[1] = fstep(rn.y, true);
    if (double(rn.y) > zi) ys[0] = fstep(rn.y, false);
    if (xs[0] != xs[1] || ys[0] != ys[1]) {
      // squared distances: the same order as the distances, without square roots
      auto dist2 = [&](float x, float y) { return (x - zr) * (x - zr) + (y - zi) * (y - zi); };
      double best_m = std::abs(double(rn.x) * rn.x + double(rn.y) * rn.y - 1.0);
      double best_d = dist2(rn.x, rn.y);
      for (int k = 0; k < 4; ++k) {
        const float x = xs[k & 1], y = ys[k >> 1];
        const double m = std::abs(double(x) * x + double(y) * y - 1.0);
        const double d = dist2(x, y);
        if (m < best_m || (m == best_m && d < best_d)) {
          best = make_float2(x, y);
          best_m = m;
          best_d = d;
        }
      }
    }
  }
  ent.re = kre;
  ent.im = kim;
  ent.r = best;
  ent.used = true;
  return best;
}

// One phase factor of a merged diagonal op: multiply the amplitudes with local
// position `tgt` set (tgt 4: the whole group) by v when the group's physical
// bit f is 1 (f 0xFF: always).
struct DiagEnt {
  int tgt;
  uint8_t f;
  float2 v;
};

// The phase factors of a diagonal op whose action is such a product (every
// diagonal op except a local-local one and a far target under a far
// control), or 0.  diag(d0, d1) = d0 diag(1, d1 / d0): with d0 exactly 1 one
// factor, else two.
int diag_entries(const FusedOp& op, DiagEnt* e) {
  const int code = op.code;
  const bool one = op.d0one != 0;
  const float2 d0 = op.m[0], d1 = op.m[1], r = op.m[2];
  if (code >= OPC_DLN && code < OPC_DLF) {  // local target, uncontrolled
    const int t = code - OPC_DLN;
    if (one) { e[0] = {t, 0xFF, r}; return 1; }
    e[0] = {4, 0xFF, d0};
    e[1] = {t, 0xFF, r};
    return 2;
  }
  if (code >= OPC_DLF && code < OPC_DFL) {  // local target, far control
    const int t = code - OPC_DLF;
    if (one) { e[0] = {t, op.fbit, r}; return 1; }
    e[0] = {4, op.fbit, d0};
    e[1] = {t, op.fbit, r};
    return 2;
  }
  if (code >= OPC_DFL && code < OPC_DFF) {  // far target, local control c
    const int c = code - OPC_DFL;
    if (one) { e[0] = {c, op.tbit, d1}; return 1; }
    e[0] = {c, 0xFF, d0};
    e[1] = {c, op.tbit, r};
    return 2;
  }
  if (code == OPC_DFF && op.fbit == 0xFF) {  // far target, uncontrolled
    if (one) { e[0] = {4, op.tbit, d1}; return 1; }
    e[0] = {4, 0xFF, d0};
    e[1] = {4, op.tbit, r};
    return 2;
  }
  return 0;
}

// u = diag(alpha, gamma) H diag(1, beta) with alpha, beta, gamma in
// {1, -1, i, -i}: true when u has that form (to 1e-14); d2 = diag(1, beta)
// acts first, then H, then d1.
bool hadamard_split(const Mat2& u, Mat2& d2, Mat2& d1) {
  const double s = 1.0 / std::sqrt(2.0);
  for (int i = 0; i < 4; ++i)  // |u_i|^2 = 1/2
    if (std::abs(std::norm(u.m[i]) - 0.5) > 2e-14) return false;
  // only phases that FP32 holds exactly (1, -1, i, -i): multiplying by them
  // is exact, so the split keeps the amplitudes' norm as the dense form does
  auto snap = [](cd z, cd& out) {
    const double re = std::round(z.real()), im = std::round(z.imag());
    if (std::abs(z - cd(re, im)) > 1e-14 || std::abs(re) + std::abs(im) != 1.0) return false;
    out = cd(re, im);
    return true;
  };
  cd alpha, gamma, beta;
  if (!snap(u.m[0] / s, alpha) || !snap(u.m[2] / s, gamma) || !snap(u.m[1] / u.m[0], beta)) return false;
  if (std::abs(s * alpha * beta - u.m[1]) > 1e-14 || std::abs(-s * gamma * beta - u.m[3]) > 1e-14)
    return false;
  d2 = {{1.0, 0.0, 0.0, beta}};
  d1 = {{alpha, 0.0, 0.0, gamma}};
  return true;
}

bool is_identity2(const Mat2& u) {
  return std::norm(u.m[0] - 1.0) <= 1e-30 && std::norm(u.m[3] - 1.0) <= 1e-30 &&
         std::norm(u.m[1]) <= 1e-30 && std::norm(u.m[2]) <= 1e-30;
}

// True when z is 1, -1, i or -i (to 1e-14): FP32 holds it exactly and a
// multiply by it is exact.
bool exact_phase(cd z) {
  const double re = std::round(z.real()), im = std::round(z.imag());
  return std::abs(z - cd(re, im)) <= 1e-14 && std::abs(re) + std::abs(im) == 1.0;
}

// Relative cost of an uncontrolled single-qubit factor as the kernel runs it
// (unit: one unscaled Hadamard or exchange; exact phases accumulate per bit
// and cost half; a dense butterfly with FP32 hi + lo coefficients several).
// A phase that FP32 does not hold exactly counts as much as a dense
// butterfly: as a factor of its own it multiplies the amplitudes by a
// coefficient whose modulus is off 1 by up to an FP32 ulp, and over many
// such factors that adds up in the norm, while fused into a neighbouring
// non-diagonal factor it rides on the hi + lo coefficients.
double single_cost(const Mat2& u, bool is_h) {
  if (is_h) return 1.0;
  if (is_identity2(u)) return 0.0;
  switch (classify_mat(u)) {
    case G_DIAG: return exact_phase(u.m[0]) && exact_phase(u.m[3]) ? 0.5 : 3.5;
    case G_ANTI:
      if (u.m[1] == cd(1.0) && u.m[2] == cd(1.0)) return 1.0;
      return exact_phase(u.m[1]) && exact_phase(u.m[2]) ? 1.5 : 3.5;
    default: {
      Mat2 d1, d2;
      return hadamard_split(u, d2, d1) ? 1.5 : 3.5;
    }
  }
}

// Local target position of a non-diagonal op.
int nondiag_target(int code) {
  if (code >= OPC_XL && code < OPC_ANTI) return (code - OPC_XL) >> 2;
  return code & 3;
}

// Merge the pass's phase factors (ops [begin, end)) into OPC_DLIST ops of up
// to 8 factors per target.  The kernel only accumulates such factors (per
// local position, or for the group) and multiplies them in before the next
// non-diagonal op on that position or at the end of the pass, so factors on
// one position between two non-diagonal ops on it commute with everything in
// between: each list is emitted just before the next non-diagonal op on its
// position (or at the end of the pass).
constexpr size_t kMaxCachedRun = 12;  // longest run of local phases whose product is cached

void merge_diagonals(std::vector<FusedOp>& ops, size_t begin) {
  {
    // nothing to merge: no phase factor and no two local-local factors in a row
    bool any = false;
    for (size_t i = begin; i < ops.size() && !any; ++i) {
      DiagEnt es[2];
      any = diag_entries(ops[i], es) > 0 ||
            (ops[i].code == OPC_DLL && i + 1 < ops.size() && ops[i + 1].code == OPC_DLL);
    }
    if (!any) return;
  }
  static thread_local std::vector<FusedOp> out;
  out.clear();
  DiagEnt open[5][8];
  int nopen[5] = {0, 0, 0, 0, 0};
  auto flush = [&](int t) {
    if (nopen[t] == 0) return;
    if (nopen[t] == 1 && (t < 4 || open[t][0].f != 0xFF)) {
      // one factor: the single diagonal op with d0 exactly 1 that does the
      // same (header only, no factor list to load)
      const DiagEnt& e = open[t][0];
      FusedOp op{};
      op.d0one = 1;
      op.act = 0xFFFF;
      op.tbit = 0xFF;
      op.fbit = 0xFF;
      op.m[0] = make_float2(1.f, 0.f);
      op.m[1] = e.v;
      op.m[2] = e.v;
      op.hc = e.v;
      if (t == 4) {
        op.code = OPC_DFF;
        op.tbit = e.f;
      } else if (e.f == 0xFF) {
        op.code = static_cast<uint8_t>(OPC_DLN + t);
      } else {
        op.code = static_cast<uint8_t>(OPC_DLF + t);
        op.fbit = e.f;
      }
      out.push_back(op);
      nopen[t] = 0;
      return;
    }
    FusedOp op{};
    op.code = OPC_DLIST;
    op.t = static_cast<uint8_t>(t);
    op.c = static_cast<uint8_t>(nopen[t]);
    op.tbit = 0xFF;
    op.fbit = 0xFF;
    op.act = 0xFFFF;
    uint8_t fb[8];
    float2 v[8];
    for (int k = 0; k < 8; ++k) {
      fb[k] = k < nopen[t] ? open[t][k].f : 0xFF;
      v[k] = k < nopen[t] ? open[t][k].v : make_float2(1.f, 0.f);
    }
    std::memcpy(&op.hc, fb, 8);
    for (int k = 0; k < 4; ++k) {
      op.m[k] = v[k];
      op.lo[k] = v[4 + k];
    }
    out.push_back(op);
    nopen[t] = 0;
  };
  for (size_t i = begin; i < ops.size(); ++i) {
    const FusedOp& op = ops[i];
    DiagEnt es[2];
    const int ne = diag_entries(op, es);
    if (ne > 0) {
      for (int k = 0; k < ne; ++k) {
        if (nopen[es[k].tgt] == 8) flush(es[k].tgt);
        open[es[k].tgt][nopen[es[k].tgt]++] = es[k];
      }
      continue;
    }
    if (op.code < OPC_DLN) flush(nondiag_target(op.code));
    out.push_back(op);
  }
  // At the end of the pass: lists of two or more targets over the same factor
  // bits (the far-controlled phases of a QFT pass) run as one OPC_DLISTM op,
  // which tests the bits once; the rest flush one by one.
  {
    bool done[5] = {false, false, false, false, false};
    for (int t = 0; t < 5; ++t) {
      if (done[t] || nopen[t] < 2) continue;
      auto sorted_bits = [&](int u, uint8_t* fb, float2* v) {
        // the list's entries in order of their bits (stable)
        int idx[8];
        for (int k = 0; k < nopen[u]; ++k) idx[k] = k;
        std::stable_sort(idx, idx + nopen[u], [&](int x, int y) { return open[u][x].f < open[u][y].f; });
        for (int k = 0; k < 8; ++k) {
          fb[k] = k < nopen[u] ? open[u][idx[k]].f : 0xFF;
          v[k] = k < nopen[u] ? open[u][idx[k]].v : make_float2(1.f, 0.f);
        }
      };
      uint8_t fb_t[8];
      float2 v_t[5][8];
      sorted_bits(t, fb_t, v_t[t]);
      unsigned mask = 1u << t;
      for (int u = t + 1; u < 5; ++u) {
        if (done[u] || nopen[u] != nopen[t]) continue;
        uint8_t fb_u[8];
        sorted_bits(u, fb_u, v_t[u]);
        if (std::memcmp(fb_u, fb_t, 8) == 0) mask |= 1u << u;
      }
      if ((mask & (mask - 1)) == 0) continue;  // no other target with the same bits
      bool first = true;
      for (int u = 0; u < 5; ++u) {
        if (!((mask >> u) & 1)) continue;
        FusedOp op{};
        op.code = first ? OPC_DLISTM : OPC_NOP;
        op.t = static_cast<uint8_t>(first ? mask : 0);
        op.c = static_cast<uint8_t>(first ? nopen[t] : 0);
        op.tbit = 0xFF;
        op.fbit = 0xFF;
        op.act = 0xFFFF;
        if (first) std::memcpy(&op.hc, fb_t, 8);
        for (int k = 0; k < 4; ++k) {
          op.m[k] = v_t[u][k];
          op.lo[k] = v_t[u][4 + k];
        }
        out.push_back(op);
        first = false;
        done[u] = true;
        nopen[u] = 0;
      }
    }
  }
  for (int t = 0; t < 5; ++t) flush(t);
  // Runs of two or more local-local diagonal factors (OPC_DLL) become one
  // 16-entry diagonal: entry j is the product, in FP64 of the factors' FP32
  // values, of the run's factors at local index j, rounded once (they
  // commute, so the run's order does not matter).
  ops.resize(begin);
  for (size_t i = 0; i < out.size();) {
    size_t j = i;
    while (j < out.size() && out[j].code == OPC_DLL) ++j;
    if (j - i < 2) {
      ops.push_back(out[i]);
      ++i;
      continue;
    }
    // The same runs recur across the circuits of a batch (every QFT of one
    // size has the same ones): a small direct-mapped cache per host thread,
    // keyed by the run's factors (positions and FP32 values), holds the two
    // records of the result.
    struct RunEntry {
      uint32_t key[kMaxCachedRun * 5];
      size_t len = 0;
      FusedOp a, b;
    };
    static thread_local RunEntry run_cache[64];
    const size_t len = j - i;
    uint32_t key[kMaxCachedRun * 5];
    uint64_t h = 0x9E3779B97F4A7C15ull;
    if (len <= kMaxCachedRun) {
      for (size_t k = 0; k < len; ++k) {
        const FusedOp& op = out[i + k];
        uint32_t* w = key + 5 * k;
        w[0] = static_cast<uint32_t>(op.t) | (static_cast<uint32_t>(op.c) << 8);
        std::memcpy(w + 1, &op.m[0], 8);
        std::memcpy(w + 3, &op.m[1], 8);
        for (int x = 0; x < 5; ++x) h = (h ^ w[x]) * 0x100000001B3ull;
      }
      RunEntry& ce = run_cache[h >> 58];
      if (ce.len == len && std::memcmp(ce.key, key, len * 5 * sizeof(uint32_t)) == 0) {
        ops.push_back(ce.a);
        ops.push_back(ce.b);
        i = j;
        continue;
      }
    }
    cd d[16];
    for (int e = 0; e < 16; ++e) d[e] = 1.0;
    for (size_t k = i; k < j; ++k) {
      const FusedOp& op = out[k];
      const cd d0(op.m[0].x, op.m[0].y), d1(op.m[1].x, op.m[1].y);
      for (int e = 0; e < 16; ++e)
        if ((e >> op.c) & 1) d[e] *= ((e >> op.t) & 1) ? d1 : d0;
    }
    FusedOp a{}, b{};
    a.code = OPC_DIAG16;
    b.code = OPC_NOP;
    for (FusedOp* r : {&a, &b}) {
      r->fbit = 0xFF;
      r->tbit = 0xFF;
      r->act = 0xFFFF;
    }
    for (int e = 0; e < 4; ++e) {
      a.m[e] = to_unit_f2(d[e]);
      a.lo[e] = to_unit_f2(d[4 + e]);
      b.m[e] = to_unit_f2(d[8 + e]);
      b.lo[e] = to_unit_f2(d[12 + e]);
    }
    if (len <= kMaxCachedRun) {
      RunEntry& ce = run_cache[h >> 58];
      std::memcpy(ce.key, key, len * 5 * sizeof(uint32_t));
      ce.len = len;
      ce.a = a;
      ce.b = b;
    }
    ops.push_back(a);
    ops.push_back(b);
    i = j;
  }
}

// `act` of a factor with local control position c: the local indices with bit c set.
constexpr uint16_t kLocalControlMask[4] = {0xAAAA, 0xCCCC, 0xF0F0, 0xFF00};

// Local positions (bits 0..3) that an op reads or changes: its target, its
// local control, the positions its phases depend on.
unsigned touched_positions(const FusedOp& op) {
  const int code = op.code;
  if (code < OPC_XL) return 1u << (code & 3);                   // H, X, XF
  if (code < OPC_HMASK) return (1u << ((code - OPC_XL) >> 2)) | (1u << ((code - OPC_XL) & 3));
  if (code == OPC_HMASK) return op.t & 15u;
  if (code == OPC_XP) return (1u << (op.t & 3)) | (op.c & 15u);
  if (code < OPC_CDENSE) return 1u << (code & 3);               // DENSE
  if (code < OPC_DLN) {                                         // CDENSE
    unsigned m = 1u << (code & 3);
    for (int c = 0; c < 4; ++c)
      if (op.act == kLocalControlMask[c]) m |= 1u << c;
    return m;
  }
  if (code < OPC_DFF) return 1u << (code & 3);                  // DLN, DLF, DFL
  if (code == OPC_DFF) return 0u;
  if (code == OPC_DLL) return (1u << op.t) | (1u << op.c);
  if (code == OPC_DLIST) return op.t < 4 ? 1u << op.t : 0u;
  if (code == OPC_DLISTM) return op.t & 15u;
  if (code == OPC_NOP) return 0u;  // a continuation record of the op before it
  return 15u;                                                   // DIAG16, NOP
}

// Uncontrolled Hadamards of a pass (ops [begin, end)) move later past ops on
// other positions (they commute: different tensor factors) until an op on
// their position or another Hadamard comes; Hadamards that meet run as one
// OPC_HMASK op (one dispatch instead of several).
// An exchange op (X, CNOT) on one local position as (target, local control
// positions, active local indices, far control mask); false for other ops.
bool exchange_parts(const FusedOp& op, int& t, unsigned& cmask, unsigned& act, uint32_t& far) {
  const int code = op.code;
  if (code >= OPC_X && code < OPC_XF) {  // uncontrolled
    t = code & 3, cmask = 0, act = 0xFFFF, far = 0;
  } else if (code >= OPC_XF && code < OPC_XL) {  // far control
    if (op.fbit >= 32) return false;  // the far mask covers bits 0..31
    t = code & 3, cmask = 0, act = 0, far = 1u << op.fbit;  // on iff the far bit is 1
  } else if (code >= OPC_XL && code < OPC_HMASK) {  // local control
    const int c = (code - OPC_XL) & 3;
    t = (code - OPC_XL) >> 2, cmask = 1u << c, act = kLocalControlMask[c], far = 0;
  } else if (code == OPC_XP) {
    uint32_t f;
    std::memcpy(&f, &op.hc, 4);
    t = op.t, cmask = op.c, act = op.act, far = f;
  } else {
    return false;
  }
  return true;
}

// Adjacent exchange ops on one local target (a fan of CNOTs into one qubit,
// as in the Deutsch-Jozsa oracle) commute and compose: the pair swaps when an
// odd number of them is active, so the run becomes one OPC_XP op whose active
// set is the parity of the factors' (XOR of their masks) (one dispatch).
void merge_exchanges(std::vector<FusedOp>& ops, size_t begin) {
  {
    // nothing to merge without two adjacent exchanges on one target
    bool pair = false;
    int t0 = -1;
    for (size_t i = begin; i < ops.size() && !pair; ++i) {
      int t;
      unsigned cm, act;
      uint32_t far;
      const bool ex = exchange_parts(ops[i], t, cm, act, far);
      pair = ex && t == t0;
      t0 = ex ? t : -1;
    }
    if (!pair) return;
  }
  static thread_local std::vector<FusedOp> out;
  out.clear();
  bool any = false;
  for (size_t i = begin; i < ops.size();) {
    int t0;
    unsigned cm0, act0;
    uint32_t far0;
    if (!exchange_parts(ops[i], t0, cm0, act0, far0)) {
      out.push_back(ops[i++]);
      continue;
    }
    size_t j = i + 1;
    for (; j < ops.size(); ++j) {
      int t;
      unsigned cm, act;
      uint32_t far;
      if (!exchange_parts(ops[j], t, cm, act, far) || t != t0) break;
      cm0 |= cm;
      act0 ^= act;
      far0 ^= far;
    }
    if (j == i + 1) {
      out.push_back(ops[i++]);
      continue;
    }
    any = true;
    i = j;
    if (act0 == 0 && far0 == 0) continue;  // an even number of every factor: the identity
    FusedOp x{};
    x.tbit = 0xFF;
    x.fbit = 0xFF;
    if (act0 == 0xFFFF && far0 == 0) {
      x.code = static_cast<uint8_t>(OPC_X + t0);
      x.act = 0xFFFF;
    } else {
      x.code = OPC_XP;
      x.t = static_cast<uint8_t>(t0);
      x.c = static_cast<uint8_t>(cm0);
      x.act = static_cast<uint16_t>(act0);
      std::memcpy(&x.hc, &far0, 4);
    }
    out.push_back(x);
  }
  if (!any) return;
  ops.resize(begin);
  ops.insert(ops.end(), out.begin(), out.end());
}

void group_hadamards(std::vector<FusedOp>& ops, size_t begin) {
  size_t nh = 0;
  for (size_t i = begin; i < ops.size(); ++i) nh += ops[i].code < OPC_X;
  if (nh < 2) return;
  static thread_local std::vector<FusedOp> out;
  out.clear();
  unsigned pend = 0;  // positions with a Hadamard held back
  auto flush = [&]() {
    if (pend == 0) return;
    FusedOp h{};
    h.fbit = 0xFF;
    h.tbit = 0xFF;
    h.act = 0xFFFF;
    if ((pend & (pend - 1)) == 0) {
      h.code = static_cast<uint8_t>(OPC_H + __builtin_ctz(pend));
    } else {
      h.code = OPC_HMASK;
      h.t = static_cast<uint8_t>(pend);
    }
    out.push_back(h);
    pend = 0;
  };
  for (size_t i = begin; i < ops.size(); ++i) {
    const FusedOp& op = ops[i];
    if (op.code < OPC_X) {
      const unsigned b = 1u << (op.code & 3);
      if (pend & b) flush();  // two on one position: keep their order
      pend |= b;
      continue;
    }
    if (touched_positions(op) & pend) flush();
    out.push_back(op);
  }
  flush();
  ops.resize(begin);
  ops.insert(ops.end(), out.begin(), out.end());
}

}  // namespace

void compile_program(int n, const std::vector<const Gate*>& gs_in, Program& P,
                      bool fold_x, bool absorb) {
  P.n = n;
  P.nint = std::max(n, 4);
  // scratch reused across calls on this thread (no allocation per circuit)
  static thread_local std::vector<const Gate*> gs_tls;
  static thread_local std::vector<int> pending_tls, still_tls, order_tls;
  static thread_local std::vector<CompileRaw> raw_tls;
  static thread_local std::vector<uint32_t> qmask_tls;  // per entry of gs: its qubit mask
  static thread_local std::vector<GClass> cls_tls;      // per entry of gs: its class
  std::vector<const Gate*>& gs = gs_tls;
  gs.clear();
  P.gen_index = 0;
  gs.assign(gs_in.begin(), gs_in.end());
  // Trailing permutation gates: an X, CNOT or SWAP with no later gate of
  // another kind on its qubits only permutes the final amplitudes, psi(y) =
  // phi(F(y)) with F an affine map over GF(2) (X: y ^ e_q; CNOT(c, t):
  // y ^ y_c e_t; SWAP: exchange two bits; each its own inverse).  Such gates
  // are taken out of the program and F goes into the output map.  Gates of
  // one step act on disjoint qubits, so the scan in step order is the
  // circuit's own order up to commuting gates.
  static thread_local std::vector<const Gate*> tail_tls;
  std::vector<const Gate*>& tail = tail_tls;
  tail.clear();
  if (absorb) {
    static thread_local std::vector<char> take_tls;
    std::vector<char>& take = take_tls;
    // scan from the end; once every qubit has a later gate that stays, no
    // earlier gate can join the tail, so the scan stops there (at `from`)
    const uint32_t all_q = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);
    uint32_t blocked = 0;  // qubits with a later gate that stays in the program
    size_t from = gs.size();
    take.assign(gs.size(), 0);
    while (from > 0 && blocked != all_q) {
      const Gate& g = *gs[--from];
      const uint32_t qm = qubit_mask(g);
      const bool perm = g.kind == TQS_X || g.kind == TQS_CNOT || g.kind == TQS_SWAP;
      if (perm && !(qm & blocked)) take[from] = 1;
      else blocked |= qm;
    }
    size_t k = from;
    for (size_t i = from; i < gs.size(); ++i) {
      if (take[i]) tail.push_back(gs[i]);
      else gs[k++] = gs[i];
    }
    gs.resize(k);
  }
  // Leading uncontrolled X factors on a qubit that nothing has touched yet act
  // on the basis input |0...0> only by flipping that qubit: fold them into the
  // start index instead of spending butterflies (input |0...0> only; before
  // the fusion below could merge them into later gates).
  {
    static thread_local std::vector<const Gate*> xf_tls;
    std::vector<const Gate*>& xf = xf_tls;
    xf.clear();
    uint32_t touched = 0;
    for (const Gate* g : gs) {
      if (fold_x && g->kind == TQS_X && !((touched >> g->q[0]) & 1)) {
        P.gen_index ^= 1 << g->q[0];
        continue;
      }
      touched |= qubit_mask(*g);
      xf.push_back(g);
    }
    gs.swap(xf);
  }
  // Circuit-wide fusion of single-qubit factors: consecutive uncontrolled
  // single-qubit gates on one qubit (no other gate on it in between; the
  // gates in between act on other qubits and commute) multiply into one
  // factor at the first one's place, by the mixed-product property of the
  // Kronecker product, unless the product runs costlier than the two apart.
  // Products equal to the identity (H H, X X, ...) disappear; an exact X
  // product is an X gate (an exchange).
  static thread_local std::deque<Gate> fused_tls;
  static thread_local std::vector<const Gate*> fl_tls;
  std::deque<Gate>& fused = fused_tls;
  std::vector<const Gate*>& fl = fl_tls;
  fused.clear();
  fl.clear();
  {
    int open[32];
    for (int q = 0; q < 32; ++q) open[q] = -1;
    for (const Gate* g : gs) {
      const bool single = g->nq == 1 && !is_instruction(g->kind) && !is_two_qubit(g->kind);
      if (!single) {
        fl.push_back(g);
        for (uint32_t m = qubit_mask(*g); m; m &= m - 1) open[__builtin_ctz(m)] = -1;
        continue;
      }
      const int q = g->q[0];
      if (open[q] >= 0) {
        const Gate* pg = fl[static_cast<size_t>(open[q])];
        const Mat2 uf = mat_mul(g->u, pg->u);
        if (single_cost(uf, false) <=
            single_cost(pg->u, pg->kind == TQS_H) + single_cost(g->u, g->kind == TQS_H)) {
          if (is_identity2(uf)) {
            fl[static_cast<size_t>(open[q])] = nullptr;
            open[q] = -1;
            continue;
          }
          fused.push_back(*pg);
          Gate& f = fused.back();
          f.u = uf;
          f.cm.reset();
          const bool is_x = uf.m[0] == cd(0.0) && uf.m[3] == cd(0.0) && uf.m[1] == cd(1.0) && uf.m[2] == cd(1.0);
          f.kind = is_x ? TQS_X : TQS_U3;
          fl[static_cast<size_t>(open[q])] = &f;
          continue;
        }
      }
      fl.push_back(g);
      open[q] = static_cast<int>(fl.size()) - 1;
    }
  }
  gs.clear();
  for (const Gate* g : fl)
    if (g != nullptr) gs.push_back(g);

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
        // consecutive factors on one qubit multiply (the mixed-product
        // property), unless the product is costlier than the two apart
        // (a Hadamard and a general phase: a dense butterfly)
        Raw& r = raw[last];
        const Mat2 uf = mat_mul(g.u, r.u);
        if (single_cost(uf, false) <= single_cost(r.u, r.is_h) + single_cost(g.u, g.kind == TQS_H)) {
          if (r.is_h) --h_in_pass;
          r.u = uf;
          r.is_h = false;
          r.cls = classify_mat(r.u);
          return;
        }
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
    auto emit_raw = [&](const Raw& r) {
      // a factor that fused to the identity (H H, X X, ...) does nothing
      if (!r.is_h && is_identity2(r.u)) return;
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
        if (cl >= 0) op.act = kLocalControlMask[cl];
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
        if (u.m[0] == cd(1.0)) {  // a phase gate: d1 and d1 / d0 are the same value
          op.m[0] = make_float2(1.f, 0.f);
          op.m[1] = op.m[2] = to_unit_f2(u.m[3]);
        } else {
          op.m[0] = to_unit_f2(u.m[0]);
          op.m[1] = to_unit_f2(u.m[3]);
          op.m[2] = to_unit_f2(u.m[3] / u.m[0]);
        }
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
    };
    for (const Raw& r : raw) {
      // An uncontrolled factor diag(alpha, gamma) H diag(1, beta) with phases
      // in {1, -1, i, -i} (X H, H X, Z H, H Z, Y H, ...) runs as an exact
      // unscaled Hadamard between exact phase factors instead of a dense
      // butterfly.
      Mat2 d1, d2;
      if (r.single && !r.is_h && r.cls != G_DIAG && h_count < kMaxHPerPass &&
          hadamard_split(r.u, d2, d1)) {
        emit_raw({d2, G_DIAG, false, true, r.t, -1});
        emit_raw({gate_matrix(TQS_H, nullptr), G_DENSE, true, true, r.t, -1});
        emit_raw({d1, G_DIAG, false, true, r.t, -1});
        continue;
      }
      // An uncontrolled anti-diagonal factor [[0, b], [c, 0]] other than X
      // with exact phases (Y, X Z, ...) is X diag(c, b): phases, then an
      // exchange.
      if (r.single && !r.is_h && r.cls == G_ANTI && !(r.u.m[1] == cd(1.0) && r.u.m[2] == cd(1.0)) &&
          exact_phase(r.u.m[1]) && exact_phase(r.u.m[2])) {
        emit_raw({Mat2{{r.u.m[2], 0.0, 0.0, r.u.m[1]}}, G_DIAG, false, true, r.t, -1});
        emit_raw({gate_matrix(TQS_X, nullptr), G_ANTI, false, true, r.t, -1});
        continue;
      }
      emit_raw(r);
    }
    merge_diagonals(P.ops, ps.op_begin);
    group_hadamards(P.ops, ps.op_begin);
    merge_exchanges(P.ops, ps.op_begin);
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
  // A register pass last multiplies every amplitude by its scale 2^-k (an
  // exact power of two).  The leftover 2^-1/2 is folded into that scale, so
  // the output phase multiplies by nothing (where the pass applies no phase
  // scalar the result is bitwise that of a separate multiply by 2^-1/2).
  if (P.out_scale != 1.0f && P.passes.back().L[0] != kInstrPass && P.passes.back().L[0] != kWidePass) {
    P.passes.back().scale *= P.out_scale;
    P.out_scale = 1.0f;
  }
  // Output map: F (the folded tail, columns over logical bits, offset v)
  // composed with the relabeling phys.  F(y) = g_1(g_2(... g_k(y))) for the
  // tail g_1 .. g_k: built by F <- F o g for g in order.
  uint32_t fcol[32];
  uint32_t fv = 0;
  for (int q = 0; q < 32; ++q) fcol[q] = 1u << q;
  for (const Gate* g : tail) {
    if (g->kind == TQS_X) {
      fv ^= fcol[g->q[0]];
    } else if (g->kind == TQS_CNOT) {
      fcol[g->q[0]] ^= fcol[g->q[1]];
    } else {
      std::swap(fcol[g->q[0]], fcol[g->q[1]]);
    }
  }
  auto relabel = [&](uint32_t v) {
    uint32_t r = 0;
    for (; v != 0; v &= v - 1) r |= 1u << phys[__builtin_ctz(v)];
    return r;
  };
  for (int q = 0; q < 16; ++q)
    P.col[q] = static_cast<uint16_t>(q < n ? relabel(fcol[q]) : (1u << q));
  P.col_off = static_cast<uint16_t>(relabel(fv));
  P.cost += 2.0 * static_cast<double>(1u << n);
}

}  // namespace tqs
