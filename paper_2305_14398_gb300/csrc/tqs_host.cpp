// Host side of the C ABI (include/tqs.h): gate data, the circuit model and its
// step packing, the fused-pass compiler, batches, and the entry points.
//
// Sec. 5.2: the circuit model records operations and creates steps as they
// are added; the data provider supplies each operation's matrix separately
// from the circuit structure.  Sec. 5.3: stages 1-3 (steps, operations per
// step, operation data) run here; stages 4-6 run in the kernels.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <new>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tqs.h"
#include "tqs_internal.h"

namespace tqs {

// ---------------------------------------------------------------- errors

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_last_error(const char* msg) { g_last_error = msg; }

static tqs_status fail(tqs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

static tqs_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? TQS_ERR_NOMEM : TQS_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define TQS_CUDA(call, what)                      \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Device allocator of the library's scratch: cudaMalloc / cudaFree, or the
// caller's callbacks (tqs_set_allocator).  Every buffer remembers the
// allocator that made it and is returned to that one.
struct Allocator {
  tqs_alloc_fn alloc = nullptr;  // nullptr: cudaMalloc / cudaFree
  tqs_free_fn free = nullptr;
  void* ctx = nullptr;
};
static std::mutex g_alloc_mu;
static Allocator g_alloc;

static Allocator current_allocator() {
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  return g_alloc;
}

// Allocate `bytes` of device memory for use on `s` with allocator A.
static cudaError_t dev_alloc(const Allocator& A, void** p, size_t bytes, cudaStream_t s) {
  if (!A.alloc) return cudaMalloc(p, bytes);
  *p = A.alloc(bytes, s, A.ctx);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

// Return p to allocator A.  With s = nullptr the device is synchronised
// first (as cudaFree does), so no queued work still reads the buffer when the
// caller's allocator hands it out again; with a stream, frees are
// stream-ordered on it.
static void dev_free(const Allocator& A, void* p, cudaStream_t s) {
  if (!p) return;
  if (!A.alloc) {
    cudaFree(p);
    return;
  }
  if (!s) cudaDeviceSynchronize();
  A.free(p, s, A.ctx);
}

// A device buffer owned by a handle.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  Allocator by;  // the allocator that made p
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) dev_free(by, p, nullptr);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t n) {
    if (n <= bytes && p) return cudaSuccess;
    release();
    by = current_allocator();
    cudaError_t e = dev_alloc(by, &p, n ? n : 16, nullptr);
    if (e == cudaSuccess) bytes = n;
    else p = nullptr;
    return e;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------ gate data
// Table 1 (Sec. 2.3), S and T (Sec. 5.2), textbook rotations, eq. 7 / eq. 8.

using cd = std::complex<double>;

struct Mat2 {
  cd m[4];  // [[m0, m1], [m2, m3]]
};

static bool is_controlled(int g) { return g == TQS_CNOT || g == TQS_CZ || g == TQS_CP || g == TQS_CU; }
static bool is_instruction(int g) { return g == TQS_MEASURE || g == TQS_RESET; }
static bool is_two_qubit(int g) { return is_controlled(g) || g == TQS_SWAP; }
static int n_params(int g) {
  switch (g) {
    case TQS_R: case TQS_RX: case TQS_RY: case TQS_RZ: case TQS_CP: return 1;
    case TQS_U3: return 3;
    case TQS_CU: return 8;
    default: return 0;
  }
}

// Single-qubit matrix of a gate, or the U of a controlled gate.
static Mat2 gate_matrix(int g, const double* p) {
  const double r2 = 1.0 / std::sqrt(2.0);
  const cd I(0.0, 1.0);
  Mat2 u;
  switch (g) {
    case TQS_H: u = {{r2, r2, r2, -r2}}; break;
    case TQS_X: case TQS_CNOT: u = {{0.0, 1.0, 1.0, 0.0}}; break;
    case TQS_Y: u = {{0.0, -I, I, 0.0}}; break;
    case TQS_Z: case TQS_CZ: u = {{1.0, 0.0, 0.0, -1.0}}; break;
    case TQS_S: u = {{1.0, 0.0, 0.0, I}}; break;
    case TQS_T: u = {{1.0, 0.0, 0.0, std::polar(1.0, M_PI / 4.0)}}; break;
    case TQS_R: case TQS_CP: u = {{1.0, 0.0, 0.0, std::polar(1.0, p[0])}}; break;
    case TQS_RX: {
      const double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      u = {{c, -I * s, -I * s, c}};
      break;
    }
    case TQS_RY: {
      const double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      u = {{c, -s, s, c}};
      break;
    }
    case TQS_RZ: u = {{std::polar(1.0, -p[0] / 2), 0.0, 0.0, std::polar(1.0, p[0] / 2)}}; break;
    case TQS_U3: {
      const double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      u = {{c, -std::polar(1.0, p[2]) * s, std::polar(1.0, p[1]) * s,
            std::polar(1.0, p[1] + p[2]) * c}};
      break;
    }
    case TQS_CU: u = {{cd(p[0], p[1]), cd(p[2], p[3]), cd(p[4], p[5]), cd(p[6], p[7])}}; break;
    default: u = {{1.0, 0.0, 0.0, 1.0}}; break;
  }
  return u;
}

static bool is_unitary(const Mat2& u, double tol) {
  const cd a = u.m[0], b = u.m[1], c = u.m[2], d = u.m[3];
  // U^dagger U
  const cd e00 = std::conj(a) * a + std::conj(c) * c;
  const cd e01 = std::conj(a) * b + std::conj(c) * d;
  const cd e11 = std::conj(b) * b + std::conj(d) * d;
  return std::abs(e00 - 1.0) <= tol && std::abs(e11 - 1.0) <= tol && std::abs(e01) <= tol;
}

// A registered custom unitary (Sec. 5.2: custom unitary data is registered
// with the operation data provider, then applied to qubits).
struct CustomMat {
  int k = 0;              // qubits
  std::vector<cd> m;      // 2^k x 2^k, row-major; local index bit t = qubit t of the gate
};

// Internal kind of a custom unitary (outside the tqs_gate range).
constexpr int kCustomKind = 64;

// One recorded operation.
struct Gate {
  int kind;
  int q[kMaxCustomQubits];  // qubits (controlled: {control, target}; custom: local bit order)
  int nq;
  double p[8];
  Mat2 u;     // single-qubit matrix, the controlled U, or a 1-qubit custom matrix
  int step;   // step index (ASAP)
  std::shared_ptr<const CustomMat> cm;  // custom unitaries with k >= 2
};

static bool is_wide(const Gate& g) { return g.kind == kCustomKind && g.nq >= 2; }
static uint32_t qubit_mask(const Gate& g) {
  uint32_t m = 0;
  for (int i = 0; i < g.nq; ++i) m |= 1u << g.q[i];
  return m;
}

static inline float2 to_f2(cd z) {
  return make_float2(static_cast<float>(z.real()), static_cast<float>(z.imag()));
}

// ---------------------------------------------------------- fused compile

enum GClass { G_DENSE, G_ANTI, G_DIAG, G_SWAP };

static GClass classify_mat(const Mat2& u) {
  if (u.m[1] == cd(0.0) && u.m[2] == cd(0.0)) return G_DIAG;
  if (u.m[0] == cd(0.0) && u.m[3] == cd(0.0)) return G_ANTI;
  return G_DENSE;
}

static GClass classify(const Gate& g) {
  if (g.kind == TQS_SWAP) return G_SWAP;
  return classify_mat(g.u);
}

// a * b (apply b, then a)
static Mat2 mat_mul(const Mat2& a, const Mat2& b) {
  Mat2 r;
  r.m[0] = a.m[0] * b.m[0] + a.m[1] * b.m[2];
  r.m[1] = a.m[0] * b.m[1] + a.m[1] * b.m[3];
  r.m[2] = a.m[2] * b.m[0] + a.m[3] * b.m[2];
  r.m[3] = a.m[2] * b.m[1] + a.m[3] * b.m[3];
  return r;
}

struct Program {
  int n = 0, nint = 4;
  std::vector<FusedPass> passes;
  std::vector<FusedOp> ops;
  uint8_t pos[16];
  int identity = 1;
  float out_scale = 1.0f;
  int gen_index = 0;  // basis state the program starts from (leading X gates folded)
  int n_instr = 0;    // measure / reset instructions (one pass each)
  std::vector<float2> coef;  // custom unitaries' coefficients (wide passes)
  double cost = 0.0;
  // Empty the program for reuse (keeps the vectors' capacity).
  void reset() {
    passes.clear();
    ops.clear();
    coef.clear();
    n = 0;
    nint = 4;
    identity = 1;
    out_scale = 1.0f;
    gen_index = 0;
    n_instr = 0;
    cost = 0.0;
  }
};

// A scheduled factor of the pass being built (compile_program).
struct CompileRaw {
  Mat2 u;
  GClass cls;
  bool is_h;    // unfused uncontrolled Hadamard
  bool single;  // uncontrolled single-qubit factor
  int t, c;     // physical bits (c = -1: uncontrolled)
};

// Full-state-vector program: per pass the tile bits, the far bits it tests
// and its tile program (FusedCirc k of `progs`, compiled by compile_program).
struct FsvPassInfo {
  uint64_t mask = 0;
  int nfar = 0;
  uint8_t far[kFsvMaxFar + 1] = {};
};
struct FsvProgram {
  int T = 0;  // tile bits per pass
  int max_gates = 0;  // gates per pass at most (0: no limit) it was compiled with
  std::vector<FsvPassInfo> passes;
  std::vector<Program> progs;  // one per pass
};

// At most this many unscaled Hadamard butterflies per pass (bounds the growth
// of the unscaled amplitudes to 2^kMaxHPerPass before the pass rescale).
constexpr int kMaxHPerPass = 48;

// Turn the circuit (gates in step order) into passes of 4 local bits.  One
// in-order scan per pass: a gate is ready when no earlier unscheduled gate
// shares a qubit with it (tracked as `blocked` qubits); a ready non-diagonal
// gate is scheduled if its target bit is or can become local; diagonal gates
// are always scheduled; SWAPs relabel qubits.  Within a pass, consecutive
// uncontrolled single-qubit factors on the same qubit are multiplied in FP64
// (the mixed-product property of the Kronecker product: consecutive steps'
// factors on one qubit compose).  The result does not depend on the other
// circuits of a batch.
static void compile_program(int n, const std::vector<const Gate*>& gs_in, Program& P,
                            bool fold_x = true) {
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

static int team_for(int nint) {
  if (nint <= kWarpMaxQ) return TEAM_WARP;
  if (nint <= kCtaMaxQ) return TEAM_CTA;
  return TEAM_GLOBAL;
}

static int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

}  // namespace tqs

using namespace tqs;

// ------------------------------------------------------------------ circuit

// Allocator whose value-initialisation is a no-op: resize() of a large image
// leaves the new elements for the parallel fill to write.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind { using other = NoInitAlloc<U>; };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    if constexpr (sizeof...(Args) == 0) ::new (static_cast<void*>(p)) U;
    else ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};

// Allocator for image buffers: host memory that is page-locked when the CUDA
// runtime allows it (cudaHostRegister), so that uploads of the image are
// asynchronous DMA rather than copies through a driver staging buffer.  It
// falls back to plain memory (no GPU, or registration refused).  Image buffers
// are recycled, so the registration cost is paid once per buffer.
template <class T>
struct LockedAlloc {
  using value_type = T;
  LockedAlloc() = default;
  template <class U>
  LockedAlloc(const LockedAlloc<U>&) noexcept {}
  template <class U>
  struct rebind { using other = LockedAlloc<U>; };
  T* allocate(size_t n) {
    const size_t bytes = std::max<size_t>(n * sizeof(T), 1);
    void* p = std::malloc(bytes);
    if (!p) throw std::bad_alloc();
    if (bytes >= (size_t(1) << 16) && cudaHostRegister(p, bytes, cudaHostRegisterDefault) != cudaSuccess)
      cudaGetLastError();
    return static_cast<T*>(p);
  }
  void deallocate(T* p, size_t n) {
    if (n * sizeof(T) >= (size_t(1) << 16) && cudaHostUnregister(p) != cudaSuccess) cudaGetLastError();
    std::free(p);
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    if constexpr (sizeof...(Args) == 0) ::new (static_cast<void*>(p)) U;
    else ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
  template <class U>
  bool operator==(const LockedAlloc<U>&) const { return true; }
  template <class U>
  bool operator!=(const LockedAlloc<U>&) const { return false; }
};

// Passes, ops and custom coefficients of a run of programs (one host worker's
// share of a batch, or all of a small image).
struct ImageSeg {
  std::vector<FusedPass, LockedAlloc<FusedPass>> passes;
  std::vector<FusedOp, LockedAlloc<FusedOp>> ops;
  std::vector<float2, LockedAlloc<float2>> coef;
  void clear() {
    passes.clear();
    ops.clear();
    coef.clear();
  }
};

// Where a compiled program of a batch sits before the image is assembled:
// its header fields and its passes / ops / coefficients at local offsets of
// segment `seg` (passes still numbered program-locally).
struct CircMeta {
  int n = 0, nint = 4, n_instr = 0, identity = 1, gen_index = 0;
  float out_scale = 1.0f;
  double cost = 0.0;
  uint8_t pos[16] = {};
  int seg = 0;
  size_t lp = 0, np = 0, lo = 0, no = 0, lc = 0, nc = 0;
};

// Append program P's parts to segment sg (program-local numbering) and
// describe where they went.
static CircMeta append_program(const Program& P, ImageSeg& sg, int seg) {
  CircMeta m;
  m.n = P.n;
  m.nint = P.nint;
  m.n_instr = P.n_instr;
  m.identity = P.identity;
  m.gen_index = P.gen_index;
  m.out_scale = P.out_scale;
  m.cost = P.cost;
  std::memcpy(m.pos, P.pos, 16);
  m.seg = seg;
  m.lp = sg.passes.size();
  m.np = P.passes.size();
  m.lo = sg.ops.size();
  m.no = P.ops.size();
  m.lc = sg.coef.size();
  m.nc = P.coef.size();
  sg.passes.insert(sg.passes.end(), P.passes.begin(), P.passes.end());
  sg.ops.insert(sg.ops.end(), P.ops.begin(), P.ops.end());
  sg.coef.insert(sg.coef.end(), P.coef.begin(), P.coef.end());
  return m;
}

// Recycled segments: a destroyed batch hands its buffers back, so a steady
// stream of batches reuses memory that is already mapped.
static std::mutex g_seg_mu;
static std::vector<ImageSeg> g_seg_pool;

static ImageSeg take_seg() {
  std::lock_guard<std::mutex> lock(g_seg_mu);
  if (g_seg_pool.empty()) return ImageSeg();
  ImageSeg sg = std::move(g_seg_pool.back());
  g_seg_pool.pop_back();
  sg.clear();
  return sg;
}

static void give_segs(std::vector<ImageSeg>& segs) {
  std::lock_guard<std::mutex> lock(g_seg_mu);
  for (ImageSeg& sg : segs)
    if (g_seg_pool.size() < 64) g_seg_pool.push_back(std::move(sg));
  segs.clear();
}

// Large circuit-descriptor arrays are recycled like the segments, so a
// stream of batches pins no fresh pages for them either.
using CircVec = std::vector<FusedCirc, LockedAlloc<FusedCirc>>;
static std::mutex g_circ_mu;
static std::vector<CircVec> g_circ_pool;

static CircVec take_circs(size_t count) {
  CircVec v;
  if (count * sizeof(FusedCirc) >= (size_t(1) << 16)) {
    std::lock_guard<std::mutex> lock(g_circ_mu);
    for (size_t i = 0; i < g_circ_pool.size(); ++i)
      if (g_circ_pool[i].capacity() >= count) {
        v = std::move(g_circ_pool[i]);
        g_circ_pool.erase(g_circ_pool.begin() + static_cast<std::ptrdiff_t>(i));
        break;
      }
  }
  v.resize(count);  // default-initialised: every entry is written by the caller
  return v;
}

static void give_circs(CircVec& v) {
  if (v.capacity() * sizeof(FusedCirc) >= (size_t(1) << 16)) {
    std::lock_guard<std::mutex> lock(g_circ_mu);
    if (g_circ_pool.size() < 8) g_circ_pool.push_back(std::move(v));
  }
  v = CircVec();
}

// Device image of one or more programs:
// [FusedCirc x count][FusedPass...][FusedOp...][custom coefficients (float2)...]
// The passes, ops and coefficients are held as consecutive segments.
struct Image {
  CircVec circs;
  std::vector<ImageSeg> segs;
  size_t npass = 0, nop = 0, ncoef = 0;  // totals over the segments
  ~Image() {
    give_segs(segs);
    give_circs(circs);
  }
  Image() = default;
  Image(const Image&) = delete;
  Image& operator=(const Image&) = delete;
  Image(Image&& o) noexcept { *this = std::move(o); }
  Image& operator=(Image&& o) noexcept {
    give_segs(segs);
    give_circs(circs);
    circs = std::move(o.circs);
    segs = std::move(o.segs);
    npass = o.npass;
    nop = o.nop;
    ncoef = o.ncoef;
    o.npass = o.nop = o.ncoef = 0;
    return *this;
  }
  size_t circ_bytes() const { return circs.size() * sizeof(FusedCirc); }
  size_t pass_bytes() const { return npass * sizeof(FusedPass); }
  size_t op_bytes() const { return nop * sizeof(FusedOp); }
  size_t coef_bytes() const { return ncoef * sizeof(float2); }
  size_t coef_at() const { return circ_bytes() + pass_bytes() + op_bytes(); }
  size_t bytes() const { return coef_at() + coef_bytes(); }
  // Device pointers of the parts of an image uploaded at `base`.
  void point(FusedLaunch& L, const char* base) const {
    L.circs = reinterpret_cast<const FusedCirc*>(base);
    L.passes = reinterpret_cast<const FusedPass*>(base + circ_bytes());
    L.ops = reinterpret_cast<const FusedOp*>(base + circ_bytes() + pass_bytes());
    L.coef = reinterpret_cast<const float2*>(base + coef_at());
  }
  // Pass record with its op / instruction / coefficient offset rebased.
  static FusedPass rebase(FusedPass ps, int64_t op0, int64_t instr0, int64_t coef0) {
    if (ps.L[0] == kInstrPass) ps.op_begin += static_cast<uint32_t>(instr0);
    else if (ps.L[0] == kWidePass) ps.op_begin += static_cast<uint32_t>(coef0);
    else ps.op_begin += static_cast<uint32_t>(op0);
    return ps;
  }
  static FusedCirc circ_of(const Program& P, int64_t pass0, int64_t op0, int64_t out_off) {
    FusedCirc fc{};
    fc.n = static_cast<int16_t>(P.n);
    fc.nint = static_cast<int16_t>(P.nint);
    fc.pass_begin = static_cast<int32_t>(pass0);
    fc.pass_count = static_cast<int32_t>(P.passes.size());
    fc.out_off = out_off;
    fc.op_begin = static_cast<int32_t>(op0);
    fc.op_count = static_cast<int32_t>(P.ops.size());
    fc.identity = P.identity;
    std::memcpy(fc.pos, P.pos, 16);
    fc.init = nullptr;
    fc.out_scale = P.out_scale;
    fc.gen_index = P.gen_index;
    return fc;
  }
  // Append program P (its outputs at amplitude offset out_off).
  void add(const Program& P, int64_t out_off) {
    if (segs.empty()) segs.push_back(take_seg());
    ImageSeg& sg = segs.back();
    circs.push_back(circ_of(P, static_cast<int64_t>(npass), static_cast<int64_t>(nop), out_off));
    for (const FusedPass& ps : P.passes)
      sg.passes.push_back(rebase(ps, static_cast<int64_t>(nop), 0, static_cast<int64_t>(ncoef)));
    sg.ops.insert(sg.ops.end(), P.ops.begin(), P.ops.end());
    sg.coef.insert(sg.coef.end(), P.coef.begin(), P.coef.end());
    npass += P.passes.size();
    nop += P.ops.size();
    ncoef += P.coef.size();
  }
  // Copy the image, laid out as on the device, to host memory at dst.
  void copy_to(char* dst) const {
    std::memcpy(dst, circs.data(), circ_bytes());
    size_t p = circ_bytes(), o = p + pass_bytes(), c = coef_at();
    for (const ImageSeg& sg : segs) {
      if (!sg.passes.empty()) std::memcpy(dst + p, sg.passes.data(), sg.passes.size() * sizeof(FusedPass));
      if (!sg.ops.empty()) std::memcpy(dst + o, sg.ops.data(), sg.ops.size() * sizeof(FusedOp));
      if (!sg.coef.empty()) std::memcpy(dst + c, sg.coef.data(), sg.coef.size() * sizeof(float2));
      p += sg.passes.size() * sizeof(FusedPass);
      o += sg.ops.size() * sizeof(FusedOp);
      c += sg.coef.size() * sizeof(float2);
    }
  }
  cudaError_t upload(void* dst, cudaStream_t s) const {
    char* d = static_cast<char*>(dst);
    cudaError_t e = cudaMemcpyAsync(d, circs.data(), circ_bytes(), cudaMemcpyHostToDevice, s);
    size_t p = circ_bytes(), o = p + pass_bytes(), c = coef_at();
    for (const ImageSeg& sg : segs) {
      if (e == cudaSuccess && !sg.passes.empty())
        e = cudaMemcpyAsync(d + p, sg.passes.data(), sg.passes.size() * sizeof(FusedPass),
                            cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && !sg.ops.empty())
        e = cudaMemcpyAsync(d + o, sg.ops.data(), sg.ops.size() * sizeof(FusedOp),
                            cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && !sg.coef.empty())
        e = cudaMemcpyAsync(d + c, sg.coef.data(), sg.coef.size() * sizeof(float2),
                            cudaMemcpyHostToDevice, s);
      p += sg.passes.size() * sizeof(FusedPass);
      o += sg.ops.size() * sizeof(FusedOp);
      c += sg.coef.size() * sizeof(float2);
    }
    return e;
  }
};

struct tqs_circuit {
  int n = 0;
  int n_instr = 0;  // measure / reset instructions
  std::vector<Gate> gates;
  std::vector<int> last;  // last step touching each qubit
  int nsteps = 0;
  // cached fused program and its device copy
  bool prog_valid = false;
  Program prog;       // for the input |0...0> (leading X gates folded)
  bool prog_init_valid = false;
  Program prog_init;  // for a given input state (nothing folded)
  DevBuf d_prog;      // FusedCirc + passes + ops
  // what d_prog holds: the program (prog or prog_init) and the initial-state
  // pointer it was uploaded with (valid while `uploaded`)
  bool uploaded = false;
  const void* uploaded_prog = nullptr;
  const void* uploaded_init = nullptr;
  cudaEvent_t upload_done = nullptr;  // recorded after the upload, on upload_stream
  cudaStream_t upload_stream = nullptr;
  DevBuf d_counter;   // job counter
  DevBuf d_gscratch;  // TEAM_GLOBAL slot
  // cached plain-form step table
  bool steps_valid = false;
  std::vector<StepFactor> factors;
  std::vector<int64_t> factor_coef;  // per factor: offset in coef_pool, -1 if none
  std::vector<float2> coef_pool;     // custom factors' entries (row-major, FP32)
  std::vector<StepDesc> steps;
  DevBuf d_factors;
  DevBuf d_plain;     // S scratch + two state vectors
  DevBuf d_partials;  // probability partials
  DevBuf d_collapse;  // simulateAndCollapse: state + probabilities
  bool fsv_valid = false;
  FsvProgram fsv;     // full-state-vector passes
  Image fsv_img;      // their tile programs
  DevBuf d_fsv;       // device copy of fsv_img
  DevBuf d_sample;    // sampling scratch
  // chain scratch
  DevBuf d_chain;
  DevBuf d_err;
  ~tqs_circuit() {
    if (upload_done) cudaEventDestroy(upload_done);
  }
};

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

static tqs_status check_gate(int n, int gate, const int* qubits, int nq, const double* params,
                             int np, Gate& g) {
  if (gate < 0 || gate >= TQS_GATE_COUNT) return fail(TQS_ERR_ARG, "unknown gate id %d", gate);
  const int want = is_two_qubit(gate) ? 2 : 1;
  if (!qubits || nq != want)
    return fail(TQS_ERR_ARG, "gate %d takes %d qubit(s), got %d", gate, want, nq);
  const int need = n_params(gate);
  if (np < need || (need > 0 && !params))
    return fail(TQS_ERR_ARG, "gate %d takes %d parameter(s), got %d", gate, need, np);
  for (int i = 0; i < nq; ++i)
    if (qubits[i] < 0 || qubits[i] >= n)
      return fail(TQS_ERR_QUBIT_RANGE, "qubit %d outside [0, %d)", qubits[i], n);
  if (nq == 2 && qubits[0] == qubits[1])
    return fail(TQS_ERR_QUBIT_DUP, "gate %d uses qubit %d twice", gate, qubits[0]);
  g.kind = gate;
  g.nq = nq;
  g.q[0] = qubits[0];
  g.q[1] = nq == 2 ? qubits[1] : qubits[0];
  for (int i = 2; i < kMaxCustomQubits; ++i) g.q[i] = g.q[0];
  g.step = 0;
  if (g.cm) g.cm.reset();
  for (int i = 0; i < 8; ++i) g.p[i] = (i < need) ? params[i] : 0.0;
  for (int i = 0; i < need; ++i)
    if (!std::isfinite(g.p[i])) return fail(TQS_ERR_ARG, "gate %d: non-finite parameter", gate);
  g.u = gate_matrix(gate, g.p);
  if (gate == TQS_CU && !is_unitary(g.u, 1e-9))
    return fail(TQS_ERR_ARG, "CU matrix is not unitary to 1e-9");
  return TQS_OK;
}

}  // extern "C"

// ASAP step of the next operation (Sec. 5.2): after the last step touching any
// of its qubits (`last`: per qubit, -1 if none).  An instruction is a barrier:
// a step of its own after every earlier step, and every later operation comes
// after it.
static void assign_step(std::vector<int>& last, Gate& g) {
  int step = 0;
  if (is_instruction(g.kind)) {
    for (int v : last) step = std::max(step, v + 1);
    for (int& v : last) v = step;
  } else {
    for (int i = 0; i < g.nq; ++i) step = std::max(step, last[g.q[i]] + 1);
    for (int i = 0; i < g.nq; ++i) last[g.q[i]] = step;
  }
  g.step = step;
}

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

// Gates in step order (stable within a step).
// The first `count` gates in step order: counting sort by step, stable, into
// scratch reused on this thread.
static const std::vector<const Gate*>& step_order(const Gate* gates, size_t count) {
  static thread_local std::vector<const Gate*> v;
  static thread_local std::vector<int> start;
  int nsteps = 0;
  for (size_t i = 0; i < count; ++i) nsteps = std::max(nsteps, gates[i].step + 1);
  start.assign(static_cast<size_t>(nsteps) + 1, 0);
  for (size_t i = 0; i < count; ++i) ++start[gates[i].step + 1];
  for (int k = 0; k < nsteps; ++k) start[k + 1] += start[k];
  v.resize(count);
  for (size_t i = 0; i < count; ++i) v[start[gates[i].step]++] = &gates[i];
  return v;
}
static const std::vector<const Gate*>& step_order(const std::vector<Gate>& gates) {
  return step_order(gates.data(), gates.size());
}

static const Program& ensure_program(tqs_circuit* c, bool with_init = false) {
  if (with_init) {
    if (!c->prog_init_valid) {
      c->prog_init = Program();
      compile_program(c->n, step_order(c->gates), c->prog_init, false);
      c->prog_init_valid = true;
    }
    return c->prog_init;
  }
  if (!c->prog_valid) {
    c->prog = Program();
    compile_program(c->n, step_order(c->gates), c->prog);
    c->prog_valid = true;
  }
  return c->prog;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
extern "C" tqs_status tqs_circuit_program(tqs_circuit* c, int* n_passes, int* n_ops, void* h_passes,
                                          void* h_ops, uint8_t* h_pos, float* h_out_scale,
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
  if (h_pos) std::memcpy(h_pos, c->prog.pos, 16);
  if (h_out_scale) *h_out_scale = c->prog.out_scale;
  return TQS_OK;
}


// Everything after the C-ABI entry points below shares these launch helpers.
struct LaunchPlan {
  int team;
  int warps;
  int slice_q;
  int grid;
};

// TQS_OPT_WARPS_PER_CTA table, indexed by the warp slice's log2 amplitudes.
static std::atomic<int> g_warps_for_q[16] = {4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4};
// TQS_OPT_TEAM_WARPS table: warps per circuit of the warp class (1 or 2).
// Gates per full-state-vector pass at most (0: as many as fit a tile).
static std::atomic<int> g_fsv_max_gates{0};
static std::atomic<int> g_team_warps_for_q[16] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};

static LaunchPlan plan_for(int team, int max_nint, int jobs, int warps_hint) {
  LaunchPlan lp{team, 1, 4, 1};
  if (team == TEAM_WARP) {
    lp.slice_q = std::max(4, max_nint);
    const int tw = g_team_warps_for_q[lp.slice_q].load();
    // warps_hint > 0: that many circuits per CTA (a single simulate uses 1)
    int w = warps_hint > 0 ? warps_hint * tw : g_warps_for_q[lp.slice_q].load();
    const size_t slice = (size_t(1) << lp.slice_q) * sizeof(float2);
    if (tw == 2) {
      // warp pairs: an even number of warps, one slice per pair
      lp.team = TEAM_PAIR;
      w = std::max(2, w & ~1);
      while (w > 2 && size_t(w / 2) * slice > 200 * 1024) w -= 2;
    } else {
      while (w > 1 && size_t(w) * slice > 200 * 1024) w >>= 1;
    }
    lp.warps = w;
    const int per_sm = std::max(1, fused_max_ctas_per_sm(lp.team, w, lp.slice_q));
    const int circuits_per_cta = lp.team == TEAM_PAIR ? w / 2 : w;
    const int want = (jobs + circuits_per_cta - 1) / circuits_per_cta;
    lp.grid = std::max(1, std::min(want, per_sm * device_sms()));
  } else if (team == TEAM_CTA) {
    lp.slice_q = std::max(4, max_nint);
    const int per_sm = std::max(1, fused_max_ctas_per_sm(TEAM_CTA, 1, lp.slice_q));
    lp.grid = std::max(1, std::min(jobs, per_sm * device_sms()));
  } else {
    lp.slice_q = kGlobalSlotQ;
    lp.grid = std::max(1, std::min(jobs, device_sms()));
  }
  return lp;
}

// CTAs for a single global-class circuit: one per 512 groups of a pass (a
// thread per group), at most TQS_OPT_MULTI_CTAS; 1 when the program holds
// instructions or custom unitaries, or the device has no cooperative launch.
static std::atomic<int> g_multi_ctas{8};
// TQS_OPT_EXACT_PROBS: the fused kernels' |psi_i|^2 in FP32 arithmetic (0,
// default) or as exact squares rounded once in FP64 (1).
static std::atomic<int> g_exact_probs{0};
constexpr int kMaxMultiJobs = 60;  // barrier counters that fit the server's counter block
static int multi_ctas_for(const Program& P) {
  const int limit = g_multi_ctas.load();
  if (limit < 2 || P.nint <= kCtaMaxQ) return 1;
  for (const FusedPass& ps : P.passes)
    if (ps.L[0] == kInstrPass || ps.L[0] == kWidePass) return 1;
  static int coop = -1;
  if (coop < 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) v = 0;
    coop = v;
  }
  if (!coop) return 1;
  const int groups = 1 << (P.nint - 4);
  return std::max(1, std::min(limit, groups / kGlobalThreads));
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

static void ensure_steps(tqs_circuit* c) {
  if (c->steps_valid) return;
  c->factors.clear();
  c->factor_coef.clear();
  c->coef_pool.clear();
  c->steps.assign(c->nsteps, StepDesc{0, 0, 0, 0});
  const uint32_t all = (1u << c->n) - 1u;
  std::vector<std::vector<const Gate*>> by_step(c->nsteps);
  for (const Gate& g : c->gates) by_step[g.step].push_back(&g);
  for (int k = 0; k < c->nsteps; ++k) {
    StepDesc d{static_cast<int32_t>(c->factors.size()), 0, all, 0};
    for (const Gate* g : by_step[k]) {
      StepFactor f{};
      int64_t coef_at = -1;
      if (is_wide(*g)) {
        f.nq = static_cast<uint8_t>(g->nq);
        f.custom = 1;
        for (int t = 0; t < g->nq; ++t) f.qc[t] = static_cast<uint8_t>(g->q[t]);
        coef_at = static_cast<int64_t>(c->coef_pool.size());
        for (const cd& v : g->cm->m) c->coef_pool.push_back(to_f2(v));
        d.idle &= ~qubit_mask(*g);
      } else if (!is_two_qubit(g->kind)) {
        f.nq = 1;
        f.q0 = f.q1 = static_cast<uint8_t>(g->q[0]);
        for (int i = 0; i < 4; ++i) f.m[i] = to_f2(g->u.m[i]);
        d.idle &= ~(1u << g->q[0]);
      } else {
        f.nq = 2;
        f.q0 = static_cast<uint8_t>(g->q[0]);
        f.q1 = static_cast<uint8_t>(g->q[1]);
        cd M[16] = {};
        if (g->kind == TQS_SWAP) {
          // |a b> -> |b a> in the (q0, q1) labelling
          M[0 * 4 + 0] = 1.0;
          M[1 * 4 + 2] = 1.0;
          M[2 * 4 + 1] = 1.0;
          M[3 * 4 + 3] = 1.0;
        } else {
          // eq. 7: diag(I, U) with the control first
          M[0 * 4 + 0] = 1.0;
          M[1 * 4 + 1] = 1.0;
          M[2 * 4 + 2] = g->u.m[0];
          M[2 * 4 + 3] = g->u.m[1];
          M[3 * 4 + 2] = g->u.m[2];
          M[3 * 4 + 3] = g->u.m[3];
        }
        for (int i = 0; i < 16; ++i) f.m[i] = to_f2(M[i]);
        d.idle &= ~((1u << g->q[0]) | (1u << g->q[1]));
      }
      c->factors.push_back(f);
      c->factor_coef.push_back(coef_at);
      ++d.f_count;
    }
    c->steps[k] = d;
  }
  c->steps_valid = true;
}

// Device step table: [StepFactor...][custom entries (float2)...]; each custom
// factor's `coef` points into the second part.
static tqs_status upload_factors(tqs_circuit* c, cudaStream_t s) {
  ensure_steps(c);
  const size_t fbytes = (std::max<size_t>(c->factors.size(), 1) * sizeof(StepFactor) + 15) & ~size_t(15);
  const size_t bytes = fbytes + c->coef_pool.size() * sizeof(float2);
  TQS_CUDA(c->d_factors.ensure(bytes), "cudaMalloc step table");
  const float2* pool = reinterpret_cast<const float2*>(c->d_factors.as<char>() + fbytes);
  std::vector<StepFactor> fs = c->factors;
  for (size_t i = 0; i < fs.size(); ++i)
    if (c->factor_coef[i] >= 0) fs[i].coef = pool + c->factor_coef[i];
  if (!fs.empty())
    TQS_CUDA(cudaMemcpyAsync(c->d_factors.p, fs.data(), fs.size() * sizeof(StepFactor),
                             cudaMemcpyHostToDevice, s),
             "upload step table");
  if (!c->coef_pool.empty())
    TQS_CUDA(cudaMemcpyAsync(c->d_factors.as<char>() + fbytes, c->coef_pool.data(),
                             c->coef_pool.size() * sizeof(float2), cudaMemcpyHostToDevice, s),
             "upload custom entries");
  return TQS_OK;
}

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

// ------------------------------------------------------------------ batch

// Segment tables of an inverse-CDF sampling call (see k_sample.cu).
struct SamplePlan {
  std::vector<SampleSeg> gsegs, ssegs;
  int64_t nblocks = 0, probs_end = 0, n_segs = 0;
  int smem_q = 0;
  size_t off_g = 0, off_s = 0, off_bsum = 0, off_bpre = 0, off_cpre = 0, off_tot = 0, bytes = 0;
  void layout() {
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    off_g = 0;
    off_s = up(gsegs.size() * sizeof(SampleSeg));
    off_bsum = off_s + up(ssegs.size() * sizeof(SampleSeg));
    off_bpre = off_bsum + up(size_t(nblocks) * sizeof(double));
    off_cpre = off_bpre + up(size_t(nblocks) * sizeof(double));
    off_tot = off_cpre + up(size_t(nblocks) * (kSampleBlk / kSampleChunk) * sizeof(double));
    bytes = off_tot + up(gsegs.size() * sizeof(double));
  }
  // Segment `index` of 2^n probabilities at p_off; small ones go to the
  // shared-memory path when allowed.
  void add(int64_t index, int64_t p_off, int n, bool allow_smem) {
    probs_end = std::max(probs_end, p_off + (int64_t(1) << n));
    n_segs = std::max(n_segs, index + 1);
    if (allow_smem && n <= kSampleSmemMaxQ) {
      ssegs.push_back(SampleSeg{p_off, n, 0, index});
      smem_q = std::max(smem_q, n);
    } else {
      gsegs.push_back(SampleSeg{p_off, n, static_cast<int32_t>(nblocks), index});
      nblocks += sample_blocks(n);
    }
  }
  cudaError_t upload(char* base, cudaStream_t s) const {
    cudaError_t e = cudaSuccess;
    if (!gsegs.empty())
      e = cudaMemcpyAsync(base + off_g, gsegs.data(), gsegs.size() * sizeof(SampleSeg),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !ssegs.empty())
      e = cudaMemcpyAsync(base + off_s, ssegs.data(), ssegs.size() * sizeof(SampleSeg),
                          cudaMemcpyHostToDevice, s);
    return e;
  }
  SampleLaunch launch(char* base, const double* probs, const double* u, int64_t shots,
                      int64_t* out) const {
    SampleLaunch L{};
    L.probs = probs;
    L.gsegs = reinterpret_cast<const SampleSeg*>(base + off_g);
    L.n_gseg = static_cast<int32_t>(gsegs.size());
    L.nblocks = nblocks;
    L.bsum = reinterpret_cast<double*>(base + off_bsum);
    L.bpre = reinterpret_cast<double*>(base + off_bpre);
    L.cpre = reinterpret_cast<double*>(base + off_cpre);
    L.tot = reinterpret_cast<double*>(base + off_tot);
    L.ssegs = reinterpret_cast<const SampleSeg*>(base + off_s);
    L.n_sseg = static_cast<int32_t>(ssegs.size());
    L.smem_q = smem_q;
    L.u = u;
    L.shots = shots;
    L.out = out;
    L.probs_len = probs_end;
    L.n_segs = n_segs;
    return L;
  }
};

struct tqs_batch {
  int count = 0;
  int64_t total_steps = 0;
  std::vector<int64_t> offsets;  // count + 1
  std::vector<int64_t> instr_off;  // count + 1: instruction (uniform / outcome) offsets
  Image img;
  std::vector<int32_t> order;    // [warp jobs][cta jobs][global jobs]
  int n_team[3] = {0, 0, 0};
  int max_nint[3] = {4, 4, 4};
  DevBuf d_img;                  // image + order + counters
  size_t order_off = 0, counter_off = 0;
  bool uploaded = false;
  DevBuf d_gscratch;
  DevBuf d_sample;               // sampling: segment tables + block sums / prefixes
  std::unique_ptr<SamplePlan> sample_plan;
  LaunchPlan plans[3];
  // graph cache
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* g_states = nullptr;
  void* g_probs = nullptr;
  void* g_norms = nullptr;
  const void* g_u = nullptr;
  void* g_outcomes = nullptr;
  int g_exact = -1;
  int exact_probs = 0;             // TQS_OPT_EXACT_PROBS when the batch last ran
  int graph_kernels = 0;
  ~tqs_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

// Run body(i) for i in [0, count) on the host cores.
// Persistent host worker threads for parallel_for: created on first use and
// kept, so per-thread scratch (compile buffers) survives from one batch to
// the next.  One job runs at a time; the calling thread takes part.  A child
// process after fork() gets its own pool.
class HostPool {
 public:
  static HostPool& get() {
    static std::mutex mu;
    static HostPool* pool = nullptr;
    static pid_t owner = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!pool || owner != getpid()) {  // the parent's threads do not exist after fork()
      pool = new HostPool();           // kept until exit: its threads wait for work
      owner = getpid();
    }
    return *pool;
  }
  int size() const { return static_cast<int>(threads_.size()) + 1; }
  // body(i) for i in [0, count) on up to `width` threads (the caller included),
  // handed out `chunk` consecutive indices at a time.
  void run(int count, int width, int chunk, const std::function<void(int)>& body) {
    std::lock_guard<std::mutex> one_job(run_mu_);
    {
      std::lock_guard<std::mutex> lock(mu_);
      body_ = &body;
      count_ = count;
      chunk_ = std::max(1, chunk);
      next_.store(0);
      width_ = std::min(width, size());
      pending_ = width_ - 1;
      ++generation_;
    }
    cv_.notify_all();
    drain();
    std::unique_lock<std::mutex> lock(mu_);
    done_cv_.wait(lock, [&] { return pending_ == 0; });
    body_ = nullptr;
  }

 private:
  HostPool() {
    const int hw = static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
    for (int t = 1; t < std::min(hw, 32); ++t) threads_.emplace_back([this, t] { loop(t); });
  }
  void drain() {
    for (int c = next_.fetch_add(1); c * chunk_ < count_; c = next_.fetch_add(1)) {
      const int end = std::min(count_, (c + 1) * chunk_);
      for (int i = c * chunk_; i < end; ++i) (*body_)(i);
    }
  }
  void loop(int index) {
    uint64_t seen = 0;
    for (;;) {
      std::unique_lock<std::mutex> lock(mu_);
      cv_.wait(lock, [&] { return generation_ != seen; });
      seen = generation_;
      const bool take_part = index < width_;
      lock.unlock();
      if (!take_part) continue;
      drain();
      lock.lock();
      if (--pending_ == 0) done_cv_.notify_all();
    }
  }
  std::vector<std::thread> threads_;
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* body_ = nullptr;
  int count_ = 0, width_ = 1, pending_ = 0, chunk_ = 1;
  uint64_t generation_ = 0;
  std::atomic<int> next_{0};
};

// Run body(i) for i in [0, count) on the host cores (at most TQS_HOST_THREADS
// of them when that variable is set), `grain` items per thread at least.
template <class F>
static void parallel_for(int count, int grain, F body) {
  int hw = static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
  if (const char* env = std::getenv("TQS_HOST_THREADS")) hw = std::max(1, std::atoi(env));
  const int width = std::min({hw, 32, std::max(1, count / std::max(1, grain))});
  if (width <= 1) {
    for (int i = 0; i < count; ++i) body(i);
    return;
  }
  const std::function<void(int)> fn = body;
  // chunks of about grain indices, several per thread for balance
  const int chunk = std::max(1, std::min(grain, count / (4 * width)));
  HostPool::get().run(count, width, chunk, fn);
}

// Assemble the batch image from compiled programs held in segments: the
// device arrays are the segments concatenated in order, so a program's global
// offsets are its segment's base plus its local offsets.  Headers are written
// and passes renumbered in parallel, in place.
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
    fc.identity = m.identity;
    std::memcpy(fc.pos, m.pos, 16);
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
  // the gate counts of its range (fusion only shrinks a program: at most one
  // op per gate and one pass per gate plus one), so it never reallocates.
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
      sg.ops.reserve(static_cast<size_t>(span));
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
    TQS_CUDA(launch_fused(L, s), "tqs_batch: launch");
    first += b->n_team[t];
    ++k;
  }
  if (kernels) *kernels = k;
  return TQS_OK;
}

static tqs_status batch_enqueue(tqs_batch* b, float2* states, double* probs, double* norms,
                                cudaStream_t s, int* kernels, const double* u = nullptr,
                                int32_t* outcomes = nullptr) {
  return batch_enqueue_at(b, b->d_img.as<char>(), b->order_off, b->counter_off,
                          b->d_gscratch.as<float2>(), states, probs, norms, s, kernels, u, outcomes);
}

// Keep freed stream-ordered allocations in the device's default memory pool
// (the process's own pool) so that repeated calls do not go back to the driver.
static void keep_pool_memory() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
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

}  // extern "C"

// Device alias of a host range the GPU can write directly: page-locked,
// mapped into the device's address space, one contiguous alias over the whole
// range (on Grace-Blackwell the kernel's stores then cross NVLink-C2C straight
// into host memory).  nullptr when any check fails; the caller then stages
// through device memory.
// TQS_OPT_HOST_WRITES: 1 (default) lets tqs_batch_run_host's kernels write
// page-locked host outputs directly; 0 stages them in device memory and copies.
static std::atomic<int> g_host_writes{1};

static void* mapped_alias(void* h, size_t bytes) {
  if (!h || bytes == 0) return nullptr;
  char* first = static_cast<char*>(h);
  char* last = first + bytes - 1;
  void* d0 = nullptr;
  void* d1 = nullptr;
  for (char* p : {first, last}) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return nullptr;
    }
  }
  if (cudaHostGetDevicePointer(&d0, first, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(&d1, last, 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (static_cast<char*>(d1) != static_cast<char*>(d0) + (bytes - 1) || !aligned16(d0)) return nullptr;
  return d0;
}

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

tqs_status tqs_circuit_unitary(tqs_circuit* c, int prec, tqs_c64* d_U, void* stream) {
  if (c && c->n_instr > 0)
    return fail(TQS_ERR_UNSUPPORTED,
                "tqs_circuit_unitary: measure/reset instructions have no circuit unitary");
  if (!c || !d_U) return fail(TQS_ERR_ARG, "tqs_circuit_unitary: NULL argument");
  if (!aligned16(d_U)) return fail(TQS_ERR_ARG, "tqs_circuit_unitary: d_U must be 16-byte aligned");
  if (c->n > TQS_MAX_DENSE_QUBITS)
    return fail(TQS_ERR_TOO_MANY_QUBITS, "tqs_circuit_unitary: n %d > %d", c->n, TQS_MAX_DENSE_QUBITS);
  if (prec != TQS_PREC_FP32_SIMT && prec != TQS_PREC_TC_BF16X3 && prec != TQS_PREC_TC_TF32X3)
    return fail(TQS_ERR_ARG, "tqs_circuit_unitary: unknown precision %d", prec);
  if (prec != TQS_PREC_FP32_SIMT && c->n < 7)
    return fail(TQS_ERR_ARG, "tqs_circuit_unitary: the tensor-core chain needs n >= 7");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tqs_status st = upload_factors(c, s);
  if (st != TQS_OK) return st;
  float2* U = reinterpret_cast<float2*>(d_U);
  if (c->nsteps <= 1) {
    // Algorithm 1 with at most one step: U = S_1 (or the identity).
    StepDesc d = c->nsteps == 1 ? c->steps[0] : StepDesc{0, 0, (1u << c->n) - 1u, 0};
    TQS_CUDA(launch_materialize(c->d_factors.as<StepFactor>(), d, c->n, U, s),
             "tqs_circuit_unitary: materialize");
    return TQS_OK;
  }
  if (prec == TQS_PREC_FP32_SIMT) {
    TQS_CUDA(c->d_chain.ensure(chain_simt_scratch_bytes(c->n)), "tqs_circuit_unitary: cudaMalloc");
    TQS_CUDA(chain_simt(c->d_factors.as<StepFactor>(), c->steps.data(), c->nsteps, c->n, U,
                        c->d_chain.p, s),
             "tqs_circuit_unitary: SIMT chain");
    return TQS_OK;
  }
  TQS_CUDA(c->d_chain.ensure(chain_tc_scratch_bytes(c->n, prec)), "tqs_circuit_unitary: cudaMalloc");
  TQS_CUDA(c->d_err.ensure(sizeof(int)), "tqs_circuit_unitary: cudaMalloc");
  TQS_CUDA(cudaMemsetAsync(c->d_err.p, 0, sizeof(int), s), "tqs_circuit_unitary: memset");
  TQS_CUDA(chain_tc(c->d_factors.as<StepFactor>(), c->steps.data(), c->nsteps, c->n, prec, U,
                    c->d_chain.p, c->d_err.as<int>(), s),
           "tqs_circuit_unitary: tensor-core chain");
  int err = 0;
  TQS_CUDA(cudaMemcpyAsync(&err, c->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s),
           "tqs_circuit_unitary: read status");
  TQS_CUDA(cudaStreamSynchronize(s), "tqs_circuit_unitary: sync");
  if (err) return fail(TQS_ERR_TIMEOUT, "tqs_circuit_unitary: a device wait ran out");
  return TQS_OK;
}

}  // extern "C"

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

static tqs_status compile_fsv(int n, const std::vector<Gate>& gates, int max_gates, FsvProgram& P) {
  P = FsvProgram();
  P.max_gates = max_gates;
  // 2^13-amplitude tiles from 24 qubits on (fewer passes); below that 2^12,
  // so that a state still spreads over enough tiles to fill the GPU
  const int T = std::min(n, n >= 24 ? kFsvTileQ : kFsvTileQ - 1);
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
    compile_program(T + info.nfar, ptrs, tp, false);
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
  if (!c->fsv_valid || c->fsv.max_gates != max_gates) {
    tqs_status st = compile_fsv(c->n, c->gates, max_gates, c->fsv);
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
  if (!c->fsv_valid || c->fsv.max_gates != max_gates) {
    tqs_status st = compile_fsv(c->n, c->gates, max_gates, local);
    if (st != TQS_OK) return st;
    P = &local;
  }
  if (n_passes) *n_passes = static_cast<int>(P->passes.size());
  if (tile_bits) *tile_bits = P->T;
  return TQS_OK;
}

}  // extern "C"
