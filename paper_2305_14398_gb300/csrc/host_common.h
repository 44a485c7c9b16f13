// Host-side internals shared by the C-ABI translation units (tqs_host.cpp,
// host_compile.cpp, host_batch.cpp, host_server.cpp, host_fsv.cpp): errors, the device
// allocator hook, gate data, the fused-pass compiler's types, program images,
// the circuit, batch and sampling structures, the host thread pool and the
// launch options.  Not part of the public interface (include/tqs.h).
#pragma once

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

inline thread_local std::string g_last_error;
inline std::atomic<int64_t> g_launches{0};

inline tqs_status fail(tqs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

inline tqs_status cuda_fail(cudaError_t e, const char* what) {
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
inline std::mutex g_alloc_mu;
inline Allocator g_alloc;

inline Allocator current_allocator() {
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  return g_alloc;
}

// Allocate `bytes` of device memory for use on `s` with allocator A.
inline cudaError_t dev_alloc(const Allocator& A, void** p, size_t bytes, cudaStream_t s) {
  if (!A.alloc) return cudaMalloc(p, bytes);
  *p = A.alloc(bytes, s, A.ctx);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

// Return p to allocator A.  With s = nullptr the device is synchronised
// first (as cudaFree does), so no queued work still reads the buffer when the
// caller's allocator hands it out again; with a stream, frees are
// stream-ordered on it.
inline void dev_free(const Allocator& A, void* p, cudaStream_t s) {
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

inline bool is_controlled(int g) { return g == TQS_CNOT || g == TQS_CZ || g == TQS_CP || g == TQS_CU; }
inline bool is_instruction(int g) { return g == TQS_MEASURE || g == TQS_RESET; }
inline bool is_two_qubit(int g) { return is_controlled(g) || g == TQS_SWAP; }
inline int n_params(int g) {
  switch (g) {
    case TQS_R: case TQS_RX: case TQS_RY: case TQS_RZ: case TQS_CP: return 1;
    case TQS_U3: return 3;
    case TQS_CU: return 8;
    default: return 0;
  }
}

// e^{i phi} (std::polar), remembered per host thread in a small direct-mapped
// table keyed by phi's bits: the phase gates of a batch repeat the same few
// angles (a QFT's controlled phases), and sin/cos dominate building them.
inline cd unit_phase(double phi) {
  struct Entry {
    uint64_t key = 0;
    cd v;
    bool used = false;
  };
  static thread_local Entry table[128];
  uint64_t k;
  std::memcpy(&k, &phi, 8);
  Entry& e = table[(k * 0x9E3779B97F4A7C15ull) >> 57];
  if (e.used && e.key == k) return e.v;
  e.key = k;
  e.v = std::polar(1.0, phi);
  e.used = true;
  return e.v;
}

// Single-qubit matrix of a gate, or the U of a controlled gate.
inline Mat2 gate_matrix(int g, const double* p) {
  const double r2 = 1.0 / std::sqrt(2.0);
  const cd I(0.0, 1.0);
  Mat2 u;
  switch (g) {
    case TQS_H: u = {{r2, r2, r2, -r2}}; break;
    case TQS_X: case TQS_CNOT: u = {{0.0, 1.0, 1.0, 0.0}}; break;
    case TQS_Y: u = {{0.0, -I, I, 0.0}}; break;
    case TQS_Z: case TQS_CZ: u = {{1.0, 0.0, 0.0, -1.0}}; break;
    case TQS_S: u = {{1.0, 0.0, 0.0, I}}; break;
    case TQS_T: u = {{1.0, 0.0, 0.0, unit_phase(M_PI / 4.0)}}; break;
    case TQS_R: case TQS_CP: u = {{1.0, 0.0, 0.0, unit_phase(p[0])}}; break;
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
    case TQS_RZ: u = {{unit_phase(-p[0] / 2), 0.0, 0.0, unit_phase(p[0] / 2)}}; break;
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

inline bool is_unitary(const Mat2& u, double tol) {
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

inline bool is_wide(const Gate& g) { return g.kind == kCustomKind && g.nq >= 2; }
inline uint32_t qubit_mask(const Gate& g) {
  uint32_t m = 0;
  for (int i = 0; i < g.nq; ++i) m |= 1u << g.q[i];
  return m;
}

inline float2 to_f2(cd z) {
  return make_float2(static_cast<float>(z.real()), static_cast<float>(z.imag()));
}

// ---------------------------------------------------------- fused compile

enum GClass { G_DENSE, G_ANTI, G_DIAG, G_SWAP };

inline GClass classify_mat(const Mat2& u) {
  if (u.m[1] == cd(0.0) && u.m[2] == cd(0.0)) return G_DIAG;
  if (u.m[0] == cd(0.0) && u.m[3] == cd(0.0)) return G_ANTI;
  return G_DENSE;
}

inline GClass classify(const Gate& g) {
  if (g.kind == TQS_SWAP) return G_SWAP;
  return classify_mat(g.u);
}

// a * b (apply b, then a)
inline Mat2 mat_mul(const Mat2& a, const Mat2& b) {
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
  uint16_t col[16];       // output map (FusedCirc)
  uint16_t col_off = 0;
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
    col_off = 0;
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
  int tile_opt = 0;   // TQS_OPT_FSV_TILE_Q it was compiled with
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
// absorb: fold the trailing permutation gates into the output map (not in
// the full-state-vector tile programs, whose write-back is the tile's own).
void compile_program(int n, const std::vector<const Gate*>& gs_in, Program& P,
                     bool fold_x = true, bool absorb = true);

inline int team_for(int nint) {
  if (nint <= kWarpMaxQ) return TEAM_WARP;
  if (nint <= kCtaMaxQ) return TEAM_CTA;
  return TEAM_GLOBAL;
}

inline int device_sms() {
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
  int n = 0, nint = 4, n_instr = 0, gen_index = 0;
  float out_scale = 1.0f;
  double cost = 0.0;
  uint16_t col[16] = {};
  uint16_t col_off = 0;
  int seg = 0;
  size_t lp = 0, np = 0, lo = 0, no = 0, lc = 0, nc = 0;
};

// Append program P's parts to segment sg (program-local numbering) and
// describe where they went.
inline CircMeta append_program(const Program& P, ImageSeg& sg, int seg) {
  CircMeta m;
  m.n = P.n;
  m.nint = P.nint;
  m.n_instr = P.n_instr;
  m.col_off = P.col_off;
  m.gen_index = P.gen_index;
  m.out_scale = P.out_scale;
  m.cost = P.cost;
  std::memcpy(m.col, P.col, sizeof(m.col));
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
inline std::mutex g_seg_mu;
inline std::vector<ImageSeg> g_seg_pool;

inline ImageSeg take_seg() {
  std::lock_guard<std::mutex> lock(g_seg_mu);
  if (g_seg_pool.empty()) return ImageSeg();
  ImageSeg sg = std::move(g_seg_pool.back());
  g_seg_pool.pop_back();
  sg.clear();
  return sg;
}

inline void give_segs(std::vector<ImageSeg>& segs) {
  std::lock_guard<std::mutex> lock(g_seg_mu);
  for (ImageSeg& sg : segs)
    if (g_seg_pool.size() < 64) g_seg_pool.push_back(std::move(sg));
  segs.clear();
}

// Large circuit-descriptor arrays are recycled like the segments, so a
// stream of batches pins no fresh pages for them either.
using CircVec = std::vector<FusedCirc, LockedAlloc<FusedCirc>>;
inline std::mutex g_circ_mu;
inline std::vector<CircVec> g_circ_pool;

inline CircVec take_circs(size_t count) {
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

inline void give_circs(CircVec& v) {
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
    fc.col_off = P.col_off;
    std::memcpy(fc.col, P.col, sizeof(fc.col));
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

// ---------------------------------------------- shared helpers of the entry points

inline tqs_status check_gate(int n, int gate, const int* qubits, int nq, const double* params,
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

// ASAP step of the next operation (Sec. 5.2): after the last step touching any
// of its qubits (`last`: per qubit, -1 if none).  An instruction is a barrier:
// a step of its own after every earlier step, and every later operation comes
// after it.
inline void assign_step(std::vector<int>& last, Gate& g) {
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

// Gates in step order (stable within a step).
// The first `count` gates in step order: counting sort by step, stable, into
// scratch reused on this thread.
inline const std::vector<const Gate*>& step_order(const Gate* gates, size_t count) {
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
inline const std::vector<const Gate*>& step_order(const std::vector<Gate>& gates) {
  return step_order(gates.data(), gates.size());
}

inline const Program& ensure_program(tqs_circuit* c, bool with_init = false) {
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

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Everything after the C-ABI entry points below shares these launch helpers.
struct LaunchPlan {
  int team;
  int warps;
  int slice_q;
  int grid;
};

// TQS_OPT_WARPS_PER_CTA table, indexed by the warp slice's log2 amplitudes.
inline std::atomic<int> g_warps_for_q[16] = {4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4};
// TQS_OPT_TEAM_WARPS table: warps per circuit of the warp class (1 or 2).
// Gates per full-state-vector pass at most (0: as many as fit a tile).
inline std::atomic<int> g_fsv_max_gates{0};
inline std::atomic<int> g_team_warps_for_q[16] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
// TQS_OPT_CTA_THREADS: threads of the CTA team (circuits of 12..14 qubits).
inline std::atomic<int> g_cta_threads{kCtaThreads};
// TQS_OPT_FSV_TILE_Q: tile bits of the full-state-vector passes (0: automatic).
inline std::atomic<int> g_fsv_tile_q{0};
// TQS_OPT_CHAIN_GROUP: tile rows per raster band of the tensor-core chain.
inline std::atomic<int> g_chain_group{16};
// TQS_OPT_CHAIN_KCHUNK: K per accumulation chunk of the tensor-core chain
// (0: the precision's default).
inline std::atomic<int> g_chain_kchunk{0};
// TQS_OPT_CHAIN_PAIR: the chain's GEMMs as two-CTA clusters sharing B tiles (1) or not (0).
inline std::atomic<int> g_chain_pair{0};

inline LaunchPlan plan_for(int team, int max_nint, int jobs, int warps_hint) {
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
    lp.warps = g_cta_threads.load() / 32;
    const int per_sm = std::max(1, fused_max_ctas_per_sm(TEAM_CTA, lp.warps, lp.slice_q));
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
inline std::atomic<int> g_multi_ctas{8};
// TQS_OPT_EXACT_PROBS: the fused kernels' |psi_i|^2 in FP32 arithmetic (0,
// default) or as exact squares rounded once in FP64 (1).
inline std::atomic<int> g_exact_probs{0};
constexpr int kMaxMultiJobs = 60;  // barrier counters that fit the server's counter block
inline int multi_ctas_for(const Program& P) {
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

inline void ensure_steps(tqs_circuit* c) {
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
inline tqs_status upload_factors(tqs_circuit* c, cudaStream_t s) {
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
  // When the batch holds circuits of more than one team kind, their kernels run
  // side by side: forked from the caller's stream onto these streams and
  // joined back (inside a captured graph too), so the kinds share the GPU in
  // each other's tails instead of running one after the other.
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[3] = {nullptr, nullptr, nullptr};
  cudaError_t ensure_side() {
    if (ev_fork) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < 3 && e == cudaSuccess; ++t) {
      if (!side[t]) e = cudaStreamCreateWithFlags(&side[t], cudaStreamNonBlocking);
      if (e == cudaSuccess && !ev_join[t]) e = cudaEventCreateWithFlags(&ev_join[t], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    return e;
  }
  ~tqs_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (int t = 0; t < 3; ++t) {
      if (side[t]) cudaStreamDestroy(side[t]);
      if (ev_join[t]) cudaEventDestroy(ev_join[t]);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
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
inline void parallel_for(int count, int grain, F body) {
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

// Keep freed stream-ordered allocations in the device's default memory pool
// (the process's own pool) so that repeated calls do not go back to the driver.
inline void keep_pool_memory() {
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

// Device alias of a host range the GPU can write directly: page-locked,
// mapped into the device's address space, one contiguous alias over the whole
// range (on Grace-Blackwell the kernel's stores then cross NVLink-C2C straight
// into host memory).  nullptr when any check fails; the caller then stages
// through device memory.
// TQS_OPT_HOST_WRITES: 1 (default) lets tqs_batch_run_host's kernels write
// page-locked host outputs directly; 0 stages them in device memory and copies.
inline std::atomic<int> g_host_writes{1};

inline void* mapped_alias(void* h, size_t bytes) {
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
