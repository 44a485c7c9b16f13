// Internal data layouts shared by the host compiler (tqs_host.cpp) and the
// sm_103a kernels.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tqs {

// ---------------------------------------------------------------------------
// Fused step program.
//
// The host turns a circuit's steps (Algorithm 2: one Kronecker factor per gate,
// identity elsewhere) into "passes".  A pass names 4 physical qubit bits that
// are local to a thread: each thread owns the 16 amplitudes whose indices differ
// only in those bits and applies, in registers, every factor of the pass whose
// non-diagonal action stays inside them (eq. 12 butterflies; a controlled
// factor's control may be any qubit).  Diagonal factors are phases and need no
// locality.  SWAP factors are qubit relabelings done on the host.
// ---------------------------------------------------------------------------

// Dispatch code of an op (one jump per op in the kernel).  "+ t": local target
// position t (0..3); "+ 4 t + c": local target t and local control c.
//   OPC_H + t        uncontrolled Hadamard without its 2^-1/2: (x0 + x1, x0 - x1);
//                    the pass scale restores the factor exactly
//   OPC_X + t        uncontrolled exchange of the pair (X)
//   OPC_XF + t       exchange where far control bit `fbit` of the group is 1 (CNOT)
//   OPC_XL + 4t + c  exchange in the pairs whose local control bit c is 1 (CNOT)
//   OPC_HMASK        unscaled Hadamards on the local positions of the bit mask
//                    in field t (two or more, in position order; they commute);
//                    anti-diagonal factors other than X run as DENSE (fewer
//                    kernel code paths, and their coefficients get hi + lo)
//   OPC_XP           exchanges on local position t (field t) that commute and
//                    compose: the pair (j, j ^ 2^t) swaps when bit j of `act`
//                    XOR the parity of the group's physical bits in the far
//                    mask (the first 4 bytes of hc) is 1; field c = the local
//                    control positions (a run of X / CNOT factors on one target)
//   OPC_DENSE + t    uncontrolled 2x2, coefficients as FP32 hi + lo
//   OPC_CDENSE + t   controlled 2x2 (`act` mask for a local control, `fbit` far)
//   OPC_DLN + t      diag(d0, d1), local target, uncontrolled
//   OPC_DLF + t      diag(d0, d1), local target, far control `fbit`
//   OPC_DFL + c      diag(d0, d1), far target bit `tbit`, local control c
//   OPC_DFF          diag(d0, d1), far target bit `tbit`, no or far control `fbit`
//   OPC_DLL          diag(d0, d1), local target t and local control c (fields t, c)
//   OPC_DIAG16       a diagonal over the 16 local indices: entry j (the
//                    product of a run of OPC_DLL factors) multiplies
//                    amplitude j; entries 0..7 in m[0..3], lo[0..3] of this
//                    record, 8..15 in those of the next record (OPC_NOP)
//   OPC_NOP          does nothing (the second record of an OPC_DIAG16)
//   OPC_DLIST        up to 8 phase factors merged into one op: field t = the
//                    local position they multiply (0..3: the amplitudes with
//                    that local bit set; 4: the whole group), field c = their
//                    count; factor e (m[0..3], then lo[0..3]) applies when
//                    the group's physical bit hc-byte e is 1 (0xFF: always)
//   OPC_DLISTM       phase lists of several targets (field t: a mask of local
//                    positions 0..3 and bit 4 for the group) over the same
//                    factor bits (hc bytes, as for OPC_DLIST; field c = their
//                    count, padded to 8 with 0xFF): one record per target in
//                    increasing order (this one, then OPC_NOP records), each
//                    with the target's 8 factors in m[0..3], lo[0..3]; the
//                    bits are tested once for all targets
// Diagonal ops carry d0, d1, d1/d0 and `d0one` = 1 when d0 is exactly 1; the
// coefficient they use when d0 is 1 is repeated in the header (`hc`).
enum OpCode : uint8_t {
  OPC_H = 0,
  OPC_X = 4,
  OPC_XF = 8,
  OPC_XL = 12,       // 16 codes (t, c), c != t used
  OPC_ANTI = 28,      // end of the exchange codes
  OPC_HMASK = 28,
  OPC_XP = 29,
  OPC_DENSE = 32,
  OPC_CDENSE = 36,
  OPC_DLN = 40,
  OPC_DLF = 44,
  OPC_DFL = 48,
  OPC_DFF = 52,
  OPC_DLL = 53,
  OPC_DLIST = 54,
  OPC_DIAG16 = 55,
  OPC_NOP = 56,
  OPC_DLISTM = 57,
  OPC_COUNT = 58
};

struct alignas(16) FusedOp {
  uint8_t code;    // OpCode
  uint8_t t;       // local target position (OPC_DLL)
  uint8_t c;       // local control position (OPC_DLL)
  uint8_t tbit;    // physical bit of a far target (OPC_DFL, OPC_DFF)
  uint8_t d0one;   // diagonal ops: d0 == 1 exactly
  uint8_t fbit;    // physical bit of a far control, 0xFF if none
  uint16_t act;    // active-pair mask over the 16 local indices (ANTI, CDENSE)
  float2 hc;       // diagonal ops, in the header so no further load is needed in the
                   // common case: d1/d0 (DLN, DLF) or d1 (DFL, DFF, DLL)
  float2 m[4];     // DENSE: m00 m01 m10 m11 | ANTI: -, m01, m10, - | DIAG: d0, d1, d1/d0, -
  float2 lo[4];    // DENSE: m - m_fp32 rounded to FP32 (the FP64 matrix is m + lo)
};
static_assert(sizeof(FusedOp) == 80, "FusedOp layout");

struct alignas(16) FusedPass {
  uint8_t L[4];        // physical bits of local positions 0..3, ascending
  uint32_t op_begin;   // index into the op array
  uint32_t op_count;
  float scale;         // exact power of two applied to every amplitude at the pass end
};
// A measure / reset instruction is a pass of its own, marked L[0] = kInstrPass:
// L[1] = physical bit of the qubit, L[2] = 1 for a reset, op_begin = index of
// its uniform and outcome (instruction ordinal plus the circuit's offset in
// the batch), op_count = 0.
constexpr uint8_t kInstrPass = 0xFF;
// A custom k-qubit unitary (2 <= k <= 5) is a pass of its own, marked
// L[0] = kWidePass: L[1] = k, op_begin = offset of its coefficients in the
// coefficient array (2^k x 2^k FP32 hi parts then lo parts, both stored
// transposed: entry (r, c) at c * 2^k + r), op_count = the physical bit of
// matrix index bit t in bits 5t..5t+4, and the scale word holds (as a uint32)
// the mask of those k physical bits.
constexpr uint8_t kWidePass = 0xFE;
constexpr int kMaxCustomQubits = 5;
static_assert(sizeof(FusedPass) == 16, "FusedPass layout");

// TEAM_PAIR runs the circuits of the warp class (n <= kWarpMaxQ) with two
// warps per circuit sharing its shared-memory slice (a launch variant of
// TEAM_WARP: twice the warps per byte of shared memory).
// TEAM_MULTI: each circuit of the global class on K co-resident CTAs (a
// cooperative launch): they share its global scratch slot and meet at a
// bounded barrier of the K after every pass; the first of the K alone writes
// the outputs with exactly the TEAM_GLOBAL output phase, so results are
// bitwise those of TEAM_GLOBAL.  Circuits without instructions or custom
// unitaries, few enough that all their CTAs are resident at once.
enum TeamKind : int32_t { TEAM_WARP = 0, TEAM_CTA = 1, TEAM_GLOBAL = 2, TEAM_PAIR = 3, TEAM_MULTI = 4 };

// Grid barrier of TEAM_MULTI: spins at most this many SM cycles (about 1 s),
// then records a time-out in FusedLaunch::err and stops waiting.
constexpr long long kGridBarrierCycles = 2000000000LL;

// Output map: logical index y of the result is physical index
// col_off ^ (XOR of col[q] over the set bits q of y), an affine map over
// GF(2): a bit permutation (SWAP factors relabel qubits) composed with the
// permutation gates (X, CNOT, SWAP) at the end of the circuit, which are not
// applied to the amplitudes but folded into this map.
struct alignas(16) FusedCirc {
  int16_t n;            // logical qubits
  int16_t nint;         // internal qubits = max(n, 4)
  int32_t pass_begin;   // index into the pass array
  int32_t pass_count;
  uint16_t col_off;     // output map: physical index of logical index 0
  uint16_t pad;
  int64_t out_off;      // amplitude offset of this circuit's outputs
  int32_t op_begin;     // the circuit's op records: [op_begin, op_begin + op_count)
  int32_t op_count;     //   (prefetched into L1 when the circuit starts)
  uint16_t col[16];     // output map: physical index bits of logical qubit q
  const float2* init;   // initial state (logical order) or nullptr for a basis state
  float out_scale;      // 1, or 2^-1/2 when an odd Hadamard factor is left over
  int32_t gen_index;    // without init: the first pass starts from |gen_index>
};
static_assert(sizeof(FusedCirc) == 80, "FusedCirc layout");

// Team limits: a warp team holds up to 2^kWarpMaxQ amplitudes in its shared
// memory slice; a CTA team up to 2^kCtaMaxQ in its CTA's shared memory; larger
// states live in global scratch (L2-resident) and are worked by a CTA.
constexpr int kWarpMaxQ = 11;
constexpr int kCtaMaxQ = 14;
constexpr int kCtaThreads = 512;
constexpr int kGlobalThreads = 512;
constexpr int kGlobalSlotQ = 16;   // log2 amplitudes per TEAM_GLOBAL scratch slot

struct FusedLaunch {
  const FusedCirc* circs;   // device
  const FusedPass* passes;  // device
  const FusedOp* ops;       // device
  const int32_t* order;     // device: circuit indices of this team kind, costliest first
  int32_t n_jobs;
  int32_t* counter;         // device: job counter, zeroed before the launch
  float2* out;              // device outputs (logical order)
  double* probs;            // nullable
  double* norms;            // nullable
  float2* gscratch;         // TEAM_GLOBAL: per-CTA state slots (2^16 amplitudes each)
  const float2* coef;       // custom unitaries: coefficient array (nullable without them)
  const double* uniforms;   // instructions: one uniform each (nullable without instructions)
  int32_t* outcomes;        // instructions: one outcome each (nullable)
  int32_t* err;             // TEAM_MULTI: set to 1 when a grid barrier timed out
  int32_t exact_probs;      // probs: 1 exact squares rounded once in FP64, 0 FP32 |psi|^2
  int32_t ctas_per_job;     // TEAM_MULTI: CTAs per circuit; job j runs on CTAs
                            // [j K, (j + 1) K), its barrier counter is counter[j],
                            // its scratch slot gscratch + j 2^kGlobalSlotQ
  int32_t team;             // TeamKind of this launch
  int32_t warps_per_cta;    // TEAM_WARP
  int32_t slice_q;          // TEAM_WARP: log2 amplitudes per warp slice; TEAM_CTA: log2 per CTA
  int32_t grid;             // CTAs
};

cudaError_t launch_fused(const FusedLaunch& L, cudaStream_t s);
int fused_max_ctas_per_sm(int team, int warps_per_cta, int slice_q);

// ---------------------------------------------------------------------------
// Plain materialised form (stages 4 and 6 of Sec. 5.3).
// ---------------------------------------------------------------------------

struct StepFactor {
  uint8_t nq;      // 1 or 2 for built-in gates; k for a custom factor
  uint8_t q0, q1;  // built-in: qubits (q0 = control for controlled gates)
  uint8_t custom;  // 1: custom k-qubit factor, entries at `coef`
  uint8_t qc[kMaxCustomQubits];  // custom: qubit of local index bit t
  uint8_t pad[7];
  const float2* coef;  // custom: 2^k x 2^k entries, row-major (device memory)
  float2 m[16];    // nq = 1: 2x2 row-major in m[0..3]; nq = 2: 4x4 row-major,
                   // local index (bit q0 << 1) | bit q1
};
static_assert(sizeof(StepFactor) == 152, "StepFactor layout");

struct StepDesc {
  int32_t f_begin;   // index into the factor array
  int32_t f_count;
  uint32_t idle;     // mask of qubits no factor touches (identity there)
  int32_t pad;
};

cudaError_t launch_materialize(const StepFactor* d_factors, StepDesc step, int n, float2* d_S,
                               cudaStream_t s);
cudaError_t launch_matvec(const float2* d_S, const float2* d_x, float2* d_y, int n,
                          cudaStream_t s);

// ---------------------------------------------------------------------------
// Circuit-unitary chain (Algorithm 1).
// ---------------------------------------------------------------------------
// Both forms compute the columns [col0, col0 + ncols) of U = S_m ... S_1 into
// d_U[r * ldu + j] = U[r][col0 + j] (the whole U: col0 = 0, ncols = ldu = 2^n).
size_t chain_tc_scratch_bytes(int n, int prec, int ncols);
// group: output-tile rows per raster band of the GEMM grid (L2 reuse).
cudaError_t chain_tc(const StepFactor* d_factors, const StepDesc* steps, int nsteps, int n,
                     int prec, int col0, int ncols, float2* d_U, int64_t ldu, void* scratch,
                     int* d_err, int group, int kchunk, int pair, cudaStream_t s);
size_t chain_simt_scratch_bytes(int n, int ncols);
cudaError_t chain_simt(const StepFactor* d_factors, const StepDesc* steps, int nsteps, int n,
                       int col0, int ncols, float2* d_U, int64_t ldu, void* scratch, cudaStream_t s);

// ---------------------------------------------------------------------------
// Probabilities / marginals (FP64).
// ---------------------------------------------------------------------------
int probs_partial_count(int n);
cudaError_t launch_probs(const float2* d_state, int n, double* d_probs, uint64_t zero_mask,
                         double* d_partials, int n_partials, double* d_sum, cudaStream_t s);

// ---------------------------------------------------------------------------
// Inverse-CDF sampling (collapse of simulateAndCollapse, Sec. 5.2).
// ---------------------------------------------------------------------------
constexpr int kSampleBlk = 256;    // probabilities per block of the cumulative sums
constexpr int kSampleChunk = 8;    // consecutive probabilities summed by one lane
__host__ __device__ inline int64_t sample_blocks(int n) {
  return n >= 8 ? (int64_t(1) << (n - 8)) : 1;
}

struct SampleSeg {
  int64_t p_off;    // offset of the segment's probabilities
  int32_t n;        // the segment holds 2^n probabilities
  int32_t blk_off;  // offset of its blocks in bsum / bpre (global path)
  int64_t index;    // position of the segment in the caller's layout (u / out)
};
static_assert(sizeof(SampleSeg) == 24, "SampleSeg layout");

// Segments with n <= kSampleSmemMaxQ can be sampled by one CTA each, with the
// probabilities staged in shared memory; larger ones take the global path
// (block tables, block prefix, one thread per shot).  Both paths compute the
// same cumulative sums in the same order, so they give identical indices.
constexpr int kSampleSmemMaxQ = 13;

struct SampleLaunch {
  const double* probs;     // device
  const SampleSeg* gsegs;  // device: segments of the global path, ascending blk_off
  int32_t n_gseg;
  int64_t nblocks;         // sum of sample_blocks(n) over the global segments
  double* bsum;            // device scratch [nblocks]: block totals
  double* bpre;            // device scratch [nblocks]: exclusive block prefix per segment
  double* cpre;            // device scratch [nblocks * 32]: chunk bases (exclusive prefix in the
                           // block, then made absolute by adding the block prefix)
  double* tot;             // device scratch [n_gseg]: segment totals
  const SampleSeg* ssegs;  // device: segments of the shared-memory path
  int32_t n_sseg;
  int32_t smem_q;          // log2 of the largest shared-memory segment
  const double* u;         // device [segments * shots] uniforms in [0, 1)
  int64_t shots;           // per segment
  int64_t* out;            // device [segments * shots] sampled indices within the segment
  int64_t probs_len;       // entries of probs the segments span (bounds checks)
  int64_t n_segs;          // segments (bounds checks: u and out hold n_segs * shots)
};

cudaError_t launch_sample(const SampleLaunch& L, cudaStream_t s);
// d_state[i] = (i == *d_index) for i < 2^n (the collapsed basis state).
cudaError_t launch_set_basis(float2* d_state, int n, const int64_t* d_index, cudaStream_t s);

// ---------------------------------------------------------------------------
// Full-state-vector backend (Appendix A, eq. 12) for states held in HBM.
// A pass keeps a tile of 2^T amplitudes in shared memory: the amplitudes
// whose indices agree outside T "tile bits" (the kFsvLowQ lowest bits, for
// coalesced loads, plus the bits the pass's gates need).  Every op of the
// pass acts on the tile; bits outside it are fixed per tile.
// ---------------------------------------------------------------------------
constexpr int kFsvTileQ = 13;
constexpr int kFsvLowQ = 5;
constexpr int kFsvThreads = 256;

constexpr int kFsvMaxFar = 18;  // bits outside the tile a pass may test (T + far <= 31)

// One pass of the full-state-vector backend.  Its gates, relabelled to tile
// qubits (the tile bits in ascending order are tile qubits 0..T-1; the far
// bits the pass tests are virtual qubits T, T+1, ...), form a small circuit
// compiled like any fused program (FusedCirc / FusedPass / FusedOp); for each
// tile the virtual qubits carry the tile's fixed global bits.
struct FsvTile {
  float2* state;    // device, 2^n amplitudes, in place
  uint64_t mask;    // tile bits
  int32_t n;        // qubits of the state
  int32_t T;        // tile bits
  int32_t nfar;     // virtual qubits
  uint8_t far[kFsvMaxFar + 1];  // global bit of virtual qubit T + v
};

// One pass over the state: L.circs points at the pass's tile program.
cudaError_t launch_fsv_tile(const FusedLaunch& L, const FsvTile& F, cudaStream_t s);

// Out-of-range accesses counted by the bounds-checked build (-DTQS_CHECKED;
// always 0 otherwise) in the kernels of one source file, optionally reset.
// Synchronous.
cudaError_t violations_fused(unsigned int* count, bool reset);
cudaError_t violations_plain(unsigned int* count, bool reset);
cudaError_t violations_probs(unsigned int* count, bool reset);
cudaError_t violations_sample(unsigned int* count, bool reset);
cudaError_t violations_chain_simt(unsigned int* count, bool reset);
cudaError_t violations_chain_tc(unsigned int* count, bool reset);

// Process-wide count of kernel launches enqueued by this library.
void count_launches(int64_t k);

// One thread waits on an mbarrier nothing completes, for at most wait_cycles;
// on time-out it sets *status = 1 and returns.
cudaError_t launch_wait_selftest(int* status, long long wait_cycles, cudaStream_t s);

// Record the calling thread's last error message (read by tqs_last_error).
void set_last_error(const char* msg);

}  // namespace tqs
