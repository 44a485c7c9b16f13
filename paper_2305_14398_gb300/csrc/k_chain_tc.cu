// Circuit-unitary chain on tcgen05 tensor cores (sm_103a).
//
// Algorithm 1: U <- S_k U for every step k after the first (U starts as S_1).
// The chain is kept transposed, V = U^T, so that V' = V S_k^T is a GEMM whose
// operands are both K-major: A = V (row-major), B = S_k (row-major), D = V'.
// The complex product uses three real GEMMs (3M):
//   T1 = Vr Sr^T, T2 = Vi Si^T, T3 = (Vr + Vi)(Sr + Si)^T,
//   Re V' = T1 - T2, Im V' = T3 - T1 - T2,
// and every real operand X is split into planes X = Xh + Xl of the MMA input
// type (BF16, or TF32 stored in FP32 words), each real GEMM being
// Xh Yh^T + Xh Yl^T + Xl Yh^T accumulated in FP32 in TMEM.
// A matrix is stored as 6 planes [Re h, Re l, Im h, Im l, Sum h, Sum l],
// each N x N row-major, read by 3-D TMA ([plane][row][k]).
//
// GEMM tile: 128 x 128 output, K step one 128-byte swizzled row (64 BF16 or
// 32 TF32), 3 stages of {A h, A l, B h, B l} (64 KiB each).  Warp 0 issues TMA, warp 1 issues the
// MMAs (one thread), warps 2-9 read the three accumulators from TMEM once per
// chunk of K (32 MMA accumulation steps by default), add the chunk's Re and Im into FP32 registers,
// and at the end write either the 6 planes of V' or, at the last step,
// U = V'^T as complex64.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "checked.h"
#include "sm100_ptx.h"
#include "step_entry.h"
#include "../../include/tqs.h"
#include "tqs_internal.h"

namespace tqs {
namespace {

using namespace ptx;

constexpr int BM = 128, BN = 128;
constexpr int kRowBytes = 128;                 // one swizzled row of K per tile row
constexpr int kStages = 3;
constexpr int kTileBytes = BM * kRowBytes;     // 16 KiB, A and B tiles alike
constexpr int kStageBytes = 4 * kTileBytes;    // A hi, A lo, B hi, B lo
constexpr int kEpiWarps = 8;                   // 2 per TMEM lane quarter, half the columns each
constexpr int kEpiCols = BN / 2;
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;  // TMA warp, MMA warp, epilogue
constexpr uint32_t kTmemCols = 512;            // 4 slots of 128 columns for 3 accumulators
constexpr size_t kGemmSmem = size_t(kStages) * kStageBytes + 1024 + 256;
constexpr int kMaxGroupM = 64;                 // tile rows per raster band at most

// Operand precision: the element type of the planes, the MMA kind, and the
// hi/lo split of an FP32 value.
template <int PREC>
struct Prec;

template <>
struct Prec<TQS_PREC_TC_BF16X3> {
  using E = __nv_bfloat16;
  static constexpr int BK = kRowBytes / 2;  // 64
  static constexpr int kDefaultKChunk = 512;  // 32 MMAs of K = 16 per chunk
  static constexpr CUtensorMapDataType kTmaType = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    mma_bf16(d, a, b, idesc_bf16_f32(BM, BN), acc);
  }
  static __device__ __forceinline__ void split(float x, E& h, E& l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
  }
};

template <>
struct Prec<TQS_PREC_TC_TF32X3> {
  using E = float;  // TF32 values (low 13 mantissa bits zero) in FP32 words
  static constexpr int BK = kRowBytes / 4;  // 32
  static constexpr int kDefaultKChunk = 256;  // 32 MMAs of K = 8 per chunk
  static constexpr CUtensorMapDataType kTmaType = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    mma_tf32(d, a, b, idesc_tf32_f32(BM, BN), acc);
  }
  static __device__ __forceinline__ void split(float x, E& h, E& l) {
    h = to_tf32(x);
    l = to_tf32(x - h);
  }
};

template <class E>
struct GemmParams {
  int N;
  int M;           // rows of V and V' (columns of the U block): a multiple of BM, <= N
  int final_step;  // 1: write the U block = V'^T (complex64); 0: the 6 planes of V'
  E* planes;       // [6][M][N] output planes (final_step == 0)
  float2* u;       // final_step == 1: U block, entry (r, j) at u[r * ldu + j], r < N, j < M
  int64_t ldu;
  int group;       // tile rows per raster band (1..kMaxGroupM)
  int kchunk_blocks;  // k blocks per accumulation chunk (>= 1)
  int* err;
};

// Split K FP32 values into hi / lo planes and store them at hp / lp (16-byte stores).
template <int PREC, int K>
__device__ __forceinline__ void store_split(const float (&v)[K], typename Prec<PREC>::E* hp,
                                            typename Prec<PREC>::E* lp) {
  using E = typename Prec<PREC>::E;
  constexpr int per16 = 16 / sizeof(E);
  static_assert(K % per16 == 0, "whole 16-byte stores");
#pragma unroll
  for (int i0 = 0; i0 < K; i0 += per16) {
    union {
      E e[per16];
      uint4 u;
    } h, l;
    if constexpr (PREC == TQS_PREC_TC_BF16X3) {
      // two values per conversion instruction (round to nearest, as split())
#pragma unroll
      for (int i = 0; i < per16; i += 2) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[i0 + i], v[i0 + i + 1]);
        const float2 hf = __bfloat1622float2(h2);
        const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[i0 + i] - hf.x, v[i0 + i + 1] - hf.y);
        h.e[i] = h2.x;
        h.e[i + 1] = h2.y;
        l.e[i] = l2.x;
        l.e[i + 1] = l2.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < per16; ++i) Prec<PREC>::split(v[i0 + i], h.e[i], l.e[i]);
    }
    *reinterpret_cast<uint4*>(hp + i0) = h.u;
    *reinterpret_cast<uint4*>(lp + i0) = l.u;
  }
}

// PAIR: the grid runs as clusters of two CTAs on the tile rows 2i and 2i + 1 of
// one tile column; they need the same B tiles, so each loads half of every B
// tile (64 rows, hi and lo) and multicasts it into both CTAs' stage, halving the
// B traffic from L2.  A stage is then released (empty barrier) only when the
// MMAs of both CTAs have consumed it: each MMA issuer's commit arrives on the
// empty barrier of both CTAs.
template <int PREC, bool PAIR>
__global__ void __launch_bounds__(kGemmThreads, 1)
    chain_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB,
                      const GemmParams<typename Prec<PREC>::E> P) {
  constexpr int BK = Prec<PREC>::BK;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tmem_full = empty + kStages;   // a chunk's three accumulators are final
  uint64_t* tmem_empty = tmem_full + 1;    // the epilogue has read a chunk's accumulators
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tmem_empty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Grouped raster: consecutive CTAs walk down a band of P.group tile rows
  // before moving right, so the CTAs resident at one time share a few A and B
  // panels in L2 instead of streaming all of B once per tile row.
  // (PAIR: the raster runs over pairs of tile rows; the cluster's two CTAs take
  // the two rows of a pair)
  const int crank = PAIR ? static_cast<int>(cluster_ctarank()) : 0;
  const int num_m = P.M / BM / (PAIR ? 2 : 1), num_n = P.N / BN;
  const int grp = PAIR ? max(1, P.group / 2) : P.group;
  const int pid = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
  const int band = pid / (grp * num_n);
  const int first_m = band * grp;
  const int gsize = min(num_m - first_m, grp);
  const int in_band = pid - band * grp * num_n;
  const int tile_m = ((first_m + in_band % gsize) * (PAIR ? 2 : 1) + crank) * BM;  // rows of V
  const int tile_n = (in_band / gsize) * BN;            // rows of S = columns of V'
  constexpr uint16_t kPairMask = 0x3;
  const int nkb = P.N / BK;                             // k blocks
  const int kc = P.kchunk_blocks;                       // k blocks per accumulation chunk
  const int nchunks = (nkb + kc - 1) / kc;
  (void)TQS_IX(tile_m, P.M - BM + 1);                   // whole tiles inside the M x N planes
  (void)TQS_IX(tile_n, P.N - BN + 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), PAIR ? 2 : 1);
    }
    mbar_init(smem_u32(tmem_full), 1);
    mbar_init(smem_u32(tmem_empty), kEpiWarps);
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  if (PAIR) cluster_sync();  // the peer's barriers exist before any multicast or commit
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  // Order of the (k block, real GEMM j) pairs, the same for the producer and
  // the MMA issuer: chunk by chunk, and inside a chunk all k blocks of GEMM 0,
  // then of GEMM 1, then of GEMM 2.  Chunk c accumulates GEMM j in TMEM slot
  // (3c + j) mod 4 (4 slots of 128 columns), so the next chunk's GEMM 0 runs
  // in the slot its predecessor left free while the epilogue reads this one.
  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tmA);
      prefetch_tmap(&tmB);
      int it = 0;
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int kb0 = c * kc, kb1 = min(nkb, kb0 + kc);
        for (int j = 0; j < 3 && ok; ++j) {
          for (int kb = kb0; kb < kb1; ++kb, ++it) {
            const int s = it % kStages;
            const uint32_t ph = (it / kStages) & 1;
            if (it >= kStages && !mbar_wait(smem_u32(&empty[s]), ph ^ 1, P.err)) {
              ok = false;
              break;
            }
            const uint32_t st = smem_u32(stages + s * kStageBytes);
            const uint32_t fb = smem_u32(&full[s]);
            mbar_arrive_expect_tx(fb, kStageBytes);
            tma_load_3d(st, &tmA, kb * BK, tile_m, 2 * j, fb);
            tma_load_3d(st + kTileBytes, &tmA, kb * BK, tile_m, 2 * j + 1, fb);
            if (PAIR) {  // this CTA's half of the B tile (64 rows), into both CTAs
              const uint32_t half = static_cast<uint32_t>(crank) * (kTileBytes / 2);
              tma_load_3d_mc(st + 2 * kTileBytes + half, &tmB, kb * BK, tile_n + crank * (BN / 2), 2 * j,
                             fb, kPairMask);
              tma_load_3d_mc(st + 3 * kTileBytes + half, &tmB, kb * BK, tile_n + crank * (BN / 2),
                             2 * j + 1, fb, kPairMask);
            } else {
              tma_load_3d(st + 2 * kTileBytes, &tmB, kb * BK, tile_n, 2 * j, fb);
              tma_load_3d(st + 3 * kTileBytes, &tmB, kb * BK, tile_n, 2 * j + 1, fb);
            }
          }
        }
      }
      // Wait (bounded) for this thread's last copies so that none is in
      // flight when the CTA exits, whatever happened downstream.
      for (int i = (it > kStages ? it - kStages : 0); i < it; ++i)
        mbar_wait(smem_u32(&full[i % kStages]), (i / kStages) & 1, P.err);
      // PAIR: and for both MMA issuers' last releases, the arrivals that the
      // peer sends to this CTA's barriers (none may come after the exit)
      if (PAIR)
        for (int i = (it > kStages ? it - kStages : 0); i < it; ++i)
          mbar_wait(smem_u32(&empty[i % kStages]), (i / kStages) & 1, P.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, drained = 0;  // chunks the epilogue is known to have read
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int kb0 = c * kc, kb1 = min(nkb, kb0 + kc);
        for (int j = 0; j < 3 && ok; ++j) {
          // the slot's previous chunk (c - 2 for GEMM 0, c - 1 otherwise) must be read
          const int need = j == 0 ? c - 1 : c;
          while (drained < need) {
            if (!mbar_wait(smem_u32(tmem_empty), drained & 1, P.err)) {
              ok = false;
              break;
            }
            ++drained;
          }
          if (!ok) break;
          tc_fence_after();
          const uint32_t d = tmem_base + static_cast<uint32_t>(((3 * c + j) & 3) * BN);
          for (int kb = kb0; kb < kb1; ++kb, ++it) {
            const int s = it % kStages;
            const uint32_t ph = (it / kStages) & 1;
            if (!mbar_wait(smem_u32(&full[s]), ph, P.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_hi = smem_u32(stages + s * kStageBytes);
            const uint32_t a_lo = a_hi + kTileBytes;
            const uint32_t b_hi = a_hi + 2 * kTileBytes;
            const uint32_t b_lo = a_hi + 3 * kTileBytes;
#pragma unroll
            for (int ks = 0; ks < kRowBytes / 32; ++ks) {
              const uint32_t off = ks * 32;  // one MMA's K (32 bytes) inside the swizzled row
              const uint32_t acc = (kb > kb0 || ks > 0) ? 1u : 0u;
              Prec<PREC>::mma(d, sw128_kmajor_desc(a_hi + off), sw128_kmajor_desc(b_hi + off), acc);
              Prec<PREC>::mma(d, sw128_kmajor_desc(a_hi + off), sw128_kmajor_desc(b_lo + off), 1u);
              Prec<PREC>::mma(d, sw128_kmajor_desc(a_lo + off), sw128_kmajor_desc(b_hi + off), 1u);
            }
            // the stage is free once these MMAs finish (PAIR: in both CTAs)
            if (PAIR) mma_commit_mc(smem_u32(&empty[s]), kPairMask);
            else mma_commit(smem_u32(&empty[s]));
          }
        }
        if (ok) mma_commit(smem_u32(tmem_full));  // this chunk's accumulators are final
      }
    }
  } else {
    // Epilogue: 8 warps; warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows)
    // and half h of the columns.  Each chunk's Re = T1 - T2 and Im = T3 - T1 -
    // T2 are added into FP32 registers (round to nearest): the tensor cores
    // accumulate in FP32 with truncation, so a sum over K has a systematic
    // shrink proportional to the number of accumulation steps, which chunking
    // bounds by the chunk length.
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const uint32_t tl = tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                        static_cast<uint32_t>(h * kEpiCols);
    float re[kEpiCols], im[kEpiCols];
#pragma unroll
    for (int i = 0; i < kEpiCols; ++i) re[i] = im[i] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      if (!mbar_wait(smem_u32(tmem_full), c & 1, P.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t s1 = tl + static_cast<uint32_t>(((3 * c + 0) & 3) * BN);
      const uint32_t s2 = tl + static_cast<uint32_t>(((3 * c + 1) & 3) * BN);
      const uint32_t s3 = tl + static_cast<uint32_t>(((3 * c + 2) & 3) * BN);
#pragma unroll
      for (int g = 0; g < kEpiCols / 8; ++g) {
        float t1[8], t2[8], t3[8];
        tmem_ld8(s1 + g * 8, t1);
        tmem_ld8(s2 + g * 8, t2);
        tmem_ld8(s3 + g * 8, t3);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          re[g * 8 + i] += t1[i] - t2[i];
          im[g * 8 + i] += t3[i] - t1[i] - t2[i];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(tmem_empty));
    }
    if (ok) {
      const int gm = tile_m + row;
      const int col0 = tile_n + h * kEpiCols;
      if (P.final_step) {
        // U[n][m] = V'[m][n]: lanes hold consecutive m, so each store is coalesced.
        const size_t ulen = static_cast<size_t>(P.N - 1) * static_cast<size_t>(P.ldu) + P.M;
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i)
          P.u[TQS_IX(static_cast<size_t>(col0 + i) * static_cast<size_t>(P.ldu) + gm, ulen)] =
              make_float2(re[i], im[i]);
      } else {
        const size_t PS = static_cast<size_t>(P.M) * P.N;  // plane stride
        typename Prec<PREC>::E* rowp = P.planes + static_cast<size_t>(TQS_IX(gm, P.M)) * P.N +
                                       TQS_IX(col0, P.N - kEpiCols + 1);
#pragma unroll
        for (int i0 = 0; i0 < kEpiCols; i0 += 16) {
          float a[16], b[16], sm[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            a[i] = re[i0 + i];
            b[i] = im[i0 + i];
            sm[i] = a[i] + b[i];
          }
          store_split<PREC, 16>(a, rowp + i0, rowp + PS + i0);
          store_split<PREC, 16>(b, rowp + 2 * PS + i0, rowp + 3 * PS + i0);
          store_split<PREC, 16>(sm, rowp + 4 * PS + i0, rowp + 5 * PS + i0);
        }
      }
    }
  }
  tc_fence_before();
  if (PAIR) cluster_sync();  // neither CTA exits while the other may still signal it
  else __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

// Operand planes of a step unitary: for each entry, Re, Im and Re + Im, each
// split into hi + lo of the MMA input type.  transpose = 0: plane[r][c] =
// S[r][c] (the B operand, rows = N, row0 = 0); transpose = 1: plane[j][r] =
// S[r][row0 + j] for j < rows (rows row0.. of the initial V = S_1^T: the
// columns row0.. of S_1).  Planes are rows x N, `rows * N` entries apart.
//
// A thread writes 8 consecutive entries of one output row (a warp 256, so
// each store instruction of a warp covers 512 contiguous bytes of a BF16
// plane).  One index of S (the fixed one) is the same for all of them; the
// other runs over values whose low 5 bits take 8 of 32 values.  An entry is
// the product of the step's factor entries (Algorithm 2), and the factors are
// disjoint, so:
//   * factors on no qubit below 5 give one value per group of 32 entries;
//   * factors on qubits below 5 only give a 32-entry table over the low bits,
//     the same for every group of a row: when a warp's 256 entries lie in one
//     row (rows of at least 256 entries) lane v computes entry v of the table
//     and the others read it by shuffle;
//   * factors on qubits on both sides are evaluated per entry.
constexpr int kGenThreads = 256;
constexpr int kGenChunksPerThread = 8;
constexpr int kMaxFactors = 16;

// At most 40 registers (6 CTAs' worth per SM): a generator CTA then fits
// beside a GEMM CTA (320 threads x 168 registers) on one SM.
template <int PREC>
__global__ void __launch_bounds__(kGenThreads, 6)
    gen_planes_kernel(const StepFactor* __restrict__ factors, int nf, uint32_t idle, int n,
                      int transpose, int row0, int rows, typename Prec<PREC>::E* __restrict__ planes) {
  __shared__ StepFactor fs[kMaxFactors];
  __shared__ int s_cls[3][kMaxFactors];  // factor indices: high, low-only, mixed
  __shared__ int s_n[3];
  for (int i = threadIdx.x; i < nf * static_cast<int>(sizeof(StepFactor) / 8); i += blockDim.x)
    reinterpret_cast<float2*>(fs)[TQS_IX(i, int(sizeof(fs) / 8))] =
        reinterpret_cast<const float2*>(factors)[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    int cnt[3] = {0, 0, 0};
    for (int k = 0; k < nf; ++k) {
      const uint32_t qm = factor_qubits(fs[k]);
      const int cls = (qm & 31u) == 0 ? 0 : (qm & ~31u) == 0 ? 1 : 2;
      s_cls[cls][TQS_IX(cnt[cls]++, kMaxFactors)] = k;
    }
    for (int c = 0; c < 3; ++c) s_n[c] = cnt[c];
  }
  __syncthreads();
  const int nhi = s_n[0], nlo = s_n[1], nmix = s_n[2];
  const int lane = threadIdx.x & 31;
  const int64_t N = int64_t(1) << n;
  const size_t PS = static_cast<size_t>(rows) * N;  // plane stride
  const int64_t chunks = static_cast<int64_t>(PS) >> 3;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const uint32_t idle_lo = idle & 31u;
  // chunks is a multiple of 32 and a warp's threads take 32 consecutive
  // chunks, so whole warps run every iteration (the shuffles below)
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < chunks; e += stride) {
    const int64_t flat = e << 3;
    const uint32_t fixed = static_cast<uint32_t>(flat >> n) + static_cast<uint32_t>(row0);
    const uint32_t col = static_cast<uint32_t>(flat & (N - 1));
    const uint32_t fixed_lo = fixed & 31u;
    const bool shared_row = __all_sync(0xffffffffu, fixed == __shfl_sync(0xffffffffu, fixed, 0));
    // group of 32 entries this thread writes into, and the one whose common
    // value (the factors on qubits >= 5) this lane computes for the warp
    const uint32_t vary0 = col & ~31u;
    const uint32_t gvary = shared_row ? (__shfl_sync(0xffffffffu, col, 0) & ~31u) + 32u * (lane & 7) : vary0;
    float2 gbase = make_float2(0.f, 0.f);
    {
      const uint32_t r0 = transpose ? gvary : fixed, c0 = transpose ? fixed : gvary;
      if (((r0 ^ c0) & idle & ~31u) == 0) {
        gbase = make_float2(1.f, 0.f);
        for (int k = 0; k < nhi; ++k) gbase = step_cmul(gbase, factor_entry(fs[s_cls[0][k]], r0, c0));
      }
    }
    // entry `lane` of the low-bit table of the warp's row
    const uint32_t lv = static_cast<uint32_t>(lane);
    float2 tab = ((lv ^ fixed_lo) & idle_lo) ? make_float2(0.f, 0.f) : make_float2(1.f, 0.f);
    {
      const uint32_t r = transpose ? vary0 | lv : fixed, c = transpose ? fixed : vary0 | lv;
      for (int k = 0; k < nlo; ++k) tab = step_cmul(tab, factor_entry(fs[s_cls[1][k]], r, c));
    }
    float2 base = gbase;
    if (shared_row) {
      const int src = static_cast<int>((col - (__shfl_sync(0xffffffffu, col, 0) & ~31u)) >> 5);
      base = make_float2(__shfl_sync(0xffffffffu, gbase.x, src), __shfl_sync(0xffffffffu, gbase.y, src));
    }
    float re[8], im[8], sm[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t v = (col & 31u) + static_cast<uint32_t>(i);
      const uint32_t r = transpose ? vary0 | v : fixed;
      const uint32_t c = transpose ? fixed : vary0 | v;
      float2 z;
      if (shared_row) {
        z = make_float2(__shfl_sync(0xffffffffu, tab.x, static_cast<int>(v)),
                        __shfl_sync(0xffffffffu, tab.y, static_cast<int>(v)));
        z = step_cmul(base, z);
      } else {
        z = ((v ^ fixed_lo) & idle_lo) ? make_float2(0.f, 0.f) : base;
        for (int k = 0; k < nlo; ++k) z = step_cmul(z, factor_entry(fs[s_cls[1][k]], r, c));
      }
      for (int k = 0; k < nmix; ++k) z = step_cmul(z, factor_entry(fs[s_cls[2][k]], r, c));
      re[i] = z.x;
      im[i] = z.y;
      sm[i] = z.x + z.y;
    }
    typename Prec<PREC>::E* base_p = planes + TQS_IX(static_cast<size_t>(flat), PS - 7);
    store_split<PREC, 8>(re, base_p, base_p + PS);
    store_split<PREC, 8>(im, base_p + 2 * PS, base_p + 3 * PS);
    store_split<PREC, 8>(sm, base_p + 4 * PS, base_p + 5 * PS);
  }
}

// ------------------------------------------------------------ tensor maps

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// [6][rows][N] planes as a 3-D tensor {k, row, plane}, box {one 128-byte row,
// 128 rows, 1 plane}, 128-byte swizzle.
template <int PREC>
bool make_planes_map(CUtensorMap* m, void* base, int N, int rows, int box_rows = BM) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t es = sizeof(typename Prec<PREC>::E);
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(rows), 6};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(N) * es,
                                 static_cast<cuuint64_t>(rows) * N * es};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(Prec<PREC>::BK), static_cast<cuuint32_t>(box_rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, Prec<PREC>::kTmaType, 3, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int PREC>
cudaError_t launch_gen(const StepFactor* d_factors, const StepDesc& st, int n, int transpose,
                       int row0, int rows, typename Prec<PREC>::E* planes, cudaStream_t s) {
  if (st.f_count > kMaxFactors) return cudaErrorInvalidValue;
  const int64_t N = int64_t(1) << n;
  const int64_t per_block = int64_t(kGenThreads) * kGenChunksPerThread * 8;
  int64_t blocks = (int64_t(rows) * N + per_block - 1) / per_block;
  if (blocks > (int64_t(1) << 30)) blocks = int64_t(1) << 30;
  if (blocks < 1) blocks = 1;
  gen_planes_kernel<PREC><<<static_cast<int>(blocks), kGenThreads, 0, s>>>(
      d_factors + st.f_begin, st.f_count, st.idle, n, transpose, row0, rows, planes);
  count_launches(1);
  return cudaGetLastError();
}

// The chain's two internal streams: the GEMMs on the device's highest stream
// priority, the plane generators on its lowest, so that while the GEMM of step
// k runs the generator of step k + 1 fills the room its CTAs leave (one GEMM
// CTA per SM uses 198 KB of shared memory and 48 K registers) and the block
// scheduler prefers the GEMM's CTAs whenever both wait.  Created once per
// device; calls on the caller's stream are ordered against them with events.
struct ChainStreams {
  cudaStream_t gemm = nullptr, gen = nullptr;
};

cudaError_t chain_streams(ChainStreams* out) {
  static std::mutex mu;
  static ChainStreams per_dev[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  ChainStreams& cs = per_dev[dev];
  if (!cs.gemm) {
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) return e;
    cudaStream_t a = nullptr, b = nullptr;
    e = cudaStreamCreateWithPriority(&a, cudaStreamNonBlocking, greatest);
    if (e != cudaSuccess) return e;
    e = cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, least);
    if (e != cudaSuccess) {
      cudaStreamDestroy(a);
      return e;
    }
    cs.gemm = a;
    cs.gen = b;
  }
  *out = cs;
  return cudaSuccess;
}

// Events of one chain call (destroyed on every return path).
struct ChainEvents {
  cudaEvent_t start = nullptr, gen_done[2] = {nullptr, nullptr}, gemm_done[2] = {nullptr, nullptr},
              end = nullptr, end_gen = nullptr;
  cudaError_t create() {
    cudaEvent_t* all[] = {&start, &gen_done[0], &gen_done[1], &gemm_done[0], &gemm_done[1], &end,
                          &end_gen};
    for (cudaEvent_t* p : all) {
      const cudaError_t e = cudaEventCreateWithFlags(p, cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  ~ChainEvents() {
    cudaEvent_t all[] = {start, gen_done[0], gen_done[1], gemm_done[0], gemm_done[1], end, end_gen};
    for (cudaEvent_t e : all)
      if (e) cudaEventDestroy(e);
  }
};

// One GEMM launch: plain, or (pair) as clusters of two CTAs sharing B tiles.
template <int PREC>
cudaError_t launch_gemm(bool pair, int grid, const CUtensorMap& mA, const CUtensorMap& mB,
                        const GemmParams<typename Prec<PREC>::E>& P, cudaStream_t s) {
  if (!pair) {
    chain_gemm_kernel<PREC, false><<<grid, kGemmThreads, kGemmSmem, s>>>(mA, mB, P);
    count_launches(1);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kGemmThreads);
  cfg.dynamicSmemBytes = kGemmSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, chain_gemm_kernel<PREC, true>, mA, mB, P);
  count_launches(1);
  return e;
}

template <int PREC>
cudaError_t chain_tc_impl(const StepFactor* d_factors, const StepDesc* steps, int nsteps, int n,
                          int col0, int ncols, float2* d_U, int64_t ldu, void* scratch, int* d_err,
                          int group, int kchunk, int pair_opt, cudaStream_t s) {
  using E = typename Prec<PREC>::E;
  const int N = 1 << n;
  const size_t MN = size_t(ncols) * N;  // the block's V planes: ncols rows of V
  const size_t NN = size_t(N) * N;
  E* V0 = static_cast<E*>(scratch);
  E* V1 = V0 + 6 * MN;
  E* S[2] = {V1 + 6 * MN, V1 + 6 * MN + 6 * NN};  // S_k in S[(k - 1) & 1]
  // cluster pairs need an even number of tile rows
  const bool pair = pair_opt != 0 && (ncols / BM) % 2 == 0;
  CUtensorMap mV0, mV1, mS[2];
  const int b_rows = pair ? BN / 2 : BN;  // B box: a CTA's half of the tile when paired
  if (!make_planes_map<PREC>(&mV0, V0, N, ncols) || !make_planes_map<PREC>(&mV1, V1, N, ncols) ||
      !make_planes_map<PREC>(&mS[0], S[0], N, N, b_rows) || !make_planes_map<PREC>(&mS[1], S[1], N, N, b_rows))
    return cudaErrorNotSupported;
  cudaError_t e = pair ? cudaFuncSetAttribute(chain_gemm_kernel<PREC, true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(kGemmSmem))
                       : cudaFuncSetAttribute(chain_gemm_kernel<PREC, false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(kGemmSmem));
  if (e != cudaSuccess) return e;
  ChainStreams cs;
  if ((e = chain_streams(&cs)) != cudaSuccess) return e;
  ChainEvents ev;
  if ((e = ev.create()) != cudaSuccess) return e;
  // fork: both internal streams start after the work already on the caller's stream
  if ((e = cudaEventRecord(ev.start, s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(cs.gemm, ev.start, 0)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(cs.gen, ev.start, 0)) != cudaSuccess) return e;
  auto steps_loop = [&]() -> cudaError_t {
    // V = rows col0.. of S_1^T
    cudaError_t r = launch_gen<PREC>(d_factors, steps[0], n, 1, col0, ncols, V0, cs.gemm);
    if (r != cudaSuccess) return r;
    if ((r = launch_gen<PREC>(d_factors, steps[1], n, 0, 0, N, S[0], cs.gen)) != cudaSuccess) return r;
    if ((r = cudaEventRecord(ev.gen_done[0], cs.gen)) != cudaSuccess) return r;
    bool cur0 = true;
    for (int k = 1; k < nsteps; ++k) {
      const int b = (k - 1) & 1;  // S_k's buffer
      // S_{k+1} into the other buffer, once the GEMM of step k - 1 (its last reader) is done
      if (k + 1 < nsteps) {
        if (k >= 2 && (r = cudaStreamWaitEvent(cs.gen, ev.gemm_done[b ^ 1], 0)) != cudaSuccess) return r;
        if ((r = launch_gen<PREC>(d_factors, steps[k + 1], n, 0, 0, N, S[b ^ 1], cs.gen)) != cudaSuccess)
          return r;
        if ((r = cudaEventRecord(ev.gen_done[b ^ 1], cs.gen)) != cudaSuccess) return r;
      }
      if ((r = cudaStreamWaitEvent(cs.gemm, ev.gen_done[b], 0)) != cudaSuccess) return r;
      GemmParams<E> P;
      P.N = N;
      P.M = ncols;
      P.final_step = (k == nsteps - 1) ? 1 : 0;
      P.planes = cur0 ? V1 : V0;
      P.u = d_U;
      P.ldu = ldu;
      P.group = group;
      // K per accumulation chunk in whole k blocks (0: the precision's default,
      // the same number of MMA accumulation steps per chunk for both)
      P.kchunk_blocks = std::max(1, (kchunk > 0 ? kchunk : Prec<PREC>::kDefaultKChunk) / Prec<PREC>::BK);
      P.err = d_err;
      const int grid = (N / BN) * (ncols / BM);
      if ((r = launch_gemm<PREC>(pair, grid, cur0 ? mV0 : mV1, mS[b], P, cs.gemm)) != cudaSuccess) return r;
      if ((r = cudaEventRecord(ev.gemm_done[b], cs.gemm)) != cudaSuccess) return r;
      cur0 = !cur0;
    }
    return cudaSuccess;
  };
  const cudaError_t le = steps_loop();
  // join, on every path: the caller's stream continues after all work of both
  // internal streams (normally every generator has finished before the GEMM
  // that reads its planes, but not after an error in mid-chain)
  if ((e = cudaEventRecord(ev.end, cs.gemm)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(ev.end_gen, cs.gen)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(s, ev.end, 0)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(s, ev.end_gen, 0)) != cudaSuccess) return e;
  return le;
}

__global__ void wait_selftest_kernel(int* status, long long wait_cycles) {
  __shared__ uint64_t bar;
  mbar_init(smem_u32(&bar), 1);
  fence_barrier_init();
  const uint32_t b = smem_u32(&bar);
  if (mbar_try_wait(b, 0)) return;  // nothing arrives: never taken
  const long long t0 = clock64();
  while (!mbar_try_wait(b, 0)) {
    if (clock64() - t0 > wait_cycles) {
      atomicExch(status, 1);
      return;
    }
  }
}

}  // namespace

TQS_DEFINE_VIOLATIONS(violations_chain_tc)

cudaError_t launch_wait_selftest(int* status, long long wait_cycles, cudaStream_t s) {
  wait_selftest_kernel<<<1, 1, 0, s>>>(status, wait_cycles);
  count_launches(1);
  return cudaGetLastError();
}

size_t chain_tc_scratch_bytes(int n, int prec, int ncols) {
  const size_t N = size_t(1) << n;
  const size_t es = prec == TQS_PREC_TC_TF32X3 ? 4 : 2;
  // V and V' (ncols rows) and two step unitaries S (double-buffered): 6 planes each
  return (12 * size_t(ncols) * N + 12 * N * N) * es;
}

// Columns [col0, col0 + ncols) of U = S_m ... S_1 with the tensor-core chain
// in precision `prec` (TQS_PREC_TC_BF16X3 or TQS_PREC_TC_TF32X3): the rows
// col0.. of V = U^T, each step V <- V S_k^T, written as U[r][col0 + j] at
// d_U[r * ldu + j].  n >= 7; col0 and ncols multiples of 128.
cudaError_t chain_tc(const StepFactor* d_factors, const StepDesc* steps, int nsteps, int n,
                     int prec, int col0, int ncols, float2* d_U, int64_t ldu, void* scratch,
                     int* d_err, int group, int kchunk, int pair, cudaStream_t s) {
  if (n < 7 || nsteps < 2 || col0 % BM || ncols % BM || ncols < BM || col0 + ncols > (1 << n) ||
      ldu < ncols || group < 1 || group > kMaxGroupM || kchunk < 0 || kchunk % 64)
    return cudaErrorInvalidValue;
  if (prec == TQS_PREC_TC_BF16X3)
    return chain_tc_impl<TQS_PREC_TC_BF16X3>(d_factors, steps, nsteps, n, col0, ncols, d_U, ldu,
                                             scratch, d_err, group, kchunk, pair, s);
  if (prec == TQS_PREC_TC_TF32X3)
    return chain_tc_impl<TQS_PREC_TC_TF32X3>(d_factors, steps, nsteps, n, col0, ncols, d_U, ldu,
                                             scratch, d_err, group, kchunk, pair, s);
  return cudaErrorInvalidValue;
}

}  // namespace tqs
