// Circuit-unitary chain on tcgen05 tensor cores (sm_103a).
//
// Algorithm 1: U <- S_k U for every step k after the first (U starts as S_1).
// The chain is kept transposed, V = U^T, so that V' = V S_k^T is a GEMM whose
// operands are both K-major: A = V (row-major), B = S_k (row-major), D = V'.
// The complex product uses three real GEMMs (3M):
//   T1 = Vr Sr^T, T2 = Vi Si^T, T3 = (Vr + Vi)(Sr + Si)^T,
//   Re V' = T1 - T2, Im V' = T3 - T1 - T2,
// and every real operand X is split into BF16 planes X = Xh + Xl, each real
// GEMM being Xh Yh^T + Xh Yl^T + Xl Yh^T accumulated in FP32 in TMEM.
// A matrix is stored as 6 BF16 planes [Re h, Re l, Im h, Im l, Sum h, Sum l],
// each N x N row-major, read by 3-D TMA ([plane][row][k]).
//
// GEMM tile: 128 x 128 output, K step 64 (one 128-byte swizzled row), 3 stages
// of {A h, A l, B h, B l} (64 KiB each).  Warp 0 issues TMA, warp 1 issues the
// MMAs (one thread), warps 2-5 read the three accumulators from TMEM and write
// either the 6 planes of V' or, at the last step, U = V'^T as complex64.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "sm100_ptx.h"
#include "step_entry.h"
#include "tqs_internal.h"

namespace tqs {
namespace {

using namespace ptx;

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int kStages = 3;
constexpr int kTileBytes = BM * BK * 2;        // 16 KiB, A and B tiles alike
constexpr int kStageBytes = 4 * kTileBytes;    // A hi, A lo, B hi, B lo
constexpr int kGemmThreads = 192;
constexpr uint32_t kTmemCols = 512;            // 3 accumulators x 128 columns
constexpr size_t kGemmSmem = size_t(kStages) * kStageBytes + 1024 + 256;
constexpr int kGroupM = 16;                    // tile rows per raster band

struct GemmParams {
  int N;
  int final_step;            // 1: write U = V'^T (complex64); 0: the 6 planes of V'
  __nv_bfloat16* planes;     // [6][N][N] output planes (final_step == 0)
  float2* u;                 // [N][N] output (final_step == 1)
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(lo)) |
         (static_cast<uint32_t>(__bfloat16_as_ushort(hi)) << 16);
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    chain_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const GemmParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tmem_full = empty + kStages;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tmem_full + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Grouped raster: consecutive CTAs walk down a band of kGroupM tile rows
  // before moving right, so the CTAs resident at one time share a few A and B
  // panels in L2 instead of streaming all of B once per tile row.
  const int num_m = P.N / BM, num_n = P.N / BN;
  const int pid = blockIdx.x;
  const int band = pid / (kGroupM * num_n);
  const int first_m = band * kGroupM;
  const int gsize = min(num_m - first_m, kGroupM);
  const int in_band = pid - band * kGroupM * num_n;
  const int tile_m = (first_m + in_band % gsize) * BM;  // rows of V = rows of V'
  const int tile_n = (in_band / gsize) * BN;            // rows of S = columns of V'
  const int iters = (P.N / BK) * 3;                     // (k block, real GEMM j) pairs

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(tmem_full), 1);
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tmA);
      prefetch_tmap(&tmB);
      int issued = 0;
      for (int it = 0; it < iters; ++it) {
        const int s = it % kStages;
        const uint32_t ph = (it / kStages) & 1;
        if (it >= kStages && !mbar_wait(smem_u32(&empty[s]), ph ^ 1, P.err)) break;
        const int kb = it / 3, j = it % 3;
        const uint32_t st = smem_u32(stages + s * kStageBytes);
        const uint32_t fb = smem_u32(&full[s]);
        mbar_arrive_expect_tx(fb, kStageBytes);
        tma_load_3d(st, &tmA, kb * BK, tile_m, 2 * j, fb);
        tma_load_3d(st + kTileBytes, &tmA, kb * BK, tile_m, 2 * j + 1, fb);
        tma_load_3d(st + 2 * kTileBytes, &tmB, kb * BK, tile_n, 2 * j, fb);
        tma_load_3d(st + 3 * kTileBytes, &tmB, kb * BK, tile_n, 2 * j + 1, fb);
        issued = it + 1;
      }
      // Wait (bounded) for this thread's last copies so that none is in
      // flight when the CTA exits, whatever happened downstream.
      for (int it = (issued > kStages ? issued - kStages : 0); it < issued; ++it)
        mbar_wait(smem_u32(&full[it % kStages]), (it / kStages) & 1, P.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(BM, BN);
      for (int it = 0; it < iters; ++it) {
        const int s = it % kStages;
        const uint32_t ph = (it / kStages) & 1;
        if (!mbar_wait(smem_u32(&full[s]), ph, P.err)) break;
        tc_fence_after();
        const int kb = it / 3, j = it % 3;
        const uint32_t d = tmem_base + static_cast<uint32_t>(j * BN);
        const uint32_t a_hi = smem_u32(stages + s * kStageBytes);
        const uint32_t a_lo = a_hi + kTileBytes;
        const uint32_t b_hi = a_hi + 2 * kTileBytes;
        const uint32_t b_lo = a_hi + 3 * kTileBytes;
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint32_t off = ks * 32;  // 16 BF16 along K inside the swizzled row
          const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
          mma_bf16(d, sw128_kmajor_desc(a_hi + off), sw128_kmajor_desc(b_hi + off), idesc, acc);
          mma_bf16(d, sw128_kmajor_desc(a_hi + off), sw128_kmajor_desc(b_lo + off), idesc, 1u);
          mma_bf16(d, sw128_kmajor_desc(a_lo + off), sw128_kmajor_desc(b_hi + off), idesc, 1u);
        }
        mma_commit(smem_u32(&empty[s]));  // the stage is free once these MMAs finish
      }
      mma_commit(smem_u32(tmem_full));  // all accumulators final
    }
  } else {
    // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 = tile rows.
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const bool ok = mbar_wait(smem_u32(tmem_full), 0, P.err);
    tc_fence_after();
    if (ok) {
      const uint32_t tl = tmem_base + (static_cast<uint32_t>(q * 32) << 16);
      const int gm = tile_m + row;
      const size_t NN = static_cast<size_t>(P.N) * P.N;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float t1[32], t2[32], t3[32];
        tmem_ld32(tl + 0 * BN + c0, t1);
        tmem_ld32(tl + 1 * BN + c0, t2);
        tmem_ld32(tl + 2 * BN + c0, t3);
        tmem_wait_ld();
        if (P.final_step) {
          // U[n][m] = V'[m][n]: lanes hold consecutive m, so each store is coalesced.
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float re = t1[i] - t2[i];
            const float im = t3[i] - t1[i] - t2[i];
            P.u[static_cast<size_t>(tile_n + c0 + i) * P.N + gm] = make_float2(re, im);
          }
        } else {
          __nv_bfloat16* rowp = P.planes + static_cast<size_t>(gm) * P.N + tile_n + c0;
#pragma unroll
          for (int i0 = 0; i0 < 32; i0 += 8) {
            uint32_t w[6][4];
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
              float v[3][2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float a = t1[i0 + i + h], b = t2[i0 + i + h], c = t3[i0 + i + h];
                v[0][h] = a - b;          // Re
                v[1][h] = c - a - b;      // Im
                v[2][h] = v[0][h] + v[1][h];
              }
#pragma unroll
              for (int comp = 0; comp < 3; ++comp) {
                const __nv_bfloat16 h0 = __float2bfloat16_rn(v[comp][0]);
                const __nv_bfloat16 h1 = __float2bfloat16_rn(v[comp][1]);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(v[comp][0] - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(v[comp][1] - __bfloat162float(h1));
                w[2 * comp][i / 2] = pack_bf16x2(h0, h1);
                w[2 * comp + 1][i / 2] = pack_bf16x2(l0, l1);
              }
            }
#pragma unroll
            for (int p = 0; p < 6; ++p)
              *reinterpret_cast<uint4*>(rowp + p * NN + i0) =
                  make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

// Operand planes of a step unitary: for each entry, Re, Im and Re + Im, each
// split into BF16 hi + lo.  transpose = 0: plane[r][c] = S[r][c] (the B
// operand); transpose = 1: plane[c][r] = S[r][c] (the initial V = S_1^T).
// A thread produces 8 consecutive entries of one output row.
constexpr int kGenThreads = 256;
constexpr int kMaxFactors = 16;

__global__ void __launch_bounds__(kGenThreads)
    gen_planes_kernel(const StepFactor* __restrict__ factors, int nf, uint32_t idle, int n,
                      int transpose, __nv_bfloat16* __restrict__ planes) {
  __shared__ StepFactor fs[kMaxFactors];
  for (int i = threadIdx.x; i < nf * static_cast<int>(sizeof(StepFactor) / 8); i += blockDim.x)
    reinterpret_cast<float2*>(fs)[i] = reinterpret_cast<const float2*>(factors)[i];
  __syncthreads();
  const int64_t N = int64_t(1) << n;
  const size_t NN = static_cast<size_t>(N) * N;
  const int64_t chunks = (N * N) >> 3;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < chunks; e += stride) {
    const int64_t flat = e << 3;
    const uint32_t orow = static_cast<uint32_t>(flat >> n);
    const uint32_t ocol = static_cast<uint32_t>(flat & (N - 1));
    uint32_t w[6][4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      float v[3][2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t r = transpose ? ocol + i + h : orow;
        const uint32_t c = transpose ? orow : ocol + i + h;
        const float2 z = step_entry(fs, nf, idle, r, c);
        v[0][h] = z.x;
        v[1][h] = z.y;
        v[2][h] = z.x + z.y;
      }
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[comp][0]);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(v[comp][1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[comp][0] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[comp][1] - __bfloat162float(h1));
        w[2 * comp][i / 2] = pack_bf16x2(h0, h1);
        w[2 * comp + 1][i / 2] = pack_bf16x2(l0, l1);
      }
    }
#pragma unroll
    for (int p = 0; p < 6; ++p)
      *reinterpret_cast<uint4*>(planes + p * NN + flat) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
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

// [6][N][N] BF16 planes as a 3-D tensor {k, row, plane}, box {64, 128, 1},
// 128-byte swizzle.
bool make_planes_map(CUtensorMap* m, void* base, int N) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(N), 6};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(N) * 2,
                                 static_cast<cuuint64_t>(N) * N * 2};
  const cuuint32_t box[3] = {BK, BM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sms() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
  }
  return v;
}

cudaError_t launch_gen(const StepFactor* d_factors, const StepDesc& st, int n, int transpose,
                       __nv_bfloat16* planes, cudaStream_t s) {
  if (st.f_count > kMaxFactors) return cudaErrorInvalidValue;
  const int64_t N = int64_t(1) << n;
  int64_t blocks = ((N * N) / 8 + kGenThreads - 1) / kGenThreads;
  const int64_t cap = int64_t(sms()) * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  gen_planes_kernel<<<static_cast<int>(blocks), kGenThreads, 0, s>>>(
      d_factors + st.f_begin, st.f_count, st.idle, n, transpose, planes);
  count_launches(1);
  return cudaGetLastError();
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

cudaError_t launch_wait_selftest(int* status, long long wait_cycles, cudaStream_t s) {
  wait_selftest_kernel<<<1, 1, 0, s>>>(status, wait_cycles);
  count_launches(1);
  return cudaGetLastError();
}

size_t chain_tc_scratch_bytes(int n) {
  const size_t N = size_t(1) << n;
  return 18 * N * N * sizeof(__nv_bfloat16);  // V, V' and S: 6 planes each
}

// U = S_m ... S_1 with the BF16x3 tcgen05 chain.  n >= 7 (N a multiple of 128).
cudaError_t chain_tc(const StepFactor* d_factors, const StepDesc* steps, int nsteps, int n,
                     float2* d_U, void* scratch, int* d_err, cudaStream_t s) {
  if (n < 7 || nsteps < 2) return cudaErrorInvalidValue;
  const int N = 1 << n;
  const size_t NN = size_t(N) * N;
  __nv_bfloat16* V0 = static_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* V1 = V0 + 6 * NN;
  __nv_bfloat16* S = V1 + 6 * NN;
  CUtensorMap mV0, mV1, mS;
  if (!make_planes_map(&mV0, V0, N) || !make_planes_map(&mV1, V1, N) || !make_planes_map(&mS, S, N))
    return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(chain_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kGemmSmem));
  if (e != cudaSuccess) return e;
  e = launch_gen(d_factors, steps[0], n, 1, V0, s);  // V = S_1^T
  if (e != cudaSuccess) return e;
  bool cur0 = true;
  for (int k = 1; k < nsteps; ++k) {
    e = launch_gen(d_factors, steps[k], n, 0, S, s);
    if (e != cudaSuccess) return e;
    GemmParams P;
    P.N = N;
    P.final_step = (k == nsteps - 1) ? 1 : 0;
    P.planes = cur0 ? V1 : V0;
    P.u = d_U;
    P.err = d_err;
    const int grid = (N / BN) * (N / BM);
    chain_gemm_kernel<<<grid, kGemmThreads, kGemmSmem, s>>>(cur0 ? mV0 : mV1, mS, P);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cur0 = !cur0;
  }
  return cudaSuccess;
}

}  // namespace tqs
