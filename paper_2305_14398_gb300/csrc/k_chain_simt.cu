// Circuit-unitary chain in FP32 on the CUDA cores (sm_103a), the comparison
// arithmetic of Algorithm 1: U <- S_k U with every complex product done as
// four real multiply-adds (the paper's stage-5 kernel computes the same
// triple loop over separate real/imaginary arrays).
//
// Kept transposed like the tensor-core chain: V = U^T, V' = V S_k^T, so both
// operands are read along K.  Tile: 64 x 64 complex outputs per 256-thread
// block, 4 x 4 per thread, K step 16 staged in shared memory.
#include "checked.h"
#include "tqs_internal.h"

namespace tqs {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;
constexpr int kSimtThreads = 256;

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// D[m][n] = sum_k A[m][k] B[n][k] for m < M (A and D: M x N), n, k < N;
// transpose_out: write D^T instead, D[n * ldd + m].
__global__ void __launch_bounds__(kSimtThreads)
    cgemm_nt_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                    float2* __restrict__ D, int N, int M, int64_t ldd, int transpose_out) {
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < N; k0 += TK) {
    // 64 x 16 complex of A and of B: 4 elements per thread each
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = threadIdx.x + r * kSimtThreads;  // 0..1023
      const int row = idx >> 4, kk = idx & 15;
      const size_t NN = static_cast<size_t>(N) * N, MN = static_cast<size_t>(M) * N;
      As[kk][TQS_IX(row, TM)] = A[TQS_IX(static_cast<size_t>(m0 + row) * N + k0 + kk, MN)];
      Bs[kk][TQS_IX(row, TN)] = B[TQS_IX(static_cast<size_t>(n0 + row) * N + k0 + kk, NN)];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cmac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (transpose_out)
        D[TQS_IX(static_cast<size_t>(n) * static_cast<size_t>(ldd) + m,
                 static_cast<size_t>(N - 1) * static_cast<size_t>(ldd) + M)] = acc[i][j];
      else
        D[TQS_IX(static_cast<size_t>(m) * N + n, static_cast<size_t>(M) * N)] = acc[i][j];
    }
}

// The same product for small sizes (below one 64 x 64 tile): one thread per output.
__global__ void cgemm_nt_small_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                      float2* __restrict__ D, int N, int M, int64_t ldd,
                                      int transpose_out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int m = idx / N, n = idx % N;
  float2 acc = make_float2(0.f, 0.f);
  for (int k = 0; k < N; ++k) cmac(acc, A[m * N + k], B[n * N + k]);
  if (transpose_out)
    D[static_cast<int64_t>(n) * ldd + m] = acc;
  else
    D[m * N + n] = acc;
}

// dst[j][r] = src[r][col0 + j] for j < M, r < N: the columns col0.. of the
// N x N src as the rows of the M x N dst; 32 x 32 tiles through shared memory
// (grid: M / 32 x N / 32).
__global__ void transpose_kernel(const float2* __restrict__ src, float2* __restrict__ dst, int N,
                                 int col0, int M) {
  __shared__ float2 t[32][33];
  const int x = col0 + blockIdx.x * 32 + threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += 8)
    t[r][threadIdx.x] = src[TQS_IX(static_cast<size_t>(blockIdx.y * 32 + r) * N + x,
                                   static_cast<size_t>(N) * N)];
  __syncthreads();
  const int x2 = blockIdx.y * 32 + threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += 8)
    dst[TQS_IX(static_cast<size_t>(blockIdx.x * 32 + r) * N + x2, static_cast<size_t>(M) * N)] =
        t[threadIdx.x][r];
}

__global__ void transpose_small_kernel(const float2* __restrict__ src, float2* __restrict__ dst,
                                       int N, int col0, int M) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int j = idx / N, r = idx % N;
  dst[j * N + r] = src[r * N + col0 + j];
}

}  // namespace

TQS_DEFINE_VIOLATIONS(violations_chain_simt)

size_t chain_simt_scratch_bytes(int n, int ncols) {
  const size_t N = size_t(1) << n;
  return (2 * size_t(ncols) * N + N * N) * sizeof(float2);  // V, V' (ncols rows), S
}

// Columns [col0, col0 + ncols) of U = S_m ... S_1 in FP32 SIMT (n >= 1,
// nsteps >= 2): rows col0.. of V = U^T, written as U[r][col0 + j] at
// d_U[r * ldu + j].  The tiled kernels need N >= 64 and ncols a multiple of
// 64 (col0 of 32); other blocks take the one-thread-per-output kernels.
cudaError_t chain_simt(const StepFactor* d_factors, const StepDesc* steps, int nsteps, int n,
                       int col0, int ncols, float2* d_U, int64_t ldu, void* scratch, cudaStream_t s) {
  if (n < 1 || nsteps < 2 || col0 < 0 || ncols < 1 || col0 + ncols > (1 << n) || ldu < ncols)
    return cudaErrorInvalidValue;
  const int N = 1 << n;
  const int M = ncols;
  const size_t MN = size_t(M) * N;
  float2* V0 = static_cast<float2*>(scratch);
  float2* V1 = V0 + MN;
  float2* S = V1 + MN;
  const bool tiled = N >= TM && M % TM == 0 && col0 % 32 == 0;
  // V = rows col0.. of S_1^T
  cudaError_t e = launch_materialize(d_factors, steps[0], n, S, s);
  if (e != cudaSuccess) return e;
  if (tiled)
    transpose_kernel<<<dim3(M / 32, N / 32), dim3(32, 8), 0, s>>>(S, V0, N, col0, M);
  else
    transpose_small_kernel<<<(M * N + 255) / 256, 256, 0, s>>>(S, V0, N, col0, M);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  float2* cur = V0;
  float2* nxt = V1;
  for (int k = 1; k < nsteps; ++k) {
    e = launch_materialize(d_factors, steps[k], n, S, s);
    if (e != cudaSuccess) return e;
    const bool last = (k == nsteps - 1);
    float2* dst = last ? d_U : nxt;
    if (tiled)
      cgemm_nt_kernel<<<dim3(N / TN, M / TM), kSimtThreads, 0, s>>>(cur, S, dst, N, M, ldu,
                                                                      last ? 1 : 0);
    else
      cgemm_nt_small_kernel<<<(M * N + 255) / 256, 256, 0, s>>>(cur, S, dst, N, M, ldu,
                                                                 last ? 1 : 0);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    float2* t = cur;
    cur = nxt;
    nxt = t;
  }
  return cudaSuccess;
}

}  // namespace tqs
