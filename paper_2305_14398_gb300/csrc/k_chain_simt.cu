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

// D[m][n] = sum_k A[m][k] B[n][k]; transpose_out: write D^T instead.
__global__ void __launch_bounds__(kSimtThreads)
    cgemm_nt_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                    float2* __restrict__ D, int N, int transpose_out) {
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
      const size_t NN = static_cast<size_t>(N) * N;
      As[kk][TQS_IX(row, TM)] = A[TQS_IX(static_cast<size_t>(m0 + row) * N + k0 + kk, NN)];
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
      const size_t NN = static_cast<size_t>(N) * N;
      if (transpose_out)
        D[TQS_IX(static_cast<size_t>(n) * N + m, NN)] = acc[i][j];
      else
        D[TQS_IX(static_cast<size_t>(m) * N + n, NN)] = acc[i][j];
    }
}

// The same product for small N (below one 64 x 64 tile): one thread per output.
__global__ void cgemm_nt_small_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                      float2* __restrict__ D, int N, int transpose_out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const int m = idx / N, n = idx % N;
  float2 acc = make_float2(0.f, 0.f);
  for (int k = 0; k < N; ++k) cmac(acc, A[m * N + k], B[n * N + k]);
  if (transpose_out)
    D[n * N + m] = acc;
  else
    D[m * N + n] = acc;
}

// dst = src^T (N x N complex64), 32 x 32 tiles through shared memory.
__global__ void transpose_kernel(const float2* __restrict__ src, float2* __restrict__ dst, int N) {
  __shared__ float2 t[32][33];
  const int x = blockIdx.x * 32 + threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += 8)
    t[r][threadIdx.x] = src[TQS_IX(static_cast<size_t>(blockIdx.y * 32 + r) * N + x,
                                   static_cast<size_t>(N) * N)];
  __syncthreads();
  const int x2 = blockIdx.y * 32 + threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += 8)
    dst[TQS_IX(static_cast<size_t>(blockIdx.x * 32 + r) * N + x2, static_cast<size_t>(N) * N)] =
        t[threadIdx.x][r];
}

__global__ void transpose_small_kernel(const float2* __restrict__ src, float2* __restrict__ dst,
                                       int N) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const int r = idx / N, c = idx % N;
  dst[c * N + r] = src[r * N + c];
}

}  // namespace

TQS_DEFINE_VIOLATIONS(violations_chain_simt)

size_t chain_simt_scratch_bytes(int n) {
  const size_t N = size_t(1) << n;
  return 3 * N * N * sizeof(float2);  // V, V', S
}

// U = S_m ... S_1 in FP32 SIMT (any n >= 1, nsteps >= 2).
cudaError_t chain_simt(const StepFactor* d_factors, const StepDesc* steps, int nsteps, int n,
                       float2* d_U, void* scratch, cudaStream_t s) {
  if (n < 1 || nsteps < 2) return cudaErrorInvalidValue;
  const int N = 1 << n;
  const size_t NN = size_t(N) * N;
  float2* V0 = static_cast<float2*>(scratch);
  float2* V1 = V0 + NN;
  float2* S = V1 + NN;
  // V = S_1^T
  cudaError_t e = launch_materialize(d_factors, steps[0], n, S, s);
  if (e != cudaSuccess) return e;
  if (N >= 32)
    transpose_kernel<<<dim3(N / 32, N / 32), dim3(32, 8), 0, s>>>(S, V0, N);
  else
    transpose_small_kernel<<<(N * N + 255) / 256, 256, 0, s>>>(S, V0, N);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  float2* cur = V0;
  float2* nxt = V1;
  for (int k = 1; k < nsteps; ++k) {
    e = launch_materialize(d_factors, steps[k], n, S, s);
    if (e != cudaSuccess) return e;
    const bool last = (k == nsteps - 1);
    float2* dst = last ? d_U : nxt;
    if (N >= TM)
      cgemm_nt_kernel<<<dim3(N / TN, N / TM), kSimtThreads, 0, s>>>(cur, S, dst, N, last ? 1 : 0);
    else
      cgemm_nt_small_kernel<<<(N * N + 255) / 256, 256, 0, s>>>(cur, S, dst, N, last ? 1 : 0);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    float2* t = cur;
    cur = nxt;
    nxt = t;
  }
  return cudaSuccess;
}

}  // namespace tqs
