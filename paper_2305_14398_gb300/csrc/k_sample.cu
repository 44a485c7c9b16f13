// Inverse-CDF sampling of outcomes from probabilities (sm_103a): the collapse
// of simulateAndCollapse (Sec. 5.2), drawn according to p_i = |psi_i|^2
// (Sec. 2.1, eq. 2).
//
// A "segment" is one state's probability vector (one for tqs_sample, one per
// circuit for a batch), cut into blocks of 256 entries, each block into 32
// chunks of 8 consecutive entries.  The cumulative sums are defined by this
// file's FP64 summation order:
//   * chunk total: the chunk's 8 entries added in index order;
//   * chunk prefix in its block: exclusive warp scan of the 32 chunk totals
//     (Hillis-Steele, fixed order); the block total is the inclusive value of
//     the last chunk;
//   * block prefix: each thread of a CTA sums a contiguous run of block
//     totals, the runs are combined in order (warp scan, then warp totals);
//   * chunk base cbase_{b,l} = bpre_b + cpre_{b,l};
//   * C_i = cbase_{b,l} + p_{first of chunk} + ... + p_i.
// A shot with uniform u and target u T (T: the segment total) takes the last
// block b with bpre_b <= target, the last chunk l of it with cbase_{b,l} <=
// target, and the first entry i of that chunk with p_i > 0 and target <
// C_i.  If there is none (rounding, or u T >= T), the last index at or before
// that point with p_i > 0; -1 when every probability is 0.
//
// GB300's FP64 rate is about 1/64 of its FP32 rate, so the design keeps FP64
// operations few: the tables cost about 15 warp-wide FP64 additions per 256
// entries (the chunk bases bpre_b + cpre_{b,l} are stored absolute), and a
// shot is one multiply, binary searches that compare the FP64 bit patterns as
// integers (the order of non-negative doubles), and at most 8 adds.
// Two paths share that arithmetic: segments of up to 2^13 entries are staged
// in shared memory by one CTA each, which builds the tables there and runs
// every shot of the segment; larger segments use three kernels over global
// memory (block tables, block prefix, shots).
#include "checked.h"
#include "tqs_internal.h"

namespace tqs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kChunks = kSampleBlk / kSampleChunk;  // 32: one per lane
static_assert(kChunks == 32, "one chunk per lane");

__device__ __forceinline__ double warp_incl_scan(double x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

__device__ __forceinline__ int seg_of_block(const SampleSeg* segs, int nseg, int64_t gb) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].blk_off <= gb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Block b's tables (whole warp, lane = chunk): cpre[lane] = exclusive chunk
// prefix; returns the block total (same value in every lane).  `p` may be
// global or shared memory; entries past len count as 0.
__device__ __forceinline__ double block_tables(const double* p, int64_t len, int64_t b, int lane,
                                              double* cpre) {
  const int64_t i0 = b * kSampleBlk + int64_t(lane) * kSampleChunk;
  double t = 0.0;
#pragma unroll
  for (int j = 0; j < kSampleChunk; ++j) t += (i0 + j < len) ? p[TQS_IX(i0 + j, len)] : 0.0;
  const double incl = warp_incl_scan(t, lane);
  const double up = __shfl_up_sync(kFull, incl, 1);
  cpre[lane] = lane > 0 ? up : 0.0;
  return __shfl_sync(kFull, incl, 31);
}

// Exclusive prefix bp[0..nb) of the block totals bs[0..nb) and their total
// *tot, by the kThreads threads of a CTA: thread t sums the contiguous run of
// ceil(nb / kThreads) blocks starting at t * that, the runs are combined by a
// warp scan and the warp totals in order, then each thread writes its run.
__device__ void block_prefix_cta(const double* bs, double* bp, int64_t nb, double* tot,
                                 double* wtot, double* wpre) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t chunk = (nb + kThreads - 1) / kThreads;
  const int64_t b0 = int64_t(t) * chunk;
  const int64_t b1 = b0 + chunk < nb ? b0 + chunk : nb;
  double s = 0.0;
  for (int64_t b = b0; b < b1; ++b) s += bs[TQS_IX(b, nb)];
  const double incl = warp_incl_scan(s, lane);
  const double up = __shfl_up_sync(kFull, incl, 1);
  const double excl = lane > 0 ? up : 0.0;
  if (lane == 31) wtot[TQS_IX(warp, kThreads / 32)] = incl;
  __syncthreads();
  if (t == 0) {
    double a = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) { wpre[w] = a; a += wtot[w]; }
  }
  __syncthreads();
  double acc = wpre[warp] + excl;
  for (int64_t b = b0; b < b1; ++b) {
    bp[TQS_IX(b, nb)] = acc;
    acc += bs[TQS_IX(b, nb)];
  }
  if (b0 < nb && b1 == nb) *tot = acc;
}

// a <= b for non-negative doubles, as integers on their bit patterns.
__device__ __forceinline__ bool le_bits(double a, double b) {
  return __double_as_longlong(a) <= __double_as_longlong(b);
}

// Chunk prefixes of the blocks [0, nb) made absolute: cp[b * 32 + l] becomes
// bp[b] + cp[b * 32 + l] (whole CTA).
__device__ void absolute_chunks(const double* bp, double* cp, int64_t nb) {
  for (int64_t e = threadIdx.x; e < nb * kChunks; e += kThreads)
    cp[e] = bp[TQS_IX(e / kChunks, nb)] + cp[e];
}

// Last index <= i with p > 0, or -1 (one thread; reached only after rounding
// or for u T >= T).
__device__ int64_t last_nonzero_upto(const double* p, int64_t len, int64_t i) {
  for (; i >= 0; --i)
    if (__double_as_longlong(p[TQS_IX(i, len)]) > 0) return i;
  return -1;
}

// One shot (one thread).  p: the segment's entries; bp: its block prefix; cp:
// its absolute chunk bases (global or shared memory).
__device__ int64_t sample_shot(const double* p, int64_t len, const double* bp, const double* cp,
                               int64_t nb, double T, double u) {
  const double target = u * T;
  if (!(target < T)) return last_nonzero_upto(p, len, len - 1);
  int64_t lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (le_bits(bp[TQS_IX(mid, nb)], target)) lo = mid; else hi = mid - 1;
  }
  const int64_t b = lo;
  const double* cpb = cp + TQS_IX(b, nb) * kChunks;
  int l = 0, h = kChunks - 1;
  while (l < h) {
    const int mid = (l + h + 1) >> 1;
    if (le_bits(cpb[TQS_IX(mid, kChunks)], target)) l = mid; else h = mid - 1;
  }
  const int64_t i0 = b * kSampleBlk + int64_t(l) * kSampleChunk;
  double c = cpb[TQS_IX(l, kChunks)];
  for (int j = 0; j < kSampleChunk && i0 + j < len; ++j) {
    const double x = p[TQS_IX(i0 + j, len)];
    c += x;
    if (__double_as_longlong(x) > 0 && !le_bits(c, target)) return i0 + j;
  }
  const int64_t end = i0 + kSampleChunk - 1 < len - 1 ? i0 + kSampleChunk - 1 : len - 1;
  return last_nonzero_upto(p, len, end);
}

// ------------------------------------------------------------ global path

__global__ void __launch_bounds__(kThreads)
    block_tables_kernel(const SampleLaunch L) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (kThreads / 32);
  for (int64_t gb = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5); gb < L.nblocks;
       gb += warps) {
    const SampleSeg sg = L.gsegs[TQS_IX(seg_of_block(L.gsegs, L.n_gseg, gb), L.n_gseg)];
    (void)TQS_IX(sg.p_off + (int64_t(1) << sg.n) - 1, L.probs_len);
    const double t = block_tables(L.probs + sg.p_off, int64_t(1) << sg.n, gb - sg.blk_off, lane,
                                  L.cpre + TQS_IX(gb, L.nblocks) * kChunks);
    if (lane == 0) L.bsum[TQS_IX(gb, L.nblocks)] = t;
  }
}

__global__ void __launch_bounds__(kThreads)
    block_prefix_kernel(const SampleLaunch L) {
  __shared__ double wtot[kThreads / 32], wpre[kThreads / 32];
  const SampleSeg sg = L.gsegs[TQS_IX(blockIdx.x, L.n_gseg)];
  (void)TQS_IX(sg.blk_off + sample_blocks(sg.n) - 1, L.nblocks);
  block_prefix_cta(L.bsum + sg.blk_off, L.bpre + sg.blk_off, sample_blocks(sg.n),
                   L.tot + blockIdx.x, wtot, wpre);
  __syncthreads();
  absolute_chunks(L.bpre + sg.blk_off, L.cpre + int64_t(sg.blk_off) * kChunks, sample_blocks(sg.n));
}

__global__ void __launch_bounds__(kThreads)
    shots_kernel(const SampleLaunch L) {
  const int64_t total = int64_t(L.n_gseg) * L.shots;
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < total;
       k += int64_t(gridDim.x) * kThreads) {
    const int g = static_cast<int>(k / L.shots);
    const SampleSeg sg = L.gsegs[TQS_IX(g, L.n_gseg)];
    const int64_t kk = TQS_IX(sg.index * L.shots + (k - int64_t(g) * L.shots), L.n_segs * L.shots);
    L.out[kk] = sample_shot(L.probs + sg.p_off, int64_t(1) << sg.n, L.bpre + sg.blk_off,
                            L.cpre + int64_t(sg.blk_off) * kChunks, sample_blocks(sg.n), L.tot[g],
                            L.u[kk]);
  }
}

// ------------------------------------------------------ shared-memory path
// One CTA per segment (n <= kSampleSmemMaxQ).  Dynamic shared memory holds
// the 2^smem_q entries, then the chunk prefixes (32 per block: at least 32).

__global__ void __launch_bounds__(kThreads)
    segment_smem_kernel(const SampleLaunch L) {
  extern __shared__ double sm[];
  __shared__ double wtot[kThreads / 32], wpre[kThreads / 32];
  __shared__ double s_tot;
  constexpr int kMaxBlocks = 1 << (kSampleSmemMaxQ - 8);
  __shared__ double sbs[kMaxBlocks], sbp[kMaxBlocks];
  const SampleSeg sg = L.ssegs[TQS_IX(blockIdx.x, L.n_sseg)];
  const int64_t len = int64_t(1) << sg.n;
  const int64_t nb = sample_blocks(sg.n);
  double* sp = sm;
  double* scp = sm + (size_t(1) << L.smem_q);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t qlen = int64_t(1) << L.smem_q;
  const int64_t nchunks = (qlen < kSampleBlk ? kSampleBlk : qlen) / kSampleChunk;
  (void)TQS_IX(sg.p_off + len - 1, L.probs_len);
  const double2* gp = reinterpret_cast<const double2*>(L.probs + sg.p_off);
  for (int64_t i = t; i < len / 2; i += kThreads) {
    const double2 v = __ldcs(gp + i);
    sp[TQS_IX(2 * i, qlen)] = v.x;
    sp[TQS_IX(2 * i + 1, qlen)] = v.y;
  }
  __syncthreads();
  for (int64_t b = warp; b < nb; b += kThreads / 32) {
    const double bt = block_tables(sp, len, b, lane, scp + TQS_IX(b * kChunks + lane, nchunks) - lane);
    if (lane == 0) sbs[TQS_IX(b, kMaxBlocks)] = bt;
  }
  __syncthreads();
  (void)TQS_IX(nb - 1, kMaxBlocks);
  block_prefix_cta(sbs, sbp, nb, &s_tot, wtot, wpre);
  __syncthreads();
  absolute_chunks(sbp, scp, nb);
  __syncthreads();
  const double T = s_tot;
  for (int64_t k = t; k < L.shots; k += kThreads) {
    const int64_t kk = TQS_IX(sg.index * L.shots + k, L.n_segs * L.shots);
    L.out[kk] = sample_shot(sp, len, sbp, scp, nb, T, __ldcs(L.u + kk));
  }
}

__global__ void set_basis_kernel(float2* st, int64_t len, const int64_t* idx) {
  const int64_t i0 = *idx;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < len;
       i += int64_t(gridDim.x) * blockDim.x)
    st[i] = make_float2(i == i0 ? 1.f : 0.f, 0.f);
}

int grid_for(int64_t items, int per_cta) {
  const int64_t ctas = (items + per_cta - 1) / per_cta;
  const int64_t cap = 152 * 8;
  return static_cast<int>(ctas < 1 ? 1 : (ctas < cap ? ctas : cap));
}

}  // namespace

TQS_DEFINE_VIOLATIONS(violations_sample)

cudaError_t launch_sample(const SampleLaunch& L, cudaStream_t s) {
  int k = 0;
  if (L.n_gseg > 0) {
    block_tables_kernel<<<grid_for(L.nblocks, kThreads / 32), kThreads, 0, s>>>(L);
    block_prefix_kernel<<<L.n_gseg, kThreads, 0, s>>>(L);
    k += 2;
    if (L.shots > 0) {
      shots_kernel<<<grid_for(int64_t(L.n_gseg) * L.shots, kThreads), kThreads, 0, s>>>(L);
      ++k;
    }
  }
  if (L.n_sseg > 0 && L.shots > 0) {
    const size_t q = size_t(1) << L.smem_q;
    const size_t chunks = (q < kSampleBlk ? kSampleBlk : q) / kSampleChunk;
    const int smem = static_cast<int>((q + chunks) * sizeof(double));
    cudaError_t e = cudaFuncSetAttribute(segment_smem_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    segment_smem_kernel<<<L.n_sseg, kThreads, smem, s>>>(L);
    ++k;
  }
  count_launches(k);
  return cudaGetLastError();
}

cudaError_t launch_set_basis(float2* d_state, int n, const int64_t* d_index, cudaStream_t s) {
  const int64_t len = int64_t(1) << n;
  set_basis_kernel<<<grid_for(len, kThreads), kThreads, 0, s>>>(d_state, len, d_index);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tqs
