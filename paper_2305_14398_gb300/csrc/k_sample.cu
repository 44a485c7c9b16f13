// Inverse-CDF sampling of outcomes from probabilities (sm_103a): the collapse
// of simulateAndCollapse (Sec. 5.2), drawn according to p_i = |psi_i|^2
// (Sec. 2.1, eq. 2).
//
// A "segment" is one state's probability vector (one for tqs_sample, one per
// circuit for a batch), cut into blocks of 256 entries, each block into 32
// chunks of 8 consecutive entries.  The cumulative sums are defined by this
// file's summation order (FP64 on the global path; exact 64-bit fixed point,
// where the order does not matter, on the shared-memory path):
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
// operations few: on the global path the tables cost about 15 warp-wide FP64
// additions per 256 entries (the chunk bases bpre_b + cpre_{b,l} are stored
// absolute), and a shot is one multiply, binary searches that compare the FP64
// bit patterns as integers (the order of non-negative doubles), and at most 8
// adds; the shared-memory path needs one FP64 multiply per shot and nothing else.
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

// Values of the cumulative sums: FP64 (the global path) or unsigned 64-bit
// fixed point (the shared-memory path); le: a <= b (for non-negative FP64, the
// order of the bit patterns); pos: the value is above 0.
__device__ __forceinline__ bool le_val(double a, double b) {
  return __double_as_longlong(a) <= __double_as_longlong(b);
}
__device__ __forceinline__ bool le_val(unsigned long long a, unsigned long long b) { return a <= b; }
__device__ __forceinline__ bool pos_val(double a) { return __double_as_longlong(a) > 0; }
__device__ __forceinline__ bool pos_val(unsigned long long a) { return a > 0; }

template <class V>
__device__ __forceinline__ V warp_incl_scan(V x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V y = __shfl_up_sync(kFull, x, o);
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
template <class V>
__device__ __forceinline__ V block_tables(const V* p, int64_t len, int64_t b, int lane, V* cpre) {
  const int64_t i0 = b * kSampleBlk + int64_t(lane) * kSampleChunk;
  V t = V(0);
#pragma unroll
  for (int j = 0; j < kSampleChunk; ++j) t += (i0 + j < len) ? p[TQS_IX(i0 + j, len)] : V(0);
  const V incl = warp_incl_scan(t, lane);
  const V up = __shfl_up_sync(kFull, incl, 1);
  cpre[lane] = lane > 0 ? up : V(0);
  return __shfl_sync(kFull, incl, 31);
}

// Exclusive prefix bp[0..nb) of the block totals bs[0..nb) and their total
// *tot, by the kThreads threads of a CTA: thread t sums the contiguous run of
// ceil(nb / kThreads) blocks starting at t * that, the runs are combined by a
// warp scan and the warp totals in order, then each thread writes its run.
template <class V>
__device__ void block_prefix_cta(const V* bs, V* bp, int64_t nb, V* tot, V* wtot, V* wpre) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t chunk = (nb + kThreads - 1) / kThreads;
  const int64_t b0 = int64_t(t) * chunk;
  const int64_t b1 = b0 + chunk < nb ? b0 + chunk : nb;
  V s = V(0);
  for (int64_t b = b0; b < b1; ++b) s += bs[TQS_IX(b, nb)];
  const V incl = warp_incl_scan(s, lane);
  const V up = __shfl_up_sync(kFull, incl, 1);
  const V excl = lane > 0 ? up : V(0);
  if (lane == 31) wtot[TQS_IX(warp, kThreads / 32)] = incl;
  __syncthreads();
  if (t == 0) {
    V a = V(0);
    for (int w = 0; w < kThreads / 32; ++w) { wpre[w] = a; a += wtot[w]; }
  }
  __syncthreads();
  V acc = wpre[warp] + excl;
  for (int64_t b = b0; b < b1; ++b) {
    bp[TQS_IX(b, nb)] = acc;
    acc += bs[TQS_IX(b, nb)];
  }
  if (b0 < nb && b1 == nb) *tot = acc;
}

// Chunk prefixes of the blocks [0, nb) made absolute: cp[b * 32 + l] becomes
// bp[b] + cp[b * 32 + l] (whole CTA).
template <class V>
__device__ void absolute_chunks(const V* bp, V* cp, int64_t nb) {
  for (int64_t e = threadIdx.x; e < nb * kChunks; e += kThreads)
    cp[e] = bp[TQS_IX(e / kChunks, nb)] + cp[e];
}

// Last index <= i with p > 0, or -1 (one thread; reached only after rounding
// or for u T >= T).
template <class V>
__device__ int64_t last_nonzero_upto(const V* p, int64_t len, int64_t i) {
  for (; i >= 0; --i)
    if (pos_val(p[TQS_IX(i, len)])) return i;
  return -1;
}

// One shot (one thread).  p: the segment's entries; bp: its block prefix; cp:
// its absolute chunk bases (global or shared memory).
template <class V>
__device__ int64_t sample_shot(const V* p, int64_t len, const V* bp, const V* cp, int64_t nb, V T,
                               V target) {
  if (!(target < T)) return last_nonzero_upto(p, len, len - 1);
  int64_t lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (le_val(bp[TQS_IX(mid, nb)], target)) lo = mid; else hi = mid - 1;
  }
  const int64_t b = lo;
  const V* cpb = cp + TQS_IX(b, nb) * kChunks;
  int l = 0, h = kChunks - 1;
  while (l < h) {
    const int mid = (l + h + 1) >> 1;
    if (le_val(cpb[TQS_IX(mid, kChunks)], target)) l = mid; else h = mid - 1;
  }
  const int64_t i0 = b * kSampleBlk + int64_t(l) * kSampleChunk;
  V c = cpb[TQS_IX(l, kChunks)];
  for (int j = 0; j < kSampleChunk && i0 + j < len; ++j) {
    const V x = p[TQS_IX(i0 + j, len)];
    c += x;
    if (pos_val(x) && !le_val(c, target)) return i0 + j;
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
    const double T = L.tot[g];
    L.out[kk] = sample_shot(L.probs + sg.p_off, int64_t(1) << sg.n, L.bpre + sg.blk_off,
                            L.cpre + int64_t(sg.blk_off) * kChunks, sample_blocks(sg.n), T,
                            L.u[kk] * T);
  }
}

// ------------------------------------------------------ shared-memory path
// One CTA per segment (n <= kSampleSmemMaxQ).  Dynamic shared memory holds
// the 2^smem_q entries, then the chunk prefixes (32 per block: at least 32).
//
// Here the cumulative sums are exact: each probability p becomes the 64-bit
// integer floor(p 2^S), with S chosen from an FP32 estimate of the segment's
// total T so that T 2^S stays below 2^61 (each entry then loses less than
// 2^-60 T, all of them together less than 2^(n - 60) T: 4e-15 T at n = 13; a
// probability below 2^-S counts as 0); the sums are integer additions in the
// fixed order above, and a shot's target is floor(u T 2^S).  The FP64 pipe
// (1/64 of the FP32 rate on this GPU) is left to one multiply per shot.

// p as FP32 (truncated; 0 below the FP32 range), from the FP64 bits with
// integer operations only: for the estimate of the total.
__device__ __forceinline__ float approx_f32(unsigned long long bits) {
  const int e = static_cast<int>((bits >> 52) & 0x7FF);
  if (e < 1023 - 126) return 0.f;
  if (e > 1023 + 127) return __int_as_float(0x7f800000);
  return __int_as_float(((e - 1023 + 127) << 23) | static_cast<int>((bits >> 29) & 0x7FFFFF));
}

// floor(p 2^S) for a non-negative FP64 p given by its bits; S such that the
// result stays below 2^62.
__device__ __forceinline__ unsigned long long to_fixed(unsigned long long bits, int S) {
  const int e = static_cast<int>((bits >> 52) & 0x7FF);
  unsigned long long m = bits & ((1ull << 52) - 1);
  int ex = e;
  if (e == 0) ex = 1;        // subnormal: no implicit bit
  else m |= 1ull << 52;
  const int sh = ex - 1075 + S;  // p = m 2^(ex - 1075)
  if (sh >= 0) return m << sh;
  if (sh <= -64) return 0ull;
  return m >> (-sh);
}

__global__ void __launch_bounds__(kThreads)
    segment_smem_kernel(const SampleLaunch L) {
  using U = unsigned long long;
  extern __shared__ U sm[];
  __shared__ U wtot[kThreads / 32], wpre[kThreads / 32];
  __shared__ U s_tot;
  __shared__ int s_emax[kThreads / 32];
  __shared__ float s_fsum[kThreads / 32];
  constexpr int kMaxBlocks = 1 << (kSampleSmemMaxQ - 8);
  __shared__ U sbs[kMaxBlocks], sbp[kMaxBlocks];
  const SampleSeg sg = L.ssegs[TQS_IX(blockIdx.x, L.n_sseg)];
  const int64_t len = int64_t(1) << sg.n;
  const int64_t nb = sample_blocks(sg.n);
  U* sp = sm;
  U* scp = sm + (size_t(1) << L.smem_q);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t qlen = int64_t(1) << L.smem_q;
  const int64_t nchunks = (qlen < kSampleBlk ? kSampleBlk : qlen) / kSampleChunk;
  (void)TQS_IX(sg.p_off + len - 1, L.probs_len);
  // the probabilities' bits into shared memory, and their largest exponent
  const ulonglong2* gp = reinterpret_cast<const ulonglong2*>(L.probs + sg.p_off);
  int emax = 0;
  float fsum = 0.f;
  for (int64_t i = t; i < len / 2; i += kThreads) {
    const ulonglong2 v = __ldcs(gp + i);
    sp[TQS_IX(2 * i, qlen)] = v.x;
    sp[TQS_IX(2 * i + 1, qlen)] = v.y;
    emax = max(emax, max(static_cast<int>((v.x >> 52) & 0x7FF), static_cast<int>((v.y >> 52) & 0x7FF)));
    fsum += approx_f32(v.x) + approx_f32(v.y);
  }
  emax = __reduce_max_sync(kFull, emax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fsum += __shfl_xor_sync(kFull, fsum, o);
  if (lane == 0) {
    s_emax[warp] = emax;
    s_fsum[warp] = fsum;
  }
  __syncthreads();
  emax = 0;
  fsum = 0.f;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) {
    emax = max(emax, s_emax[w]);
    fsum += s_fsum[w];
  }
  // T < 2^(ET + 1) (within the estimate's error), so T 2^S < 2^61 with
  // S = 60 - ET; entries below the FP32 range (no estimate) use the largest
  // exponent instead: every p < 2^(emax - 1022), 2^n of them below 2^62
  const int ET = (__float_as_int(fsum) >> 23) - 127;
  const int S = (fsum > 0.f && fsum < 3.0e38f) ? 60 - ET : 62 - sg.n - (max(emax, 1) - 1022);
  for (int64_t i = t; i < len; i += kThreads) sp[TQS_IX(i, qlen)] = to_fixed(sp[TQS_IX(i, qlen)], S);
  __syncthreads();
  for (int64_t b = warp; b < nb; b += kThreads / 32) {
    const U bt = block_tables(sp, len, b, lane, scp + TQS_IX(b * kChunks + lane, nchunks) - lane);
    if (lane == 0) sbs[TQS_IX(b, kMaxBlocks)] = bt;
  }
  __syncthreads();
  (void)TQS_IX(nb - 1, kMaxBlocks);
  block_prefix_cta(sbs, sbp, nb, &s_tot, wtot, wpre);
  __syncthreads();
  absolute_chunks(sbp, scp, nb);
  __syncthreads();
  const U T = s_tot;
  const double Tf = static_cast<double>(T);
  for (int64_t k = t; k < L.shots; k += kThreads) {
    const int64_t kk = TQS_IX(sg.index * L.shots + k, L.n_segs * L.shots);
    // floor(u T); u < 1 keeps it below T up to the rounding of the product
    const double x = __ldcs(L.u + kk) * Tf;
    const U target = x >= Tf ? T : static_cast<U>(x);
    L.out[kk] = sample_shot(sp, len, sbp, scp, nb, T, target);
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
