// Fused on-the-fly step kernel for sm_103a.
//
// psi' = S_k psi for every step k of a circuit (eq. 11), where S_k is the
// Kronecker product of the step's factors (Algorithm 2) and is never written
// out: each factor acts as a butterfly on the amplitude pairs whose indices
// differ only in its target bit (eq. 12), restricted to control = 1 for a
// controlled factor (eq. 7).  The host compiles the steps into passes of
// 4 thread-local qubit bits (see tqs_internal.h); a team of threads holds the
// circuit's state in shared memory (or, above 2^14 amplitudes, in L2-resident
// global scratch) and runs the passes, then writes the state in logical
// order, |psi_i|^2 in FP64, and the FP64 norm.
//
// Teams: one warp per circuit (n <= 11), one CTA per circuit (n <= 14), or one
// CTA on global scratch (n <= 16).  Warps/CTAs pull circuits from an atomic
// job counter (costliest first), so one persistent launch runs a whole batch.
#include "tqs_internal.h"

namespace tqs {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Shared-memory slot of amplitude i: XOR the low 4 bits with bits 4..7 so that
// the 16-amplitude groups of a warp spread over the banks for any choice of
// local bits.  A bijection on every aligned block of 256 amplitudes.
__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 4) & 15); }

// Insert a zero bit at position b.
__device__ __forceinline__ int ins0(int x, int b) {
  return ((x >> b) << (b + 1)) | (x & ((1 << b) - 1));
}

// (ah + al) * x + (bh + bl) * y for coefficients split into FP32 hi + lo
// parts: the small lo products first, then the hi products, so that the
// coefficient rounding of a single FP32 matrix adds no bias to the norm.
__device__ __forceinline__ float2 cmac2_hl(float2 ah, float2 al, float2 x, float2 bh, float2 bl,
                                           float2 y) {
  float re = al.x * x.x;
  re = fmaf(-al.y, x.y, re);
  re = fmaf(bl.x, y.x, re);
  re = fmaf(-bl.y, y.y, re);
  re = fmaf(ah.x, x.x, re);
  re = fmaf(-ah.y, x.y, re);
  re = fmaf(bh.x, y.x, re);
  re = fmaf(-bh.y, y.y, re);
  float im = al.x * x.y;
  im = fmaf(al.y, x.x, im);
  im = fmaf(bl.x, y.y, im);
  im = fmaf(bl.y, y.x, im);
  im = fmaf(ah.x, x.y, im);
  im = fmaf(ah.y, x.x, im);
  im = fmaf(bh.x, y.y, im);
  im = fmaf(bh.y, y.x, im);
  return make_float2(re, im);
}

// ------------------------------------------------------------ butterflies
// T: local position of the target; C: local position of the control or -1.

struct Coef {
  float2 h[4], l[4];
};

template <int T, int C>
__device__ __forceinline__ void dense_t(float2 (&a)[16], const Coef& m) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int j0 = ((p >> T) << (T + 1)) | (p & ((1 << T) - 1));
    const int j1 = j0 | (1 << T);
    if (C >= 0 && !((j0 >> C) & 1)) continue;
    const float2 x0 = a[j0], x1 = a[j1];
    a[j0] = cmac2_hl(m.h[0], m.l[0], x0, m.h[1], m.l[1], x1);
    a[j1] = cmac2_hl(m.h[2], m.l[2], x0, m.h[3], m.l[3], x1);
  }
}

// Hadamard butterfly without its 2^-1/2 (restored by the pass scale).
template <int T>
__device__ __forceinline__ void h_t(float2 (&a)[16]) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int j0 = ((p >> T) << (T + 1)) | (p & ((1 << T) - 1));
    const int j1 = j0 | (1 << T);
    const float2 x0 = a[j0], x1 = a[j1];
    a[j0] = make_float2(x0.x + x1.x, x0.y + x1.y);
    a[j1] = make_float2(x0.x - x1.x, x0.y - x1.y);
  }
}

template <int T, int C>
__device__ __forceinline__ void anti_t(float2 (&a)[16], float2 m01, float2 m10) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int j0 = ((p >> T) << (T + 1)) | (p & ((1 << T) - 1));
    const int j1 = j0 | (1 << T);
    if (C >= 0 && !((j0 >> C) & 1)) continue;
    const float2 x0 = a[j0], x1 = a[j1];
    a[j0] = cmul(m01, x1);
    a[j1] = cmul(m10, x0);
  }
}

template <int T, int C>
__device__ __forceinline__ void swap_t(float2 (&a)[16]) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int j0 = ((p >> T) << (T + 1)) | (p & ((1 << T) - 1));
    const int j1 = j0 | (1 << T);
    if (C >= 0 && !((j0 >> C) & 1)) continue;
    const float2 x0 = a[j0];
    a[j0] = a[j1];
    a[j1] = x0;
  }
}

// Controlled diagonal with both qubits local.
template <int T, int C>
__device__ __forceinline__ void diag_t(float2 (&a)[16], float2 d0, float2 d1) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (C >= 0 && !((j >> C) & 1)) continue;
    a[j] = cmul(a[j], ((j >> T) & 1) ? d1 : d0);
  }
}

template <int B>
__device__ __forceinline__ void scale_bit(float2 (&a)[16], float2 ph) {
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if ((j >> B) & 1) a[j] = cmul(a[j], ph);
}

#define TQS_DISPATCH_TC(FN, ARGS)   \
  switch (sel) {                    \
    case 0: FN<0, -1> ARGS; break;  \
    case 2: FN<0, 1> ARGS; break;   \
    case 3: FN<0, 2> ARGS; break;   \
    case 4: FN<0, 3> ARGS; break;   \
    case 5: FN<1, -1> ARGS; break;  \
    case 6: FN<1, 0> ARGS; break;   \
    case 8: FN<1, 2> ARGS; break;   \
    case 9: FN<1, 3> ARGS; break;   \
    case 10: FN<2, -1> ARGS; break; \
    case 11: FN<2, 0> ARGS; break;  \
    case 12: FN<2, 1> ARGS; break;  \
    case 14: FN<2, 3> ARGS; break;  \
    case 15: FN<3, -1> ARGS; break; \
    case 16: FN<3, 0> ARGS; break;  \
    case 17: FN<3, 1> ARGS; break;  \
    case 18: FN<3, 2> ARGS; break;  \
    default: break;                 \
  }

// Pending per-bit phases: a diagonal factor that depends on one local bit is
// folded into ph[b] (applied to the amplitudes with local bit b = 1) and only
// multiplied in before a non-diagonal factor on bit b, or at the end of the
// pass.  Factors that depend on far bits only fold into the scalar `sc`.
struct Pending {
  float2 p0, p1, p2, p3;
  unsigned dirty;
};

__device__ __forceinline__ void pend_mul(Pending& pd, int b, float2 v) {
  switch (b) {
    case 0: pd.p0 = cmul(pd.p0, v); break;
    case 1: pd.p1 = cmul(pd.p1, v); break;
    case 2: pd.p2 = cmul(pd.p2, v); break;
    default: pd.p3 = cmul(pd.p3, v); break;
  }
  pd.dirty |= 1u << b;
}

__device__ __forceinline__ void pend_flush(float2 (&a)[16], Pending& pd, int b) {
  if (!((pd.dirty >> b) & 1)) return;
  const float2 one = make_float2(1.f, 0.f);
  switch (b) {
    case 0: scale_bit<0>(a, pd.p0); pd.p0 = one; break;
    case 1: scale_bit<1>(a, pd.p1); pd.p1 = one; break;
    case 2: scale_bit<2>(a, pd.p2); pd.p2 = one; break;
    default: scale_bit<3>(a, pd.p3); pd.p3 = one; break;
  }
  pd.dirty &= ~(1u << b);
}

__device__ __forceinline__ float2 f2(unsigned x, unsigned y) {
  return make_float2(__uint_as_float(x), __uint_as_float(y));
}

// Apply the ops of one pass to the 16 amplitudes of one group, then the
// pass's exact power-of-two scale.
__device__ __forceinline__ void run_ops(float2 (&a)[16], const FusedOp* __restrict__ ops,
                                        uint32_t count, int base, float scale) {
  Pending pd;
  pd.p0 = pd.p1 = pd.p2 = pd.p3 = make_float2(1.f, 0.f);
  pd.dirty = 0;
  float2 sc = make_float2(1.f, 0.f);
  bool sc_set = false;
  for (uint32_t k = 0; k < count; ++k) {
    const uint4* rec = reinterpret_cast<const uint4*>(ops + k);
    const uint4 q0 = __ldg(rec);
    const int kind = q0.x & 0xff;
    const int tloc = (q0.x >> 8) & 0xff;
    const int t = (q0.x >> 16) & 0xff;
    const int ckind = q0.x >> 24;
    const int c = q0.y & 0xff;
    const int unit = (q0.y >> 8) & 0xff;
    if (kind == OP_H) {
      pend_flush(a, pd, t);
      switch (t) {
        case 0: h_t<0>(a); break;
        case 1: h_t<1>(a); break;
        case 2: h_t<2>(a); break;
        default: h_t<3>(a); break;
      }
      continue;
    }
    const uint4 q1 = __ldg(rec + 1);
    const uint4 q2 = __ldg(rec + 2);
    const float2 m0 = f2(q1.x, q1.y);
    const float2 m1 = f2(q1.z, q1.w);
    const float2 m2 = f2(q2.x, q2.y);
    if (kind == OP_DIAG) {
      // d0 = m0, d1 = m1, ratio d1/d0 = m2
      if (tloc) {
        if (ckind == CTL_LOCAL) {
          const int sel = t * 5 + c + 1;
          TQS_DISPATCH_TC(diag_t, (a, m0, m1));
        } else if (ckind == CTL_NONE || ((base >> c) & 1)) {
          sc = cmul(sc, m0);
          sc_set = true;
          pend_mul(pd, t, m2);
        }
      } else {
        const float2 v = ((base >> t) & 1) ? m1 : m0;
        if (ckind == CTL_LOCAL) {
          pend_mul(pd, c, v);
        } else if (ckind == CTL_NONE || ((base >> c) & 1)) {
          sc = cmul(sc, v);
          sc_set = true;
        }
      }
      continue;
    }
    if (ckind == CTL_FAR && !((base >> c) & 1)) continue;
    pend_flush(a, pd, t);
    const int sel = t * 5 + (ckind == CTL_LOCAL ? c : -1) + 1;
    if (kind == OP_DENSE) {
      const uint4 q3 = __ldg(rec + 3);
      const uint4 q4 = __ldg(rec + 4);
      Coef m;
      m.h[0] = m0;
      m.h[1] = m1;
      m.h[2] = m2;
      m.h[3] = f2(q2.z, q2.w);
      m.l[0] = f2(q3.x, q3.y);
      m.l[1] = f2(q3.z, q3.w);
      m.l[2] = f2(q4.x, q4.y);
      m.l[3] = f2(q4.z, q4.w);
      TQS_DISPATCH_TC(dense_t, (a, m));
    } else if (unit) {
      TQS_DISPATCH_TC(swap_t, (a));
    } else {
      TQS_DISPATCH_TC(anti_t, (a, m1, m2));
    }
  }
  pend_flush(a, pd, 0);
  pend_flush(a, pd, 1);
  pend_flush(a, pd, 2);
  pend_flush(a, pd, 3);
  if (sc_set) {
    sc.x *= scale;  // exact: scale is a power of two
    sc.y *= scale;
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = cmul(a[j], sc);
  } else if (scale != 1.0f) {
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = make_float2(a[j].x * scale, a[j].y * scale);
  }
}

template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if (TEAM == TEAM_WARP)
    __syncwarp();
  else
    __syncthreads();
}

template <int TEAM>
__device__ void run_circuit(const FusedLaunch& L, int ci, float2* st, int rank, int size,
                            double* s_red) {
  const FusedCirc cd = L.circs[ci];
  const int nint = cd.nint;
  const int n = cd.n;
  const int G = 1 << (nint - 4);
  const float2* init = cd.init;

  if (init != nullptr) {
    const int NI = 1 << nint, N = 1 << n;
    for (int i = rank; i < NI; i += size)
      st[swz(i)] = (i < N) ? init[i] : make_float2(0.f, 0.f);
    team_sync<TEAM>();
  }

  for (int p = 0; p < cd.pass_count; ++p) {
    const uint4 pr = __ldg(reinterpret_cast<const uint4*>(L.passes + cd.pass_begin + p));
    const int l0 = pr.x & 0xff, l1 = (pr.x >> 8) & 0xff, l2 = (pr.x >> 16) & 0xff,
              l3 = pr.x >> 24;
    const FusedOp* ops = L.ops + pr.y;
    const uint32_t count = pr.z;
    const float scale = __uint_as_float(pr.w);
    const bool gen = (p == 0) && (init == nullptr);
    const int b0 = 1 << l0, b1 = 1 << l1, b2 = 1 << l2, b3 = 1 << l3;
    for (int g = rank; g < G; g += size) {
      int base = ins0(ins0(ins0(ins0(g, l0), l1), l2), l3);
      float2 a[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int off = base + ((j & 1) ? b0 : 0) + ((j & 2) ? b1 : 0) + ((j & 4) ? b2 : 0) +
                        ((j & 8) ? b3 : 0);
        if (gen)
          a[j] = make_float2(off == 0 ? 1.f : 0.f, 0.f);
        else
          a[j] = st[swz(off)];
      }
      run_ops(a, ops, count, base, scale);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int off = base + ((j & 1) ? b0 : 0) + ((j & 2) ? b1 : 0) + ((j & 4) ? b2 : 0) +
                        ((j & 8) ? b3 : 0);
        st[swz(off)] = a[j];
      }
    }
    team_sync<TEAM>();
  }

  // Output: logical index i holds the amplitude at physical index P(i).
  const int N = 1 << n;
  const uint4 posw = *reinterpret_cast<const uint4*>(cd.pos);
  const unsigned pw[4] = {posw.x, posw.y, posw.z, posw.w};
  float2* out = L.out + cd.out_off;
  double* probs = L.probs ? L.probs + cd.out_off : nullptr;
  const float oscale = cd.out_scale;
  double acc = 0.0;
  for (int i = rank * 2; i < N; i += size * 2) {
    int p0 = i, p1 = i + 1;
    if (!cd.identity) {
      p0 = 0;
      p1 = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (q < n) {
          const int b = (pw[q >> 2] >> ((q & 3) * 8)) & 0xff;
          p0 |= ((i >> q) & 1) << b;
          p1 |= (((i + 1) >> q) & 1) << b;
        }
      }
    }
    float2 v0 = st[swz(p0)];
    float2 v1 = st[swz(p1)];
    if (oscale != 1.0f) {
      v0 = make_float2(v0.x * oscale, v0.y * oscale);
      v1 = make_float2(v1.x * oscale, v1.y * oscale);
    }
    *reinterpret_cast<float4*>(out + i) = make_float4(v0.x, v0.y, v1.x, v1.y);
    // |psi|^2 in FP64: the squares of the FP32 parts are exact in FP64.
    const double x0 = v0.x, y0 = v0.y, x1 = v1.x, y1 = v1.y;
    const double q0 = fma(x0, x0, y0 * y0);
    const double q1 = fma(x1, x1, y1 * y1);
    if (probs) *reinterpret_cast<double2*>(probs + i) = make_double2(q0, q1);
    acc += q0 + q1;
  }
  // Fixed-order reduction (deterministic).
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (TEAM == TEAM_WARP) {
    if (rank == 0 && L.norms) L.norms[ci] = acc;
  } else {
    const int warp = rank >> 5, lane = rank & 31;
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    if (rank == 0) {
      double s = 0.0;
      for (int w = 0; w < (size >> 5); ++w) s += s_red[w];
      if (L.norms) L.norms[ci] = s;
    }
  }
  team_sync<TEAM>();
}

template <int TEAM>
__global__ void __launch_bounds__(TEAM == TEAM_CTA ? kCtaThreads : 512)
    fused_kernel(const __grid_constant__ FusedLaunch L) {
  extern __shared__ float4 smem_raw[];
  float2* smem = reinterpret_cast<float2*>(smem_raw);
  if (TEAM == TEAM_WARP) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* st = smem + (static_cast<size_t>(warp) << L.slice_q);
    for (;;) {
      int job = 0;
      if (lane == 0) job = atomicAdd(L.counter, 1);
      job = __shfl_sync(0xffffffffu, job, 0);
      if (job >= L.n_jobs) break;
      run_circuit<TEAM_WARP>(L, L.order[job], st, lane, 32, nullptr);
    }
  } else {
    __shared__ int s_job;
    __shared__ double s_red[32];
    float2* st = (TEAM == TEAM_CTA)
                     ? smem
                     : L.gscratch + (static_cast<size_t>(blockIdx.x) << kGlobalSlotQ);
    for (;;) {
      if (threadIdx.x == 0) s_job = atomicAdd(L.counter, 1);
      __syncthreads();
      const int job = s_job;
      __syncthreads();
      if (job >= L.n_jobs) break;
      run_circuit<TEAM>(L, L.order[job], st, threadIdx.x, blockDim.x, s_red);
    }
  }
}

size_t fused_smem_bytes(int team, int warps_per_cta, int slice_q) {
  if (team == TEAM_WARP) return (static_cast<size_t>(warps_per_cta) << slice_q) * sizeof(float2);
  if (team == TEAM_CTA) return (static_cast<size_t>(1) << slice_q) * sizeof(float2);
  return 0;
}

int fused_threads(int team, int warps_per_cta) {
  if (team == TEAM_WARP) return 32 * warps_per_cta;
  if (team == TEAM_CTA) return kCtaThreads;
  return kGlobalThreads;
}

}  // namespace

int fused_max_ctas_per_sm(int team, int warps_per_cta, int slice_q) {
  const size_t smem = fused_smem_bytes(team, warps_per_cta, slice_q);
  const int threads = fused_threads(team, warps_per_cta);
  int blocks = 0;
  cudaError_t e;
  if (team == TEAM_WARP) {
    cudaFuncSetAttribute(fused_kernel<TEAM_WARP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fused_kernel<TEAM_WARP>, threads,
                                                      smem);
  } else if (team == TEAM_CTA) {
    cudaFuncSetAttribute(fused_kernel<TEAM_CTA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fused_kernel<TEAM_CTA>, threads,
                                                      smem);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fused_kernel<TEAM_GLOBAL>, threads,
                                                      smem);
  }
  if (e != cudaSuccess) return 0;
  return blocks;
}

cudaError_t launch_fused(const FusedLaunch& L, cudaStream_t s) {
  if (L.n_jobs <= 0) return cudaSuccess;
  const size_t smem = fused_smem_bytes(L.team, L.warps_per_cta, L.slice_q);
  const int threads = fused_threads(L.team, L.warps_per_cta);
  cudaError_t e = cudaSuccess;
  if (L.team == TEAM_WARP) {
    e = cudaFuncSetAttribute(fused_kernel<TEAM_WARP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    fused_kernel<TEAM_WARP><<<L.grid, threads, smem, s>>>(L);
  } else if (L.team == TEAM_CTA) {
    e = cudaFuncSetAttribute(fused_kernel<TEAM_CTA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    fused_kernel<TEAM_CTA><<<L.grid, threads, smem, s>>>(L);
  } else {
    fused_kernel<TEAM_GLOBAL><<<L.grid, threads, 0, s>>>(L);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tqs
