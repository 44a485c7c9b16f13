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
// order, |psi_i|^2 (FP32 arithmetic, or exact in FP64) stored as FP64, and
// the FP64 norm.  A circuit that starts from a basis state works, in each
// pass, only the groups of 16 amplitudes that can be nonzero by then (the
// support rule in run_circuit); the rest of its state is zero.
//
// Teams: one warp or a pair of warps per circuit (n <= 11), one 512-thread CTA
// per circuit (n <= 14), one CTA on global scratch (n <= 16), or several
// cooperating CTAs on global scratch for a few 15-16 qubit circuits
// (TEAM_MULTI).  Warps/CTAs pull circuits from an atomic job counter
// (costliest first), so one persistent launch runs a whole batch.
#include "checked.h"
#include "exact_sq.h"
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

// The low bits of x spread over the set bits of mask, lowest first (a bit
// deposit: bit k of x lands on the k-th set bit of mask).
__device__ __forceinline__ int deposit_bits(int x, int mask) {
  int r = 0;
  while (mask != 0) {
    const int b = mask & -mask;
    if (x & 1) r |= b;
    x >>= 1;
    mask ^= b;
  }
  return r;
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
// T: local position of the target.  `act` is a 16-bit mask over the local
// amplitude index: the op acts on the pairs whose j0 bit is set in it (all
// ones when uncontrolled, the control-bit-1 half for a local control).

struct Coef {
  float2 h[4], l[4];
};

__device__ __forceinline__ float2 sel(bool on, float2 y, float2 x) {
  return make_float2(on ? y.x : x.x, on ? y.y : x.y);
}

// CTRL = false: every pair (an uncontrolled factor, no selects).
template <int T, bool CTRL>
__device__ __forceinline__ void dense_t(float2 (&a)[16], const Coef& m, unsigned act) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int j0 = ((p >> T) << (T + 1)) | (p & ((1 << T) - 1));
    const int j1 = j0 | (1 << T);
    const float2 x0 = a[j0], x1 = a[j1];
    if (CTRL) {
      const bool on = (act >> j0) & 1;
      a[j0] = sel(on, cmac2_hl(m.h[0], m.l[0], x0, m.h[1], m.l[1], x1), x0);
      a[j1] = sel(on, cmac2_hl(m.h[2], m.l[2], x0, m.h[3], m.l[3], x1), x1);
    } else {
      a[j0] = cmac2_hl(m.h[0], m.l[0], x0, m.h[1], m.l[1], x1);
      a[j1] = cmac2_hl(m.h[2], m.l[2], x0, m.h[3], m.l[3], x1);
    }
  }
}




template <int T>
__device__ __forceinline__ void swap_t(float2 (&a)[16], unsigned act) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int j0 = ((p >> T) << (T + 1)) | (p & ((1 << T) - 1));
    const int j1 = j0 | (1 << T);
    const bool on = (act >> j0) & 1;
    const float2 x0 = a[j0], x1 = a[j1];
    a[j0] = sel(on, x1, x0);
    a[j1] = sel(on, x0, x1);
  }
}

// Hadamard butterfly without its 2^-1/2 (restored by the pass scale):
// x0 <- x0 + x1, then x1 <- x0' - 2 x1 (= x0 - x1 up to one more rounding of
// the sum), so each output overwrites an input that is no longer needed and
// the butterfly needs no temporary registers.
template <int T>
__device__ __forceinline__ void h_t(float2 (&a)[16]) {
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int j0 = ((p >> T) << (T + 1)) | (p & ((1 << T) - 1));
    const int j1 = j0 | (1 << T);
    // packed FP32x2 (both parts in one instruction; each rounded as the
    // scalar operation would be)
    a[j0] = __fadd2_rn(a[j0], a[j1]);
    a[j1] = __ffma2_rn(make_float2(-2.f, -2.f), a[j1], a[j0]);
  }
}

// a <- a b in place: both products that need the old a.y are formed first,
// so the results overwrite a.x and a.y without a temporary copy.
__device__ __forceinline__ void cmul_in(float2& a, float2 b) {
  const float t = a.y * b.y, u = a.y * b.x;
  a.y = fmaf(a.x, b.y, u);
  a.x = fmaf(a.x, b.x, -t);
}

template <int B>
__device__ __forceinline__ void scale_bit(float2 (&a)[16], float2 ph) {
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if ((j >> B) & 1) cmul_in(a[j], ph);
}

// 16-bit masks of the local indices j whose bit b is set.
__device__ __forceinline__ unsigned bit_mask(int b) {
  return b == 0 ? 0xAAAAu : b == 1 ? 0xCCCCu : b == 2 ? 0xF0F0u : 0xFF00u;
}

// Controlled diagonal with both qubits local: amplitudes with the control bit
// set are multiplied by d0 (target 0) or d1 (target 1); when d0 is exactly 1
// only the control = target = 1 quarter changes.
__device__ __forceinline__ void diag_local(float2 (&a)[16], int t, int c, float2 d0, float2 d1,
                                           bool d0one) {
  const unsigned cm = bit_mask(c), tm = bit_mask(t);
  const unsigned on = d0one ? (cm & tm) : cm;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if ((on >> j) & 1) a[j] = cmul(a[j], ((tm >> j) & 1) ? d1 : d0);
  }
}

// The common controlled phase (d0 exactly 1) with both qubits local: only the
// four amplitudes with local bits T and C both set change.  Compile-time
// positions, so no predicated work on the other twelve.
template <int T, int C>
__device__ __forceinline__ void phase_tc(float2 (&a)[16], float2 d1) {
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (((j >> T) & 1) && ((j >> C) & 1)) cmul_in(a[j], d1);
}

__device__ __forceinline__ void phase_local(float2 (&a)[16], int t, int c, float2 d1) {
  switch (t * 4 + c) {
    case 1: phase_tc<0, 1>(a, d1); break;
    case 2: phase_tc<0, 2>(a, d1); break;
    case 3: phase_tc<0, 3>(a, d1); break;
    case 4: phase_tc<1, 0>(a, d1); break;
    case 6: phase_tc<1, 2>(a, d1); break;
    case 7: phase_tc<1, 3>(a, d1); break;
    case 8: phase_tc<2, 0>(a, d1); break;
    case 9: phase_tc<2, 1>(a, d1); break;
    case 11: phase_tc<2, 3>(a, d1); break;
    case 12: phase_tc<3, 0>(a, d1); break;
    case 13: phase_tc<3, 1>(a, d1); break;
    default: phase_tc<3, 2>(a, d1); break;
  }
}

// Pending per-bit phases: a diagonal factor that depends on one local bit is
// folded into p[b] (applied to the amplitudes with local bit b = 1) and only
// multiplied in before a non-diagonal factor on bit b, or at the end of the
// pass.  Factors that depend on far bits only fold into the scalar `sc`.
struct Pending {
  float2 p[4];  // indexed with compile-time positions only
  unsigned dirty;
};

__device__ __forceinline__ void pend_mul(Pending& pd, int b, float2 v) {
  switch (b) {
    case 0: pd.p[0] = cmul(pd.p[0], v); break;
    case 1: pd.p[1] = cmul(pd.p[1], v); break;
    case 2: pd.p[2] = cmul(pd.p[2], v); break;
    default: pd.p[3] = cmul(pd.p[3], v); break;
  }
  pd.dirty |= 1u << b;
}

__device__ __forceinline__ void pend_flush(float2 (&a)[16], Pending& pd, int b) {
  if (!((pd.dirty >> b) & 1)) return;
  const float2 one = make_float2(1.f, 0.f);
  switch (b) {
    case 0: scale_bit<0>(a, pd.p[0]); pd.p[0] = one; break;
    case 1: scale_bit<1>(a, pd.p[1]); pd.p[1] = one; break;
    case 2: scale_bit<2>(a, pd.p[2]); pd.p[2] = one; break;
    default: scale_bit<3>(a, pd.p[3]); pd.p[3] = one; break;
  }
  pd.dirty &= ~(1u << b);
}



__device__ __forceinline__ float2 f2(unsigned x, unsigned y) {
  return make_float2(__uint_as_float(x), __uint_as_float(y));
}

// Apply the ops of one pass to the 16 amplitudes of one group, then the
// pass's exact power-of-two scale.  The next op's header is fetched while the
// current one runs.
// SPLIT_DENSE: uncontrolled dense factors take a select-free copy of the
// butterfly (more code; the full-state-vector tiles and the CTA-sized teams,
// dominated by dense single-qubit factors, use it; the warp and pair teams
// keep one copy, measured faster on the paper-shaped circuits).
template <bool SPLIT_DENSE>
__device__ __forceinline__ void run_ops(float2 (&a)[16], const FusedOp* __restrict__ ops,
                                        uint32_t count, int base, float scale) {
  Pending pd;
#pragma unroll
  for (int b = 0; b < 4; ++b) pd.p[b] = make_float2(1.f, 0.f);
  pd.dirty = 0;
  float2 sc = make_float2(1.f, 0.f);
  bool sc_set = false;
  uint4 next = count ? __ldg(reinterpret_cast<const uint4*>(ops)) : make_uint4(0, 0, 0, 0);
  for (uint32_t k = 0; k < count; ++k) {
    const uint4* rec = reinterpret_cast<const uint4*>(ops + k);
    const uint4 q0 = next;
    if (k + 1 < count) next = __ldg(reinterpret_cast<const uint4*>(ops + k + 1));
    const int code = q0.x & 0xff;
    const int fbit = (q0.y >> 8) & 0xff;
    if (fbit != 0xff && !((base >> fbit) & 1)) continue;  // a far control is 0 here
    if (code < OPC_DLN) {
      // non-diagonal: target local position t
      int t = code & 3;
      unsigned act = q0.y >> 16;
      if (code >= OPC_XL && code < OPC_ANTI) {
        t = (code - OPC_XL) >> 2;
        act = bit_mask((code - OPC_XL) & 3);
      }
      if (code < OPC_X) {
        pend_flush(a, pd, t);
        switch (t) {
          case 0: h_t<0>(a); break;
          case 1: h_t<1>(a); break;
          case 2: h_t<2>(a); break;
          default: h_t<3>(a); break;
        }
      } else if (code < OPC_ANTI) {
        pend_flush(a, pd, t);
        switch (t) {
          case 0: swap_t<0>(a, act); break;
          case 1: swap_t<1>(a, act); break;
          case 2: swap_t<2>(a, act); break;
          default: swap_t<3>(a, act); break;
        }
      } else if (code == OPC_HMASK) {
        // Hadamards on several local positions, one dispatch
        const int hm = (q0.x >> 8) & 15;
        if (hm & 1) { pend_flush(a, pd, 0); h_t<0>(a); }
        if (hm & 2) { pend_flush(a, pd, 1); h_t<1>(a); }
        if (hm & 4) { pend_flush(a, pd, 2); h_t<2>(a); }
        if (hm & 8) { pend_flush(a, pd, 3); h_t<3>(a); }
      } else if (code == OPC_XP) {
        // exchanges on one position under a parity of local and far bits
        const int tt = (q0.x >> 8) & 3;
        unsigned act2 = q0.y >> 16;
        if (__popc(static_cast<unsigned>(base) & q0.z) & 1) act2 ^= 0xFFFFu;
        pend_flush(a, pd, tt);
        switch (tt) {
          case 0: swap_t<0>(a, act2); break;
          case 1: swap_t<1>(a, act2); break;
          case 2: swap_t<2>(a, act2); break;
          default: swap_t<3>(a, act2); break;
        }
      } else {
        pend_flush(a, pd, t);
        const uint4 q1 = __ldg(rec + 1);
        const uint4 q2 = __ldg(rec + 2);
        const uint4 q3 = __ldg(rec + 3);
        const uint4 q4 = __ldg(rec + 4);
        Coef m;
        m.h[0] = f2(q1.x, q1.y);
        m.h[1] = f2(q1.z, q1.w);
        m.h[2] = f2(q2.x, q2.y);
        m.h[3] = f2(q2.z, q2.w);
        m.l[0] = f2(q3.x, q3.y);
        m.l[1] = f2(q3.z, q3.w);
        m.l[2] = f2(q4.x, q4.y);
        m.l[3] = f2(q4.z, q4.w);
        if (SPLIT_DENSE && code < OPC_CDENSE) {
          switch (t) {
            case 0: dense_t<0, false>(a, m, act); break;
            case 1: dense_t<1, false>(a, m, act); break;
            case 2: dense_t<2, false>(a, m, act); break;
            default: dense_t<3, false>(a, m, act); break;
          }
        } else {
          switch (t) {
            case 0: dense_t<0, true>(a, m, act); break;
            case 1: dense_t<1, true>(a, m, act); break;
            case 2: dense_t<2, true>(a, m, act); break;
            default: dense_t<3, true>(a, m, act); break;
          }
        }
      }
      continue;
    }
    if (code >= OPC_DIAG16) {
      if (code == OPC_DIAG16) {
        // entry j multiplies amplitude j: 0..7 here, 8..15 in the next record
        const uint4 q1 = __ldg(rec + 1), q2 = __ldg(rec + 2), q3 = __ldg(rec + 3), q4 = __ldg(rec + 4);
        const uint4 r1 = __ldg(rec + 6), r2 = __ldg(rec + 7), r3 = __ldg(rec + 8), r4 = __ldg(rec + 9);
        const uint4 w[8] = {q1, q2, q3, q4, r1, r2, r3, r4};
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint4 v = w[j >> 1];
          cmul_in(a[j], (j & 1) ? f2(v.z, v.w) : f2(v.x, v.y));
        }
        // skip the second record (and fetch the header after it)
        ++k;
        if (k + 1 < count) next = __ldg(reinterpret_cast<const uint4*>(ops + k + 1));
      }
      if (code == OPC_DLISTM) {
        // phase lists of several targets over the same factor bits: the bits
        // are tested once, then each target's product (8 factors, padded with
        // (0xFF, 1)) goes into its pending factor or the group's scalar
        const unsigned tmask = (q0.x >> 8) & 31;
        const unsigned fb[2] = {q0.z, q0.w};
        bool on[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int f = (fb[e >> 2] >> (8 * (e & 3))) & 0xff;
          on[e] = f == 0xff || ((base >> f) & 1);
        }
        const float2 one = make_float2(1.f, 0.f);
        int rc = 0;
#pragma unroll
        for (int t = 0; t < 5; ++t) {
          if (!((tmask >> t) & 1)) continue;
          const uint4* rr = rec + 5 * rc;
          const uint4 w[4] = {__ldg(rr + 1), __ldg(rr + 2), __ldg(rr + 3), __ldg(rr + 4)};
          float2 acc = one;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint4 x = w[e >> 1];
            const float2 v = (e & 1) ? f2(x.z, x.w) : f2(x.x, x.y);
            acc = cmul(acc, on[e] ? v : one);
          }
          if (t < 4) {
            pd.p[t] = cmul(pd.p[t], acc);
            pd.dirty |= 1u << t;
          } else {
            sc = cmul(sc, acc);
            sc_set = true;
          }
          ++rc;
        }
        // skip the continuation records (and fetch the header after them)
        if (rc > 1) {
          k += rc - 1;
          if (k + 1 < count) next = __ldg(reinterpret_cast<const uint4*>(ops + k + 1));
        }
      }
      continue;  // OPC_NOP: a continuation record, skipped by its op
    }
    if (code == OPC_DLIST) {
      // up to 8 phase factors, each on when its physical bit of the group is
      // set (byte 0xFF: always), multiplied into the pending factor of one
      // local position or into the group's scalar
      // the list is padded to 4 or 8 factors with (0xFF, 1): no per-factor guard
      const int tgt = (q0.x >> 8) & 0xff, cnt = (q0.x >> 16) & 0xff;
      const uint4 q1 = __ldg(rec + 1), q2 = __ldg(rec + 2);
      float2 acc = make_float2(1.f, 0.f);
      const float2 one = make_float2(1.f, 0.f);
      const unsigned fb[2] = {q0.z, q0.w};
      const uint4 qv[2] = {q1, q2};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int f = (fb[0] >> (8 * e)) & 0xff;
        const bool on = f == 0xff || ((base >> f) & 1);
        const uint4 w = qv[e >> 1];
        const float2 v = (e & 1) ? f2(w.z, w.w) : f2(w.x, w.y);
        acc = cmul(acc, on ? v : one);
      }
      if (cnt > 4) {
        const uint4 q3 = __ldg(rec + 3), q4 = __ldg(rec + 4);
        const uint4 qw[2] = {q3, q4};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int f = (fb[1] >> (8 * e)) & 0xff;
          const bool on = f == 0xff || ((base >> f) & 1);
          const uint4 w = qw[e >> 1];
          const float2 v = (e & 1) ? f2(w.z, w.w) : f2(w.x, w.y);
          acc = cmul(acc, on ? v : one);
        }
      }
      if (tgt < 4) {
        pend_mul(pd, tgt, acc);
      } else {
        sc = cmul(sc, acc);
        sc_set = true;
      }
      continue;
    }
    // diagonal ops: d0 = m0, d1 = m1, ratio d1/d0 = m2; the header's hc holds
    // d1/d0 (local target, no local control) or d1 (the rest), so only ops
    // whose d0 is not exactly 1 load more than the header
    const bool d0one = (q0.y & 0xff) != 0;
    const float2 hc = f2(q0.z, q0.w);
    if (code < OPC_DFL) {  // local target, no or far control
      if (!d0one) {
        const uint4 q1 = __ldg(rec + 1);
        sc = cmul(sc, f2(q1.x, q1.y));
        sc_set = true;
      }
      pend_mul(pd, code & 3, hc);
      continue;
    }
    const bool tb = (base >> ((q0.x >> 24) & 0xff)) & 1;
    if (code <= OPC_DFF) {  // far target: local control c (DFL) or none / far (DFF)
      if (!tb && d0one) continue;
      float2 v = hc;
      if (!tb) {
        const uint4 q1 = __ldg(rec + 1);
        v = f2(q1.x, q1.y);
      }
      if (code < OPC_DFF) {
        pend_mul(pd, code & 3, v);
      } else {  // a phase of the group
        sc = cmul(sc, v);
        sc_set = true;
      }
      continue;
    }
    {  // OPC_DLL: both local
      const int t = (q0.x >> 8) & 0xff, c = (q0.x >> 16) & 0xff;
      if (d0one) {
        phase_local(a, t, c, hc);
      } else {
        const uint4 q1 = __ldg(rec + 1);
        diag_local(a, t, c, f2(q1.x, q1.y), hc, false);
      }
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
    const float2 s2 = make_float2(scale, scale);
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = __fmul2_rn(a[j], s2);
  }
}

// |v|^2 correctly rounded to FP64 (exact_sq.h).
__device__ __forceinline__ double prob_f64(float2 v) { return sq_sum_f64(v.x, v.y); }

// The output map's linear part (FusedCirc::col): the XOR of col[q] over the
// set bits q of v, v < 2^n.
__device__ __forceinline__ int map_lin(const FusedCirc* c, int v, int n) {
  int r = 0;
  for (int q = 0; q < n; ++q)
    if ((v >> q) & 1) r ^= __ldg(&c->col[q]);
  return r;
}
// Prefetch [p, p + bytes) into L1, one 128-byte line per thread of the team.
__device__ __forceinline__ void prefetch_l1_range(const void* p, size_t bytes, int rank, int size) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t end = a + bytes;
  for (uintptr_t l = (a & ~uintptr_t(127)) + uintptr_t(rank) * 128; l < end; l += uintptr_t(size) * 128)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(l));
}

// Barrier of the threads working on one circuit: the warp, the warp pair
// (named barrier 1 + pair index, 64 threads) or the CTA.
template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if (TEAM == TEAM_WARP)
    __syncwarp();
  else if (TEAM == TEAM_PAIR)
    asm volatile("bar.sync %0, 64;" ::"r"(1 + (static_cast<int>(threadIdx.x) >> 6)) : "memory");
  else
    __syncthreads();
}

// Barrier of the K TEAM_MULTI CTAs of one circuit (all co-resident:
// cooperative launch).  Thread 0 of each arrives on the circuit's monotone
// counter (zeroed before the launch) and waits, at most kGridBarrierCycles,
// until all K have arrived as often; a time-out is recorded and later
// barriers do not wait.
struct GridBar {
  unsigned int* ctr;
  int* err;
  unsigned int target;
  unsigned int nblocks;  // CTAs that meet at this barrier
  bool leader;           // the first of them: writes the outputs
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void grid_sync(GridBar& b) {
  __syncthreads();
  if (threadIdx.x == 0) {
    b.target += b.nblocks;
    __threadfence();
    atomicAdd(b.ctr, 1u);
    if (*reinterpret_cast<volatile int*>(b.err) == 0) {
      const long long t0 = clock64();
      while (ld_acquire_u32(b.ctr) < b.target) {
        if (clock64() - t0 > kGridBarrierCycles) {
          atomicExch(b.err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// State loads: TEAM_MULTI reads what other CTAs wrote, so it bypasses L1.
template <int TEAM>
__device__ __forceinline__ float2 ld_state(const float2* p) {
  if (TEAM == TEAM_MULTI) return __ldcg(p);
  return *p;
}

// Measure / reset instruction (Sec. 5.2 operation interface) on physical bit
// `bit`: S_0 / S_1 = the |psi|^2 mass with that bit 0 / 1 (FP64 exact squares,
// summed per thread in index order, then across the team in a fixed order),
// T = S_0 + S_1; the outcome is 0 iff u T < S_0.  The state is projected on
// the outcome and scaled by sqrt(T / S_b); a reset with outcome 1 moves the
// kept half to bit 0.  Any global scale the amplitudes carry cancels in
// S_b / T.
template <int TEAM>
__device__ __noinline__ void instr_pass(const FusedLaunch& L, int nint, int bit, bool reset, uint32_t k,
                           float2* st, int rank, int size, double* s_red) {
  const int half = 1 << (nint - 1);
  const int m = 1 << bit;
  double s0 = 0.0, s1 = 0.0;
  for (int j = rank; j < half; j += size) {
    const int i0 = ins0(j, bit);
    s0 += prob_f64(st[TQS_IX(swz(i0), 2 * half)]);
    s1 += prob_f64(st[TQS_IX(swz(i0 | m), 2 * half)]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (TEAM != TEAM_WARP) {
    const int warp = rank >> 5, lane = rank & 31, nw = size >> 5;
    team_sync<TEAM>();
    if (lane == 0) { s_red[2 * warp] = s0; s_red[2 * warp + 1] = s1; }
    team_sync<TEAM>();
    s0 = 0.0;
    s1 = 0.0;
    for (int w = 0; w < nw; ++w) { s0 += s_red[2 * w]; s1 += s_red[2 * w + 1]; }
    team_sync<TEAM>();
  }
  const double T = s0 + s1;
  int outcome = (L.uniforms[k] * T < s0) ? 0 : 1;
  if ((outcome ? s1 : s0) == 0.0) outcome ^= 1;  // u outside [0, 1): never pick an empty half
  const double sb = outcome ? s1 : s0;
  const float sc = sb > 0.0 ? static_cast<float>(sqrt(T / sb)) : 1.0f;
  if (rank == 0 && L.outcomes) L.outcomes[k] = outcome;
  const float2 zero = make_float2(0.f, 0.f);
  for (int j = rank; j < half; j += size) {
    const int a0 = TQS_IX(swz(ins0(j, bit)), 2 * half), a1 = TQS_IX(swz(ins0(j, bit) | m), 2 * half);
    const float2 v = outcome ? st[a1] : st[a0];
    const float2 w = make_float2(v.x * sc, v.y * sc);
    st[a0] = (outcome == 0 || reset) ? w : zero;
    st[a1] = (outcome == 1 && !reset) ? w : zero;
  }
  team_sync<TEAM>();
}

// Custom k-qubit unitary (Sec. 5.2 operation interface), 2 <= k <= 5 (the
// pass's scale word holds the mask of the k physical bits): the
// amplitudes fall into groups of G = 2^k whose indices differ only in the k
// physical bits; out[r] = sum_c M[r][c] in[c] per group (the per-gate update
// of eq. 12 widened to k qubits).  A warp takes 32 / G groups at a time, lane
// r of a group computing row r from the group's amplitudes (read by all its
// lanes) and the transposed coefficients (consecutive lanes, consecutive
// words); FP32 lo parts are accumulated before hi parts.  Warps work on
// disjoint groups; within a warp every read of a group precedes its writes.
// Physical index of matrix-local index j: bit t of j goes to bit (bits >> 5t) & 31.
__device__ __forceinline__ int wide_local(int j, int k, uint32_t bits) {
  int v = 0;
#pragma unroll
  for (int t = 0; t < kMaxCustomQubits; ++t)
    if (t < k) v |= ((j >> t) & 1) << ((bits >> (5 * t)) & 31);
  return v;
}

template <int TEAM>
__device__ __noinline__ void wide_pass(const FusedLaunch& L, int nint, int k, uint32_t coef_off,
                          uint32_t bits, uint32_t mask, float2* st, int rank, int size) {
  const int G = 1 << k;
  const int lane = rank & 31, warp = rank >> 5, nwarps = size >> 5;
  const int per_warp = 32 >> k;
  const int sub = lane >> k, r = lane & (G - 1);
  const int loc_r = wide_local(r, k, bits);
  const int ngroups = 1 << (nint - k);
  const float2* mh = L.coef + coef_off;
  const float2* ml = mh + G * G;
  for (int g0 = warp * per_warp; g0 < ngroups; g0 += nwarps * per_warp) {
    const int g = g0 + sub;
    const bool on = g < ngroups;
    int base = g;
    for (uint32_t m = mask; m != 0; m &= m - 1) base = ins0(base, __ffs(m) - 1);
    float ar = 0.f, ai = 0.f;  // lo products
    float br = 0.f, bi = 0.f;  // hi products
    if (on) {
      for (int c = 0; c < G; ++c) {
        const float2 x = st[TQS_IX(swz(base | wide_local(c, k, bits)), 1 << nint)];
        const float2 h = __ldg(mh + c * G + r), l = __ldg(ml + c * G + r);
        ar = fmaf(l.x, x.x, fmaf(-l.y, x.y, ar));
        ai = fmaf(l.x, x.y, fmaf(l.y, x.x, ai));
        br = fmaf(h.x, x.x, fmaf(-h.y, x.y, br));
        bi = fmaf(h.x, x.y, fmaf(h.y, x.x, bi));
      }
    }
    __syncwarp();
    if (on) st[TQS_IX(swz(base | loc_r), 1 << nint)] = make_float2(ar + br, ai + bi);
    __syncwarp();
  }
  team_sync<TEAM>();
}

template <int TEAM>
__device__ void run_circuit(const FusedLaunch& L, int ci, float2* st, int rank, int size,
                            double* s_red, int& next_job, int& next_ci, int* s_slot,
                            GridBar* bar = nullptr) {
  const FusedCirc cd = L.circs[ci];
  const int nint = cd.nint;
  const int n = cd.n;
  // The team brings the circuit's pass and op records into L1 together: one
  // L2 round trip, instead of one per op for the first group of each pass.
  prefetch_l1_range(L.passes + cd.pass_begin, cd.pass_count * sizeof(FusedPass), rank, size);
  prefetch_l1_range(L.ops + cd.op_begin, cd.op_count * sizeof(FusedOp), rank, size);
  const int G = 1 << (nint - 4);
  const float2* init = cd.init;
  if (init != nullptr) {
    const int NI = 1 << nint, N = 1 << n;
    for (int i = rank; i < NI; i += size)
      st[TQS_IX(swz(i), NI)] = (i < N) ? init[i] : make_float2(0.f, 0.f);
    if (TEAM == TEAM_MULTI) grid_sync(*bar); else team_sync<TEAM>();
  }
  // Support of a state started from the basis state |gen_index>: a register
  // pass mixes amplitudes only within its groups (indices that differ in its
  // local positions), so once the passes so far have had the positions T as
  // local ones, every amplitude whose index differs from gen_index in a bit
  // outside T is still exactly zero.  `touched` holds T (all ones: no such
  // knowledge, after an initial state, a measurement or a custom unitary).
  // A pass's groups whose far bits differ from gen_index outside T are zero
  // and stay zero under its ops, so the team works only the others: the
  // group counter is deposited into the far bits inside T, the far bits
  // outside T are those of gen_index.  The generation pass first writes
  // zeros over the whole state; later passes leave the zero groups as they are.
  int touched = init == nullptr ? 0 : -1;
  for (int p = 0; p < cd.pass_count; ++p) {
    const uint4 pr = __ldg(reinterpret_cast<const uint4*>(L.passes + cd.pass_begin + p));
    const int l0 = pr.x & 0xff, l1 = (pr.x >> 8) & 0xff, l2 = (pr.x >> 16) & 0xff, l3 = pr.x >> 24;
    if (l0 == kInstrPass) {
      instr_pass<TEAM>(L, nint, l1, (l2 & 1) != 0, pr.y, st, rank, size, s_red);
      touched = -1;
      continue;
    }
    if (l0 == kWidePass) {
      wide_pass<TEAM>(L, nint, l1, pr.y, pr.z, pr.w, st, rank, size);
      touched = -1;
      continue;
    }
    const FusedOp* ops = L.ops + pr.y;
    const uint32_t count = pr.z;
    const float scale = __uint_as_float(pr.w);
    const bool gen = (p == 0) && (init == nullptr);
    const int w0 = swz(1 << l0), w1 = swz(1 << l1), w2 = swz(1 << l2), w3 = swz(1 << l3);
    const int b0 = 1 << l0, b1 = 1 << l1, b2 = 1 << l2, b3 = 1 << l3;
    const int far = ((1 << nint) - 1) & ~(b0 | b1 | b2 | b3);
    const int free_far = far & touched;
    const bool sparse = free_far != far;
    const int fixed = cd.gen_index & far & ~touched;
    const int Gs = sparse ? (1 << __popc(free_far)) : G;
    if (sparse && gen) {
      float4* const st4 = reinterpret_cast<float4*>(st);
      const int NH = 1 << (nint - 1);
      for (int i = rank; i < NH; i += size) st4[TQS_IX(i, NH)] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (TEAM == TEAM_MULTI) grid_sync(*bar); else team_sync<TEAM>();
    }
    touched |= b0 | b1 | b2 | b3;
    for (int g = rank; g < Gs; g += size) {
      const int base = sparse ? (fixed | deposit_bits(g, free_far))
                              : ins0(ins0(ins0(ins0(g, l0), l1), l2), l3);
      const int sb = swz(base);
      float2 a[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (gen) {
          const int off = base | ((j & 1) ? b0 : 0) | ((j & 2) ? b1 : 0) | ((j & 4) ? b2 : 0) | ((j & 8) ? b3 : 0);
          a[j] = make_float2(off == cd.gen_index ? 1.f : 0.f, 0.f);
        } else {
          a[j] = ld_state<TEAM>(&st[TQS_IX(sb ^ ((j & 1) ? w0 : 0) ^ ((j & 2) ? w1 : 0) ^ ((j & 4) ? w2 : 0) ^ ((j & 8) ? w3 : 0), 1 << nint)]);
        }
      }
      // select-free dense butterflies where they pay: the CTA-sized teams,
      // whose random-circuit workloads are dense-gate heavy
      run_ops<TEAM != TEAM_WARP && TEAM != TEAM_PAIR>(a, ops, count, base, scale);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        st[TQS_IX(sb ^ ((j & 1) ? w0 : 0) ^ ((j & 2) ? w1 : 0) ^ ((j & 4) ? w2 : 0) ^ ((j & 8) ? w3 : 0), 1 << nint)] = a[j];
    }
    if (TEAM == TEAM_MULTI) grid_sync(*bar); else team_sync<TEAM>();
  }
  // TEAM_MULTI: the first CTA alone writes the outputs, as a TEAM_GLOBAL CTA would.
  if (TEAM == TEAM_MULTI) {
    if (!bar->leader) return;
    rank = threadIdx.x;
    size = blockDim.x;
  }
  // Warp and pair teams: the next job (its atomic was issued when this
  // circuit started) is shared with the team here and its circuit index is
  // loaded, so both latencies hide behind the output phase.
  if (TEAM == TEAM_WARP) {
    next_job = __shfl_sync(0xffffffffu, next_job, 0);
  } else if (TEAM == TEAM_PAIR) {
    if (rank == 0) *s_slot = next_job;
    team_sync<TEAM>();
    next_job = *s_slot;
  }
  if (TEAM == TEAM_WARP || TEAM == TEAM_PAIR)
    next_ci = next_job < L.n_jobs ? __ldg(L.order + next_job) : 0;
  // Output: logical index i holds the amplitude at physical index P(i) =
  // col_off ^ lin(i) (the output map), whose shared-memory slot is A(i) =
  // swz(P(i)).  lin and swz are linear over GF(2), so A(i) is swz(col_off)
  // XOR the columns swz(col[q]) over the set bits q of i.  A thread writes the pairs
  // i, i + 1 with i = 2 rank + 2 size g (one 16-byte store of the state, one
  // of the probabilities); g runs in blocks of 8 in Gray-code order, so each
  // step changes A by one XOR of a column held in a register.
  const int N = 1 << n;
  float2* const outc = L.out + cd.out_off;
  double* const probc = L.probs ? L.probs + cd.out_off : nullptr;
  double acc = 0.0;
  {
    const FusedCirc* cg = L.circs + ci;
    // log2 of the index stride between a thread's pairs (2 size): fixed for
    // the warp and pair teams, so the stores take immediate offsets
    constexpr int kSh = TEAM == TEAM_WARP ? 6 : TEAM == TEAM_PAIR ? 7 : 0;
    const int sh = kSh ? kSh : 31 - __clz(2 * size);
    const int i0 = 2 * rank;
    if (i0 < N) {
      const float oscale = cd.out_scale;
      const bool exact = L.exact_probs != 0;
      auto col = [&](int q) { return q < n ? swz(__ldg(&cg->col[q])) : 0; };
      const int a1 = col(0);
      const int c0 = col(sh), c1 = col(sh + 1), c2 = col(sh + 2);
      const int a_i0 = swz(cd.col_off ^ map_lin(cg, i0, n));
      const int iters = N > (1 << sh) ? (N >> sh) : 1;  // pairs per thread
      const int NI = 1 << nint;
#pragma unroll 1
      for (int blk = 0; blk < iters; blk += 8) {
        // A at the block's first pair: the block index's bits sh + 3 ...
        int ab = a_i0;
        for (int q = 3; (blk >> q) != 0; ++q)
          if ((blk >> q) & 1) ab ^= col(sh + q);
        const int ib = i0 + (blk << sh);  // the block's first pair
        float s[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          s[r] = 0.f;
          const int gr = r ^ (r >> 1);  // Gray code: consecutive r differ in one bit
          if (r < iters) {
            const int a = ab ^ ((gr & 1) ? c0 : 0) ^ ((gr & 2) ? c1 : 0) ^ ((gr & 4) ? c2 : 0);
            float2 v0 = ld_state<TEAM>(&st[TQS_IX(a, NI)]);
            float2 v1 = ld_state<TEAM>(&st[TQS_IX(a ^ a1, NI)]);
            if (oscale != 1.0f) {
              v0 = make_float2(v0.x * oscale, v0.y * oscale);
              v1 = make_float2(v1.x * oscale, v1.y * oscale);
            }
            const int i = ib + (gr << sh);
            *reinterpret_cast<float4*>(outc + TQS_IX(i, N - 1)) = make_float4(v0.x, v0.y, v1.x, v1.y);
            const float q0 = fmaf(v0.x, v0.x, v0.y * v0.y), q1 = fmaf(v1.x, v1.x, v1.y * v1.y);
            if (probc) {
              // |psi|^2 in FP32 arithmetic, stored as FP64; or (exact_probs) the
              // exact squares correctly rounded once in FP64
              *reinterpret_cast<double2*>(probc + TQS_IX(i, N - 1)) =
                  exact ? make_double2(prob_f64(v0), prob_f64(v1)) : make_double2(q0, q1);
            }
            s[r] = q0 + q1;
          }
        }
        // the block's 16 values summed as a tree in FP32, then added in FP64
        acc += static_cast<double>(((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])));
      }
    }
  }
  // Fixed-order reduction (deterministic): per-thread FP64 partials, warp
  // butterfly, then the warps of the team in order.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (TEAM == TEAM_WARP) {
    if (rank == 0 && L.norms) L.norms[ci] = acc;
  } else {
    const int warp = rank >> 5, lane = rank & 31;
    if (lane == 0) s_red[warp] = acc;
    team_sync<TEAM>();
    if (rank == 0) { double s = 0.0; for (int w = 0; w < (size >> 5); ++w) s += s_red[w]; if (L.norms) L.norms[ci] = s; }
  }
  if (TEAM == TEAM_MULTI && rank == 0 && *reinterpret_cast<volatile int*>(L.err) != 0) {
    // a grid barrier timed out: the outputs are not valid, make that visible
    const float nan = __int_as_float(0x7fffffff);
    if (L.norms) L.norms[ci] = static_cast<double>(nan);
    outc[0] = make_float2(nan, nan);
  }
  if ((TEAM == TEAM_WARP || TEAM == TEAM_PAIR) && rank == 0 && next_job < L.n_jobs)
    prefetch_l1_range(L.circs + next_ci, sizeof(FusedCirc), 0, 1);
  team_sync<TEAM>();
}

template <int TEAM>
__global__ void __launch_bounds__(TEAM == TEAM_CTA ? kCtaThreads : 512)
    fused_kernel(const __grid_constant__ FusedLaunch L) {
  extern __shared__ float4 smem_raw[];
  float2* smem = reinterpret_cast<float2*>(smem_raw);
  if (TEAM == TEAM_PAIR) {
    // two warps per circuit; pair p uses slice p and named barrier 1 + p
    __shared__ int s_job[8];
    __shared__ double s_red[8][4];
    const int pair = threadIdx.x >> 6, rank = threadIdx.x & 63;
    float2* st = smem + (static_cast<size_t>(pair) << L.slice_q);
    // Each circuit takes the team's next job from the counter when it starts
    // and hands it over before its output phase (run_circuit).
    if (rank == 0) s_job[pair] = atomicAdd(L.counter, 1);
    team_sync<TEAM_PAIR>();
    int job = s_job[pair];
    team_sync<TEAM_PAIR>();
    int ci = job < L.n_jobs ? __ldg(L.order + job) : 0;
    while (job < L.n_jobs) {
      int next_job = rank == 0 ? atomicAdd(L.counter, 1) : 0;
      int next_ci = 0;
      run_circuit<TEAM_PAIR>(L, ci, st, rank, 64, s_red[pair], next_job, next_ci, &s_job[pair]);
      job = next_job;
      ci = next_ci;
    }
  } else if (TEAM == TEAM_WARP) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* st = smem + (static_cast<size_t>(warp) << L.slice_q);
    int job = lane == 0 ? atomicAdd(L.counter, 1) : 0;
    job = __shfl_sync(0xffffffffu, job, 0);
    int ci = job < L.n_jobs ? __ldg(L.order + job) : 0;
    while (job < L.n_jobs) {
      int next_job = lane == 0 ? atomicAdd(L.counter, 1) : 0;
      int next_ci = 0;
      run_circuit<TEAM_WARP>(L, ci, st, lane, 32, nullptr, next_job, next_ci, nullptr);
      job = next_job;
      ci = next_ci;
    }
  } else if (TEAM == TEAM_MULTI) {
    __shared__ double s_red[32];
    const int K = L.ctas_per_job;
    const int job = blockIdx.x / K, local = blockIdx.x - job * K;
    GridBar bar{reinterpret_cast<unsigned int*>(L.counter) + job, L.err, 0u,
                static_cast<unsigned int>(K), local == 0};
    int unused_job = 0, unused_ci = 0;
    run_circuit<TEAM_MULTI>(L, L.order[job], L.gscratch + (static_cast<size_t>(job) << kGlobalSlotQ),
                            local * blockDim.x + threadIdx.x, K * blockDim.x, s_red, unused_job,
                            unused_ci, nullptr, &bar);
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
      int unused_job = 0, unused_ci = 0;
      run_circuit<TEAM>(L, L.order[job], st, threadIdx.x, blockDim.x, s_red, unused_job, unused_ci,
                        nullptr);
    }
  }
}

// ------------------------------------------------- full state vector tiles
// One pass of the full-state-vector backend (Appendix A, eq. 12, on states in
// HBM): the CTA streams the state through shared memory one tile at a time
// (the 2^T amplitudes that agree outside the tile bits; the lowest bits are
// tile bits, so loads and stores move 256-byte runs), runs the pass's tile
// program on it exactly like a fused program on a CTA team (4-bit register
// passes, wide passes for custom unitaries), and writes it back through the
// program's final qubit map.  Far controls and far diagonal bits of the
// program are virtual qubits T, T+1, ... whose values, fixed per tile, are
// or-ed into each group's index.

// The bits of v deposited, lowest first, at the set bits of mask.
__device__ __forceinline__ uint64_t deposit64(uint64_t v, uint64_t mask) {
  uint64_t r = 0;
  for (; mask != 0; mask &= mask - 1, v >>= 1)
    if (v & 1) r |= mask & (~mask + 1);
  return r;
}

constexpr int kFsvHighQ = kFsvTileQ - kFsvLowQ;

__global__ void __launch_bounds__(kFsvThreads)
    fsv_tile_kernel(const __grid_constant__ FusedLaunch L, const __grid_constant__ FsvTile F) {
  extern __shared__ float4 smem_raw[];
  float2* st = reinterpret_cast<float2*>(smem_raw);
  __shared__ uint64_t hoff[1 << kFsvHighQ];
  const int tid = threadIdx.x;
  const FusedCirc cd = L.circs[0];
  const int T = F.T, NT = 1 << T, G = NT >> 4;
  const int nlow = T < kFsvLowQ ? T : kFsvLowQ;
  const int lowm = (1 << nlow) - 1;
  const uint64_t high = F.mask & ~static_cast<uint64_t>(lowm);
  for (int h = tid; h < (NT >> nlow); h += kFsvThreads) hoff[h] = deposit64(h, high);
  const uint64_t all = (F.n >= 64) ? ~0ull : ((1ull << F.n) - 1);
  const uint64_t comp = all & ~F.mask;
  const uint64_t ntiles = 1ull << (F.n - T);
  // write-back map of tile element e = tid + kFsvThreads k: P(tid) ^ lin(kFsvThreads k),
  // the second part from the columns of the bits above the thread index
  // (T <= kFsvTileQ = kThrQ + 5)
  constexpr int kThrQ = 8;  // log2 kFsvThreads
  static_assert((1 << kThrQ) == kFsvThreads && kFsvTileQ <= kThrQ + 5, "tile threads");
  const int p_tid = cd.col_off ^ map_lin(L.circs, tid, T);
  int hcol[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) hcol[j] = kThrQ + j < T ? __ldg(&L.circs->col[kThrQ + j]) : 0;
  float2* g = F.state;
  __syncthreads();
  for (uint64_t j = blockIdx.x; j < ntiles; j += gridDim.x) {
    const uint64_t gbase = deposit64(j, comp);
    int ext = 0;
    for (int v = 0; v < F.nfar; ++v) ext |= static_cast<int>((gbase >> F.far[v]) & 1) << (T + v);
    for (int e = tid; e < NT; e += kFsvThreads)
      st[TQS_IX(swz(e), NT)] = g[TQS_IX(gbase + hoff[e >> nlow] + (e & lowm), 1ull << F.n)];
    __syncthreads();
    for (int p = 0; p < cd.pass_count; ++p) {
      const uint4 pr = __ldg(reinterpret_cast<const uint4*>(L.passes + cd.pass_begin + p));
      const int l0 = pr.x & 0xff, l1 = (pr.x >> 8) & 0xff, l2 = (pr.x >> 16) & 0xff, l3 = pr.x >> 24;
      if (l0 == kWidePass) {
        wide_pass<TEAM_CTA>(L, T, l1, pr.y, pr.z, pr.w, st, tid, kFsvThreads);
        continue;
      }
      const FusedOp* ops = L.ops + pr.y;
      const uint32_t count = pr.z;
      const float scale = __uint_as_float(pr.w);
      const int w0 = swz(1 << l0), w1 = swz(1 << l1), w2 = swz(1 << l2), w3 = swz(1 << l3);
      for (int gi = tid; gi < G; gi += kFsvThreads) {
        const int base = ins0(ins0(ins0(ins0(gi, l0), l1), l2), l3);
        const int sb = swz(base);
        float2 a[16];
#pragma unroll
        for (int q = 0; q < 16; ++q)
          a[q] = st[TQS_IX(sb ^ ((q & 1) ? w0 : 0) ^ ((q & 2) ? w1 : 0) ^ ((q & 4) ? w2 : 0) ^ ((q & 8) ? w3 : 0), NT)];
        run_ops<true>(a, ops, count, base | ext, scale);
#pragma unroll
        for (int q = 0; q < 16; ++q)
          st[TQS_IX(sb ^ ((q & 1) ? w0 : 0) ^ ((q & 2) ? w1 : 0) ^ ((q & 4) ? w2 : 0) ^ ((q & 8) ? w3 : 0), NT)] = a[q];
      }
      __syncthreads();
    }
    // tile qubit i of the result sits at physical tile bit pos[i]
    const float osc = cd.out_scale;
    for (int e = tid; e < NT; e += kFsvThreads) {
      const int k = e >> kThrQ;
      const int pk = ((k & 1) ? hcol[0] : 0) ^ ((k & 2) ? hcol[1] : 0) ^ ((k & 4) ? hcol[2] : 0) ^
                     ((k & 8) ? hcol[3] : 0) ^ ((k & 16) ? hcol[4] : 0);
      float2 v = st[TQS_IX(swz(p_tid ^ pk), NT)];
      if (osc != 1.0f) v = make_float2(v.x * osc, v.y * osc);
      g[TQS_IX(gbase + hoff[e >> nlow] + (e & lowm), 1ull << F.n)] = v;
    }
    __syncthreads();
  }
}

size_t fused_smem_bytes(int team, int warps_per_cta, int slice_q) {
  if (team == TEAM_WARP) return (static_cast<size_t>(warps_per_cta) << slice_q) * sizeof(float2);
  if (team == TEAM_PAIR) return (static_cast<size_t>(warps_per_cta / 2) << slice_q) * sizeof(float2);
  if (team == TEAM_CTA) return (static_cast<size_t>(1) << slice_q) * sizeof(float2);
  return 0;
}

int fused_threads(int team, int warps_per_cta) {
  if (team == TEAM_WARP || team == TEAM_PAIR) return 32 * warps_per_cta;
  if (team == TEAM_CTA) return warps_per_cta > 0 ? 32 * warps_per_cta : kCtaThreads;
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
  } else if (team == TEAM_PAIR) {
    cudaFuncSetAttribute(fused_kernel<TEAM_PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fused_kernel<TEAM_PAIR>, threads,
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

cudaError_t launch_fsv_tile(const FusedLaunch& L, const FsvTile& F, cudaStream_t s) {
  static int per_sm = 0, sms = 0;
  const int smem_max = static_cast<int>((size_t(1) << kFsvTileQ) * sizeof(float2));
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(fsv_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_max);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fsv_tile_kernel, kFsvThreads, smem_max);
    if (per_sm < 1) per_sm = 1;
  }
  const uint64_t ntiles = 1ull << (F.n - F.T);
  const uint64_t cap = static_cast<uint64_t>(per_sm) * static_cast<uint64_t>(sms > 0 ? sms : 152);
  const int grid = static_cast<int>(ntiles < cap ? ntiles : cap);
  const size_t smem = (size_t(1) << F.T) * sizeof(float2);
  fsv_tile_kernel<<<grid, kFsvThreads, smem, s>>>(L, F);
  count_launches(1);
  return cudaGetLastError();
}

TQS_DEFINE_VIOLATIONS(violations_fused)

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
  } else if (L.team == TEAM_PAIR) {
    e = cudaFuncSetAttribute(fused_kernel<TEAM_PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    fused_kernel<TEAM_PAIR><<<L.grid, threads, smem, s>>>(L);
  } else if (L.team == TEAM_CTA) {
    e = cudaFuncSetAttribute(fused_kernel<TEAM_CTA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    fused_kernel<TEAM_CTA><<<L.grid, threads, smem, s>>>(L);
  } else if (L.team == TEAM_MULTI) {
    // cooperative: the CTAs wait on one another at the grid barriers
    FusedLaunch arg = L;
    void* args[] = {&arg};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(fused_kernel<TEAM_MULTI>),
                                    dim3(L.grid), dim3(threads), args, 0, s);
    if (e != cudaSuccess) return e;
  } else {
    fused_kernel<TEAM_GLOBAL><<<L.grid, threads, 0, s>>>(L);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tqs
