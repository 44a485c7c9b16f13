// Entry <r|S|c> of a step unitary from its Kronecker factors (Algorithm 2):
// the product over the step's factors of the factor's entry at the bits it
// acts on, times the identity (a Kronecker delta) on idle qubits.  A
// two-qubit factor's 4x4 matrix is indexed by (bit q0 << 1) | bit q1 (eq. 7
// with the control first); a custom k-qubit factor's matrix by the local
// index whose bit t is the bit of qubit qc[t].  Shared by the plain
// materialiser and the chain's operand generator.
#pragma once

#include "tqs_internal.h"

namespace tqs {

__device__ __forceinline__ float2 step_cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Entry <r|F|c> of one factor F (its rows and columns indexed by the bits of
// r and c at the factor's qubits).
__device__ __forceinline__ float2 factor_entry(const StepFactor& f, uint32_t r, uint32_t c) {
  if (f.custom) {
    int rr = 0, cc = 0;
    for (int t = 0; t < f.nq; ++t) {
      rr |= ((r >> f.qc[t]) & 1) << t;
      cc |= ((c >> f.qc[t]) & 1) << t;
    }
    return f.coef[(rr << f.nq) + cc];
  }
  int idx;
  if (f.nq == 1) {
    idx = ((r >> f.q0) & 1) * 2 + ((c >> f.q0) & 1);
  } else {
    const int rr = (((r >> f.q0) & 1) << 1) | ((r >> f.q1) & 1);
    const int cc = (((c >> f.q0) & 1) << 1) | ((c >> f.q1) & 1);
    idx = rr * 4 + cc;
  }
  return f.m[idx];
}

// The qubits a factor acts on, as a bit mask.
__device__ __forceinline__ uint32_t factor_qubits(const StepFactor& f) {
  if (f.custom) {
    uint32_t m = 0;
    for (int t = 0; t < f.nq; ++t) m |= 1u << f.qc[t];
    return m;
  }
  return (1u << f.q0) | (f.nq == 2 ? 1u << f.q1 : 0u);
}

__device__ __forceinline__ float2 step_entry(const StepFactor* fs, int nf, uint32_t idle,
                                             uint32_t r, uint32_t c) {
  if ((r ^ c) & idle) return make_float2(0.f, 0.f);
  float2 v = make_float2(1.f, 0.f);
  for (int k = 0; k < nf; ++k) v = step_cmul(v, factor_entry(fs[k], r, c));
  return v;
}

}  // namespace tqs
