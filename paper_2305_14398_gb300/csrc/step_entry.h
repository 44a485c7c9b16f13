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

__device__ __forceinline__ float2 step_entry(const StepFactor* fs, int nf, uint32_t idle,
                                             uint32_t r, uint32_t c) {
  if ((r ^ c) & idle) return make_float2(0.f, 0.f);
  float2 v = make_float2(1.f, 0.f);
  for (int k = 0; k < nf; ++k) {
    const StepFactor& f = fs[k];
    int idx;
    if (f.custom) {
      int rr = 0, cc = 0;
      for (int t = 0; t < f.nq; ++t) {
        rr |= ((r >> f.qc[t]) & 1) << t;
        cc |= ((c >> f.qc[t]) & 1) << t;
      }
      v = step_cmul(v, f.coef[(rr << f.nq) + cc]);
      continue;
    }
    if (f.nq == 1) {
      idx = ((r >> f.q0) & 1) * 2 + ((c >> f.q0) & 1);
    } else {
      const int rr = (((r >> f.q0) & 1) << 1) | ((r >> f.q1) & 1);
      const int cc = (((c >> f.q0) & 1) << 1) | ((c >> f.q1) & 1);
      idx = rr * 4 + cc;
    }
    v = step_cmul(v, f.m[idx]);
  }
  return v;
}

}  // namespace tqs
