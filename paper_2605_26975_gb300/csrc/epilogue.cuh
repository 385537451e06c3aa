// The elementwise part of the Hessian-vector product of the fast path, shared
// by the stand-alone epilogue and the solver's epilogue fused with the Gram
// product, so that both produce the same bits.
//
// For the entry (i, l) of column l, with S the sparse part from the edge
// kernel, Delta = (Delta_p u)_i, v = V_il and u = U_il:
//   HV = A_l (S - L_l |u|^(p-2) v) - B_l (Delta SD_l + phi_p(u) E_l)
// where the column coefficients A, L, B, SD, E come from the edge kernel's
// reductions (the exact quotient Hessian of F_p, Section 2; B = 0 in
// Algorithm 1's form).
#pragma once

#include "common.cuh"

namespace pspec {

struct HvpCoef {
  float A, L, B, SD, E;
};

__device__ __forceinline__ float hvp_entry(float s, float u, float v, float dl, const HvpCoef& c,
                                           float pm2, bool zero_rule) {
  float su = abs_pow_pm2_clamped(u, pm2);
  const float phu = su * u;
  if (zero_rule && u == 0.0f) su = 0.0f;
  return c.A * (s - c.L * su * v) - c.B * (dl * c.SD + phu * c.E);
}

}  // namespace pspec
