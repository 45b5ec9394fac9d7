// Device side of the synthetic block model shared by the kernels: pair
// vectors under the current lattice and the radial functions of the C and V
// blocks (V_AB = M h(r), grad_d V_AB = M h'(r) d / r, on-site V = M).
#pragma once

#include <cuda_runtime.h>

#include "hfx_internal.h"

namespace hfx {
namespace model {

// d = tau_j + R.L - tau_i under the plan's current positions and lattice.
__device__ __forceinline__ void pair_vector(const DevPlan& P, int i, int j, const int* R, double d[3]) {
  const double r0 = (double)R[0], r1 = (double)R[1], r2 = (double)R[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double RL = r0 * P.L[k] + r1 * P.L[3 + k] + r2 * P.L[6 + k];
    d[k] = (P.pos[3 * j + k] + RL) - P.pos[3 * i + k];
  }
}

// Block model radial functions: f(r) = (1-(r/R_C)^2)^3 exp(-r^2/2) for r < R_C,
// h(r) = erfc(omega r)/(r+1), and their first derivatives.
__device__ __forceinline__ void radial_f(double r, double RC, double& f, double& fp) {
  if (r >= RC) {
    f = 0.0;
    fp = 0.0;
    return;
  }
  const double q = r / RC;
  const double x = 1.0 - q * q;
  const double e = exp(-0.5 * r * r);
  f = x * x * x * e;
  fp = 3.0 * x * x * (-2.0 * r / (RC * RC)) * e - r * (x * x * x) * e;
}

__device__ __forceinline__ void radial_h(double r, double om, double& h, double& hp) {
  const double ec = erfc(om * r);
  const double r1 = r + 1.0;
  h = ec / r1;
  const double two_over_sqrt_pi = 1.1283791670955126;
  hp = (-2.0 * om * 0.5 * two_over_sqrt_pi) * exp(-(om * r) * (om * r)) / r1 - ec / (r1 * r1);
}

// V pair p: h(r) and g = h'(r) d / r (h = 1, g = 0 on site), as stored for
// every V pair candidate by the V norm kernel of this evaluation (one FP64
// erfc/exp evaluation per pair).
__device__ __forceinline__ void v_pair(const DevPlan& P, int p, double& h, double g[3]) {
  const double* s = P.v_hg + 4 * (long long)p;
  h = s[0];
  g[0] = s[1];
  g[1] = s[2];
  g[2] = s[3];
}

// C pair p of the block model: C = G f + G' fa and grad_c C = G g_c + G' ga_c
// (G' the anisotropic template, fa = f (d.e)/R_C; on site C = G, grad C = 0).
// s = {f, fa, g0, g1, g2, ga0, ga1, ga2}.
__device__ __forceinline__ void c_pair_eval(const DevPlan& P, int p, double s[8]) {
  const int A = P.c_home[p], j = P.c_j[p];
  const int* R = P.c_R + 3 * p;
#pragma unroll
  for (int k = 0; k < 8; ++k) s[k] = 0.0;
  s[0] = 1.0;
  if (A == j && R[0] == 0 && R[1] == 0 && R[2] == 0) return;
  double d[3];
  pair_vector(P, A, j, R, d);
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double f, fp;
  radial_f(r, P.RC, f, fp);
  s[0] = f;
#pragma unroll
  for (int c = 0; c < 3; ++c) s[2 + c] = fp * d[c] / r;
  if (P.Gp) {
    const double de = d[0] * P.e[0] + d[1] * P.e[1] + d[2] * P.e[2];
    s[1] = f * de / P.RC;
#pragma unroll
    for (int c = 0; c < 3; ++c) s[5 + c] = (fp * (d[c] / r) * de + f * P.e[c]) / P.RC;
  }
}

// Element t of component c (0: C, 1..3: grad C) of C pair p from its stored
// scalars cs (c_pair_eval) rounded to FP32 (csf = (float)cs) and the FP32
// templates at offset go: within a few FP32 ulps of the FP64 value, the
// precision the split path's stores keep.
__device__ __forceinline__ float c_value_f(const DevPlan& P, const float* csf, long long go, int t, int c) {
  float v = P.Gf[go + t] * (c == 0 ? csf[0] : csf[1 + c]);
  if (P.Gpf) v = fmaf(P.Gpf[go + t], c == 0 ? csf[1] : csf[4 + c], v);
  return v;
}

}  // namespace model
}  // namespace hfx
