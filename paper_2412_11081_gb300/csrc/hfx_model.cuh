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

}  // namespace model
}  // namespace hfx
