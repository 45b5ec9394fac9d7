// The plan's cross-CTA sums (E, the virial, the pair gradients g^C and g^V
// of Eq. Fexx1, and the forces) and the exact fixed-point accumulator behind
// hfx_options.deterministic.
//
// A fixed-point cell is a two's-complement 128-bit integer in units of 2^-64,
// stored as two 64-bit words (low word first).  A double v is added as the
// integer trunc(v * 2^64) (exact for |v| >= 2^-11; bits below 2^-64 are
// dropped), with one atomic add on the low word and one on the high word
// carrying the low word's overflow, which the old value returned by the
// first add reveals.  Integer addition modulo 2^128 does not depend on the
// order of the adds, so a cell holds the same bits whatever order the CTAs
// reach it in; every contribution is itself computed in a fixed order inside
// its CTA, so deterministic plans give bit-identical E, F and sigma from run
// to run and for any launch shape.  Magnitudes must stay below 2^62 (E,
// forces and pair gradients are many orders of magnitude smaller).
#pragma once

#include <cstdint>

#include "hfx_internal.h"

namespace hfx {
namespace dev {

// trunc(v * 2^64) as (lo, hi); zero for zero, subnormals and |v| < 2^-64.
__device__ __forceinline__ void fx_split(double v, unsigned long long& lo, unsigned long long& hi) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7ff);
  lo = 0ull;
  hi = 0ull;
  if (ex == 0) return;
  const unsigned long long m = (bits & 0x000fffffffffffffull) | 0x0010000000000000ull;   // |v| = m 2^(ex - 1075)
  const int sh = ex - 1075 + 64;                                                          // |v| 2^64 = m 2^sh
  if (sh >= 64) {
    hi = m << (sh - 64);
  } else if (sh > 0) {
    lo = m << sh;
    hi = m >> (64 - sh);
  } else if (sh > -64) {
    lo = m >> (-sh);
  }
  if (bits >> 63) {   // negate the 128-bit magnitude
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
}

__device__ __forceinline__ void fx_add(unsigned long long* cell, double v) {
  unsigned long long lo, hi;
  fx_split(v, lo, hi);
  if (lo == 0ull && hi == 0ull) return;
  unsigned long long carry = 0ull;
  if (lo != 0ull) {
    const unsigned long long old = atomicAdd(cell, lo);
    carry = (old + lo < old) ? 1ull : 0ull;
  }
  if (hi + carry != 0ull) atomicAdd(cell + 1, hi + carry);
}

// The cell's value, rounded to a double.
__device__ __forceinline__ double fx_get(const unsigned long long* cell) {
  unsigned long long lo = cell[0], hi = cell[1];
  const bool neg = (hi >> 63) != 0ull;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  const double r = (double)hi + (double)lo * 0x1p-64;
  return neg ? -r : r;
}

// ------------------------------------------------------ the plan's sums
// FP64 atomic adds, or the fixed-point cells of a deterministic plan
// (P.fxC != nullptr).  Indices are those of the FP64 arrays.
__device__ __forceinline__ void add_gC(const DevPlan& P, long long i, double v) {
  if (P.fxC) fx_add(P.fxC + 2 * i, v);
  else atomicAdd(P.gC + i, v);
}
__device__ __forceinline__ void add_gV(const DevPlan& P, long long i, double v) {
  if (P.fxC) fx_add(P.fxV + 2 * i, v);
  else atomicAdd(P.gV + i, v);
}
__device__ __forceinline__ void add_E(const DevPlan& P, double v) {
  if (P.fxC) fx_add(P.fxA, v);
  else atomicAdd(P.acc + ACC_E, v);
}
__device__ __forceinline__ void add_W(const DevPlan& P, int c, double v) {   // virial component c
  if (P.fxC) fx_add(P.fxA + 2 * (1 + c), v);
  else atomicAdd(P.acc + ACC_W + c, v);
}
__device__ __forceinline__ double get_gC(const DevPlan& P, long long i) { return P.fxC ? fx_get(P.fxC + 2 * i) : P.gC[i]; }
__device__ __forceinline__ double get_gV(const DevPlan& P, long long i) { return P.fxC ? fx_get(P.fxV + 2 * i) : P.gV[i]; }
__device__ __forceinline__ double get_E(const DevPlan& P) { return P.fxC ? fx_get(P.fxA) : P.acc[ACC_E]; }
__device__ __forceinline__ double get_W(const DevPlan& P, int c) {
  return P.fxC ? fx_get(P.fxA + 2 * (1 + c)) : P.acc[ACC_W + c];
}

}  // namespace dev
}  // namespace hfx
