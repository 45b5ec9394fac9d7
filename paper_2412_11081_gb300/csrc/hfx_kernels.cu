// FP64 CUDA kernels of the HFX force/stress hot path (sm_103a).
//
// Stages of one evaluation (paper Sec. 2 and 3; the factorisation is the
// distributive law applied to Eq. exx_expand):
//   K1  block generation   C, grad C (C pairs); norms of V, grad V (V pairs);
//                          V, grad V blocks for the V pairs the items need
//   K2  screening           step 1 per-tensor norms, step 2 Cauchy-Schwarz
//                          bounds per item (Sec. 3.2, Algorithm 1)
//   K3  Y^{XZ} = sum_W C_XW D_WZ for every key an item needs
//   K4  first exchange product, per (A,B) pair over its kept F:
//          U = D_AB . Y^{BF};  R_AB += <C_AF, U>;  g^C_AF += -2 <grad C_AF, V_AB . U>
//   K5  second exchange product, per (A,B) pair:
//          R2_AB = <Y^{AB}, Y^{BA}>;  Z = V_AB . Y^{BA};  g^C_AF += -2 <grad C_AF, Z . D_FB^T>
//   K7  E = -sum <V, R>, g^V = -<grad V, R>, forces F_I += g, F_J -= g and the
//       virial sum g (x) d that gives sigma = -(1/Omega) sum g (x) d (Eq. stress)
//
// All arithmetic is FP64.  Per-pair gradient contributions from different
// CTAs meet in FP64 atomics (order-dependent only at the last bits).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>

#include "hfx_accum.cuh"
#include "hfx_internal.h"
#include "hfx_model.cuh"

namespace hfx {
namespace {

using namespace model;

constexpr int kThreads = 256;
std::atomic<long long> g_launches{0};   // host-side count of kernel launches (all threads)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block; every thread gets the result.  `red` needs
// kThreads/32 doubles of shared memory and is reused across calls.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

__device__ __forceinline__ int dlut_get(const DevPlan& P, int i, int j, int r0, int r1, int r2) {
  if (r0 < -P.HD0 || r0 > P.HD0 || r1 < -P.HD1 || r1 > P.HD1 || r2 < -P.HD2 || r2 > P.HD2) return -1;
  const long long n0 = 2 * P.HD0 + 1, n1 = 2 * P.HD1 + 1, n2 = 2 * P.HD2 + 1;
  const long long idx = (((((long long)i * P.N + j) * n0 + (r0 + P.HD0)) * n1 + (r1 + P.HD1)) * n2) + (r2 + P.HD2);
  return P.dlut[idx];
}

__device__ __forceinline__ int ylut_get(const DevPlan& P, int i, int j, int r0, int r1, int r2) {
  if (r0 < -P.HY0 || r0 > P.HY0 || r1 < -P.HY1 || r1 > P.HY1 || r2 < -P.HY2 || r2 > P.HY2) return -1;
  const long long n0 = 2 * P.HY0 + 1, n1 = 2 * P.HY1 + 1, n2 = 2 * P.HY2 + 1;
  const long long idx = (((((long long)i * P.N + j) * n0 + (r0 + P.HY0)) * n1 + (r1 + P.HY1)) * n2) + (r2 + P.HY2);
  return P.ylut[idx];
}

// ---------------------------------------------------------------- K2: D norms
__global__ void k_dnorm(DevPlan P) {
  __shared__ double red[kThreads / 32];
  unsigned long long kept = 0;
  for (long long k = blockIdx.x; k < P.n_d; k += gridDim.x) {
    const long long b = P.Doff[k], e = P.Doff[k + 1];
    double s = 0.0;
    for (long long t = b + threadIdx.x; t < e; t += blockDim.x) s += P.Dval[t] * P.Dval[t];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
      const double n = sqrt(s);
      const bool keep = n > P.thD;
      P.Dkept[k] = keep ? n : 0.0;
      kept += keep;
    }
  }
  if (threadIdx.x == 0 && kept) atomicAdd(&P.cnt[CNT_D], kept);
}

// ---------------------------------------------------------------- K1: C blocks
// One CTA per C pair: C = G f(r) [+ G' f(r) (d.e)/R_C], grad_d C, and the
// step-1 decision ||C|| > theta_C or ||grad C|| > theta_dC.
__global__ void k_cblocks(DevPlan P, int frozen) {
  __shared__ double red[kThreads / 32];
  for (int p = blockIdx.x; p < P.nC; p += gridDim.x) {
    const int A = P.c_home[p], j = P.c_j[p];
    const int* R = P.c_R + 3 * p;
    double d[3];
    pair_vector(P, A, j, R, d);
    const bool onsite = (A == j) && R[0] == 0 && R[1] == 0 && R[2] == 0;
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double f = 1.0, fp = 0.0;
    if (!onsite) radial_f(r, P.RC, f, fp);
    double g[3] = {0.0, 0.0, 0.0};
    double ga[3] = {0.0, 0.0, 0.0};
    double fa = 0.0;
    if (!onsite) {
#pragma unroll
      for (int c = 0; c < 3; ++c) g[c] = fp * d[c] / r;
      if (P.Gp) {
        const double de = d[0] * P.e[0] + d[1] * P.e[1] + d[2] * P.e[2];
        fa = f * de / P.RC;
#pragma unroll
        for (int c = 0; c < 3; ++c) ga[c] = (fp * (d[c] / r) * de + f * P.e[c]) / P.RC;
      }
    }
    const int sA = P.species[A], sj = P.species[j];
    const long long go = P.G_off[sA * P.S + sj];
    const int n = P.n_abf[sA] * P.n_ao[sA] * P.n_ao[sj];
    double* C = P.Cst + P.c_off[p];
    double* dC = P.dCst + 3 * P.c_off[p];
    double sc = 0.0, sg = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double Gv = P.G[go + t];
      double c = Gv * f;
      double g0 = Gv * g[0], g1 = Gv * g[1], g2 = Gv * g[2];
      if (P.Gp && !onsite) {
        const double Gq = P.Gp[go + t];
        c = c + Gq * fa;
        g0 = g0 + Gq * ga[0];
        g1 = g1 + Gq * ga[1];
        g2 = g2 + Gq * ga[2];
      }
      C[t] = c;
      dC[t] = g0;
      dC[n + t] = g1;
      dC[2 * n + t] = g2;
      sc += c * c;
      sg += g0 * g0 + g1 * g1 + g2 * g2;
    }
    sc = block_sum(sc, red);
    sg = block_sum(sg, red);
    if (threadIdx.x == 0) {
      const double nc = sqrt(sc), ng = sqrt(sg);
      bool keep;
      if (frozen) {
        keep = P.c_keep[p] != 0;
      } else {
        keep = (nc > P.thC) || (ng > P.thdC);
        P.c_keep[p] = keep;
      }
      P.c_norm[p] = keep ? fmax(nc, ng) : 0.0;
      if (keep) atomicAdd(&P.cnt[CNT_C], 1ull);
    }
  }
}

// Split path: one thread per C pair.  The scalars of C = G f + G' fa and
// grad_c C = G g_c + G' ga_c are stored for the kernels that write the
// operand stores, and the norms come from the template moments:
// ||C||^2 = f^2 S_GG + 2 f fa S_GG' + fa^2 S_G'G', and the same with
// (g_c, ga_c) summed over c for ||grad C||^2.
__global__ void k_cnorm(DevPlan P, int frozen) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.nC; p += gridDim.x * blockDim.x) {
    double sc[8];
    c_pair_eval(P, p, sc);
    double* o = P.c_sc + 8 * (long long)p;
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = sc[k];
    const double* mo = P.Gmom + 3 * (P.species[P.c_home[p]] * P.S + P.species[P.c_j[p]]);
    const double nc2 = sc[0] * sc[0] * mo[0] + 2.0 * sc[0] * sc[1] * mo[1] + sc[1] * sc[1] * mo[2];
    double ng2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      ng2 += sc[2 + c] * sc[2 + c] * mo[0] + 2.0 * sc[2 + c] * sc[5 + c] * mo[1] + sc[5 + c] * sc[5 + c] * mo[2];
    const double nc = sqrt(fmax(nc2, 0.0)), ng = sqrt(fmax(ng2, 0.0));
    bool keep;
    if (frozen) {
      keep = P.c_keep[p] != 0;
    } else {
      keep = (nc > P.thC) || (ng > P.thdC);
      P.c_keep[p] = keep;
    }
    P.c_norm[p] = keep ? fmax(nc, ng) : 0.0;
    if (keep) atomicAdd(&P.cnt[CNT_C], 1ull);
  }
}

// ---------------------------------------------------------------- K1: V norms
// One thread per V pair.  V = M h(r) and grad_d V = M h'(r) d/r (on-site:
// V = M, grad V = 0), so ||V|| = |h| ||M|| and ||grad V|| = |h'| ||M|| (the
// three components of d/r have unit length): the template norm ||M_st||_F is
// taken once per species pair when the plan is made.
__global__ void k_vnorm(DevPlan P, int frozen) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.nV; p += gridDim.x * blockDim.x) {
    const int A = P.v_home[p], j = P.v_j[p];
    const int* R = P.v_R + 3 * p;
    const bool onsite = (A == j) && R[0] == 0 && R[1] == 0 && R[2] == 0;
    double h = 1.0, hp = 0.0, g[3] = {0.0, 0.0, 0.0};
    if (!onsite) {
      double d[3];
      pair_vector(P, A, j, R, d);
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      radial_h(r, P.omega, h, hp);
#pragma unroll
      for (int c = 0; c < 3; ++c) g[c] = hp * d[c] / r;
    }
    double* hg = P.v_hg + 4 * (long long)p;   // for the kernels that evaluate V = M h, grad V = M g
    hg[0] = h;
    hg[1] = g[0];
    hg[2] = g[1];
    hg[3] = g[2];
    const double mn = P.Mnorm[P.species[A] * P.S + P.species[j]];
    const double nv = fabs(h) * mn, ng = fabs(hp) * mn;
    bool keep;
    if (frozen) {
      keep = P.v_keep[p] != 0;
    } else {
      keep = (nv > P.thV) || (ng > P.thdV);
      P.v_keep[p] = keep;
    }
    P.v_norm[p] = keep ? fmax(nv, ng) : 0.0;
    if (keep) atomicAdd(&P.cnt[CNT_V], 1ull);
  }
}

// ---------------------------------------------------------------- K2: yhat
// yhat_{XZ} = sum_{W in C(X), kept} c_XW d_WZ: the factor of the
// Cauchy-Schwarz bounds that sums over the inner atom (Sec. 3.2).
__global__ void k_yhat(DevPlan P) {
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < P.nY; y += gridDim.x * blockDim.x) {
    const int X = P.y_home[y], z = P.y_j[y];
    const int* Rz = P.y_R + 3 * y;
    double acc = 0.0;
    for (int q = P.c_ptr[X]; q < P.c_ptr[X + 1]; ++q) {
      const double c = P.c_norm[q];
      if (c == 0.0) continue;
      const int* Rw = P.c_R + 3 * q;
      const int di = dlut_get(P, P.c_j[q], z, Rz[0] - Rw[0], Rz[1] - Rw[1], Rz[2] - Rw[2]);
      if (di < 0) continue;
      acc += c * P.Dkept[di];
    }
    P.yhat[y] = acc;
  }
}

// ---------------------------------------------------------------- K2: items
// One thread per V pair (A,B).  First product: F in C(A) is kept iff
// c_AF v_AB d_AB yhat_BF > theta_CS.  Second product: (A,B) is kept iff
// v_AB yhat_AB yhat_BA > theta_CS.  Marks the Y keys the kept items read.
// Only home atoms A in [h0, h1) have items (the plan's share of the sum over
// A of Eq. exx_expand).
__global__ void k_screen(DevPlan P) {
  unsigned long long trip = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.nV; p += gridDim.x * blockDim.x) {
    unsigned int mask[kMaskWords];
#pragma unroll
    for (int w = 0; w < kMaskWords; ++w) mask[w] = 0u;
    int t2 = 0;
    const int A = P.v_home[p];
    const double v = (A >= P.h0 && A < P.h1) ? P.v_norm[p] : 0.0;
    if (v > 0.0) {
      const int b = P.v_j[p];
      const int* Rb = P.v_R + 3 * p;
      if (P.terms & 1) {
        const int di = P.v_didx[p];
        const double dab = di >= 0 ? P.Dkept[di] : 0.0;
        if (dab > 0.0) {
          const int q0 = P.c_ptr[A], q1 = P.c_ptr[A + 1];
          for (int q = q0; q < q1; ++q) {
            const double c = P.c_norm[q];
            if (c == 0.0) continue;
            const int* Rf = P.c_R + 3 * q;
            const int yc = ylut_get(P, b, P.c_j[q], Rf[0] - Rb[0], Rf[1] - Rb[1], Rf[2] - Rb[2]);
            if (yc < 0) continue;
            if (c * v * dab * P.yhat[yc] > P.thCS) {
              const int s = q - q0;
              mask[s >> 5] |= 1u << (s & 31);
              P.y_flag[yc] = 1;
              ++trip;
            }
          }
        }
      }
      if (P.terms & 2) {
        const int y1 = ylut_get(P, A, b, Rb[0], Rb[1], Rb[2]);
        const int y2 = ylut_get(P, b, A, -Rb[0], -Rb[1], -Rb[2]);
        if (y1 >= 0 && y2 >= 0 && v * P.yhat[y1] * P.yhat[y2] > P.thCS) {
          t2 = 1;
          P.y_flag[y1] = 1;
          P.y_flag[y2] = 1;
        }
      }
    }
    bool any = t2 != 0;
#pragma unroll
    for (int w = 0; w < kMaskWords; ++w) {
      P.v_mask[(size_t)p * kMaskWords + w] = mask[w];
      any = any || mask[w] != 0u;
    }
    P.v_t2[p] = (unsigned char)t2;
    P.v_flag[p] = any ? 1 : 0;
  }
  if (trip) atomicAdd(&P.cnt[CNT_TRIP], trip);
}

// ---------------------------------------------------------------- K1: V blocks
__global__ void k_vblocks(DevPlan P, const int* list, int n_list) {
  for (int k = blockIdx.x; k < n_list; k += gridDim.x) {
    const int p = list[k];
    const int A = P.v_home[p], j = P.v_j[p];
    double h, g[3];
    v_pair(P, p, h, g);
    const int sA = P.species[A], sj = P.species[j];
    const double* M = P.M + P.M_off[sA * P.S + sj];
    const int n = P.n_abf[sA] * P.n_abf[sj];
    double* V = P.Vst + P.v_off[p];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double m = M[t];
      V[t] = m * h;
      V[n + t] = m * g[0];
      V[2 * n + t] = m * g[1];
      V[3 * n + t] = m * g[2];
    }
  }
}

// ---------------------------------------------------------------- K3: Y
// One CTA per needed key (X; Z): Y[alpha,x,z] = sum_{W kept} sum_w
// C_XW[alpha,x,w] D_WZ[w,z], D_WZ = D(w, z, R_Z - R_W) when kept.
__global__ void k_ybuild(DevPlan P, const int* list, int n_list) {
  __shared__ int dsel[kMaxCPerAtom];
  for (int k = blockIdx.x; k < n_list; k += gridDim.x) {
    const int y = list[k];
    const int X = P.y_home[y], z = P.y_j[y];
    const int* Rz = P.y_R + 3 * y;
    const int q0 = P.c_ptr[X], nq = P.c_ptr[X + 1] - q0;
    __syncthreads();
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      const int q = q0 + t;
      int di = -1;
      if (P.c_keep[q]) {
        const int* Rw = P.c_R + 3 * q;
        di = dlut_get(P, P.c_j[q], z, Rz[0] - Rw[0], Rz[1] - Rw[1], Rz[2] - Rw[2]);
        if (di >= 0 && P.Dkept[di] == 0.0) di = -1;
      }
      dsel[t] = di;
    }
    __syncthreads();
    const int sX = P.species[X];
    const int mX = P.n_abf[sX], nX = P.n_ao[sX], nZ = P.n_ao[P.species[z]];
    const int rows = mX * nX;
    const int n = rows * nZ;
    double* Y = P.Yst + P.y_off[y];
    double fl = 0.0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int row = e / nZ, col = e - row * nZ;
      double acc = 0.0;
      for (int t = 0; t < nq; ++t) {
        const int di = dsel[t];
        if (di < 0) continue;
        const int q = q0 + t;
        const int nW = P.n_ao[P.species[P.c_j[q]]];
        const double* Cq = P.Cst + P.c_off[q] + (long long)row * nW;
        const double* Dq = P.Dval + P.Doff[di] + col;
        for (int w = 0; w < nW; ++w) acc += Cq[w] * Dq[w * nZ];
        if (e == 0) fl += 2.0 * (double)n * nW;
      }
      Y[e] = acc;
    }
    if (threadIdx.x == 0) atomicAdd(&P.acc[ACC_FY], fl);
  }
}

// ---------------------------------------------------------------- K4: term 1
// One CTA per (A,B) pair with kept F.  Shared memory: D_AB, R_AB, and a
// beta-chunk of U (bc x n_ao(A) x n_ao(F)).
__global__ void k_term1(DevPlan P, const int* list, int n_list, int BC) {
  extern __shared__ double sm[];
  __shared__ double red[kThreads / 32];
  for (int k = blockIdx.x; k < n_list; k += gridDim.x) {
    const int p = list[k];
    const int A = P.v_home[p], b = P.v_j[p];
    const int* Rb = P.v_R + 3 * p;
    const int sA = P.species[A], sB = P.species[b];
    const int nA = P.n_ao[sA], nB = P.n_ao[sB], mA = P.n_abf[sA], mB = P.n_abf[sB];
    double* Dab = sm;                      // nA*nB
    double* Rs = Dab + kMaxAO * kMaxAO;    // mA*mB
    double* Uc = Rs + mA * mB;             // BC*nA*nF
    const double* Dg = P.Dval + P.Doff[P.v_didx[p]];
    __syncthreads();
    for (int t = threadIdx.x; t < nA * nB; t += blockDim.x) Dab[t] = Dg[t];
    for (int t = threadIdx.x; t < mA * mB; t += blockDim.x) Rs[t] = 0.0;
    __syncthreads();
    const int q0 = P.c_ptr[A];
    double fl = 0.0;
    for (int w = 0; w < kMaskWords; ++w) {
      unsigned bits = P.v_mask[(size_t)p * kMaskWords + w];
      while (bits) {
        const int s = __ffs(bits) - 1;
        bits &= bits - 1u;
        const int q = q0 + w * 32 + s;
        const int f = P.c_j[q];
        const int* Rf = P.c_R + 3 * q;
        const int nF = P.n_ao[P.species[f]];
        const int yc = ylut_get(P, b, f, Rf[0] - Rb[0], Rf[1] - Rb[1], Rf[2] - Rb[2]);
        const double* Y = P.Yst + P.y_off[yc];          // [beta][b][f]
        const double* C = P.Cst + P.c_off[q];           // [alpha][a][f]
        const double* dC = P.dCst + 3 * P.c_off[q];
        const double* V = P.Vst + P.v_off[p];           // [alpha][beta]
        const int naf = nA * nF;
        const int nc = mA * naf;
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int b0 = 0; b0 < mB; b0 += BC) {
          const int bc = min(BC, mB - b0);
          // U_c[bl][a][f] = sum_b D_AB[a][b] Y[b0+bl][b][f]
          for (int e = threadIdx.x; e < bc * naf; e += blockDim.x) {
            const int bl = e / naf, af = e - bl * naf;
            const int a = af / nF, ff = af - a * nF;
            const double* Yr = Y + ((long long)(b0 + bl) * nB) * nF + ff;
            const double* Dr = Dab + a * nB;
            double s2 = 0.0;
            for (int bb = 0; bb < nB; ++bb) s2 += Dr[bb] * Yr[bb * nF];
            Uc[e] = s2;
          }
          __syncthreads();
          // R[alpha][b0+bl] += sum_{a,f} C[alpha][a][f] U_c[bl][a][f]
          for (int e = threadIdx.x; e < mA * bc; e += blockDim.x) {
            const int al = e / bc, bl = e - al * bc;
            const double* Cr = C + (long long)al * naf;
            const double* Ur = Uc + bl * naf;
            double s2 = 0.0;
            for (int t = 0; t < naf; ++t) s2 += Cr[t] * Ur[t];
            Rs[al * mB + b0 + bl] += s2;
          }
          // (V_AB . U)[alpha][a][f] over this chunk, dotted with grad C_AF
          for (int e = threadIdx.x; e < nc; e += blockDim.x) {
            const int al = e / naf, af = e - al * naf;
            const double* Vr = V + (long long)al * mB + b0;
            double s2 = 0.0;
            for (int bl = 0; bl < bc; ++bl) s2 += Vr[bl] * Uc[bl * naf + af];
            g0 += dC[e] * s2;
            g1 += dC[nc + e] * s2;
            g2 += dC[2 * nc + e] * s2;
          }
          __syncthreads();
        }
        g0 = block_sum(g0, red);
        g1 = block_sum(g1, red);
        g2 = block_sum(g2, red);
        if (threadIdx.x == 0) {
          dev::add_gC(P, 3 * q + 0, -2.0 * g0);
          dev::add_gC(P, 3 * q + 1, -2.0 * g1);
          dev::add_gC(P, 3 * q + 2, -2.0 * g2);
          fl += 2.0 * mB * nA * nB * nF + 4.0 * mA * mB * nA * nF;
        }
      }
    }
    __syncthreads();
    // E += -<V_AB, R>,  g^V += -<grad V_AB, R>
    const double* V = P.Vst + P.v_off[p];
    const int n = mA * mB;
    double e0 = 0.0, h0 = 0.0, h1 = 0.0, h2 = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const double r = Rs[t];
      e0 += V[t] * r;
      h0 += V[n + t] * r;
      h1 += V[2 * n + t] * r;
      h2 += V[3 * n + t] * r;
    }
    e0 = block_sum(e0, red);
    h0 = block_sum(h0, red);
    h1 = block_sum(h1, red);
    h2 = block_sum(h2, red);
    if (threadIdx.x == 0) {
      dev::add_E(P, -e0);
      dev::add_gV(P, 3 * p + 0, -h0);
      dev::add_gV(P, 3 * p + 1, -h1);
      dev::add_gV(P, 3 * p + 2, -h2);
      atomicAdd(&P.acc[ACC_F1], fl);
    }
  }
}

// ---------------------------------------------------------------- K5: term 2
// One CTA per (A,B) pair of the second exchange product.  Shared memory:
// an alpha-chunk of Z (ac x n_ao(A) x n_ao(B)) and per-F gradient partials.
__global__ void k_term2(DevPlan P, const int* list, int n_list, int AC) {
  extern __shared__ double sm[];
  __shared__ double red[kThreads / 32];
  for (int k = blockIdx.x; k < n_list; k += gridDim.x) {
    const int p = list[k];
    const int A = P.v_home[p], b = P.v_j[p];
    const int* Rb = P.v_R + 3 * p;
    const int sA = P.species[A], sB = P.species[b];
    const int nA = P.n_ao[sA], nB = P.n_ao[sB], mA = P.n_abf[sA], mB = P.n_abf[sB];
    const int y1 = ylut_get(P, A, b, Rb[0], Rb[1], Rb[2]);
    const int y2 = ylut_get(P, b, A, -Rb[0], -Rb[1], -Rb[2]);
    const double* Yab = P.Yst + P.y_off[y1];   // [alpha][a][b]
    const double* Yba = P.Yst + P.y_off[y2];   // [beta][b][a]
    const double* V = P.Vst + P.v_off[p];
    const int nvb = mA * mB;
    const int nab = nA * nB;
    // R2[alpha][beta] = sum_{a,b} Yab[alpha][a][b] Yba[beta][b][a], dotted at once
    double e0 = 0.0, h0 = 0.0, h1 = 0.0, h2 = 0.0;
    for (int t = threadIdx.x; t < nvb; t += blockDim.x) {
      const int al = t / mB, be = t - al * mB;
      const double* Ya = Yab + (long long)al * nab;
      const double* Yb = Yba + (long long)be * nab;
      double s2 = 0.0;
      for (int a = 0; a < nA; ++a)
        for (int bb = 0; bb < nB; ++bb) s2 += Ya[a * nB + bb] * Yb[bb * nA + a];
      e0 += V[t] * s2;
      h0 += V[nvb + t] * s2;
      h1 += V[2 * nvb + t] * s2;
      h2 += V[3 * nvb + t] * s2;
    }
    e0 = block_sum(e0, red);
    h0 = block_sum(h0, red);
    h1 = block_sum(h1, red);
    h2 = block_sum(h2, red);
    if (threadIdx.x == 0) {
      dev::add_E(P, -e0);
      dev::add_gV(P, 3 * p + 0, -h0);
      dev::add_gV(P, 3 * p + 1, -h1);
      dev::add_gV(P, 3 * p + 2, -h2);
    }
    const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
    double* Zc = sm;                         // AC*nA*nB
    double* gF = Zc + (size_t)AC * nab;      // nq*3
    double* Ds = gF + 3 * kMaxCPerAtom;      // nF*nB (one D_FB at a time)
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * nq; t += blockDim.x) gF[t] = 0.0;
    double fl = 4.0 * mA * mB * nA * nB;
    for (int a0 = 0; a0 < mA; a0 += AC) {
      const int ac = min(AC, mA - a0);
      __syncthreads();
      // Z[al][a][b] = sum_beta V[a0+al][beta] Yba[beta][b][a]
      for (int e = threadIdx.x; e < ac * nab; e += blockDim.x) {
        const int al = e / nab, ab = e - al * nab;
        const int a = ab / nB, bb = ab - a * nB;
        const double* Vr = V + (long long)(a0 + al) * mB;
        double s2 = 0.0;
        for (int be = 0; be < mB; ++be) s2 += Vr[be] * Yba[(long long)be * nab + bb * nA + a];
        Zc[e] = s2;
      }
      __syncthreads();
      for (int t = 0; t < nq; ++t) {
        const int q = q0 + t;
        if (!P.c_keep[q]) continue;
        const int f = P.c_j[q];
        const int* Rf = P.c_R + 3 * q;
        const int di = dlut_get(P, f, b, Rb[0] - Rf[0], Rb[1] - Rf[1], Rb[2] - Rf[2]);
        if (di < 0 || P.Dkept[di] == 0.0) continue;
        const int nF = P.n_ao[P.species[f]];
        const double* Dfb = P.Dval + P.Doff[di];   // [f][b]
        for (int e = threadIdx.x; e < nF * nB; e += blockDim.x) Ds[e] = Dfb[e];
        __syncthreads();
        const double* dC = P.dCst + 3 * P.c_off[q];
        const int naf = nA * nF;
        const int nc = mA * naf;
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        // Q2[a0+al][a][f] = sum_b Z[al][a][b] D_FB[f][b]
        for (int e = threadIdx.x; e < ac * naf; e += blockDim.x) {
          const int al = e / naf, af = e - al * naf;
          const int a = af / nF, ff = af - a * nF;
          const double* Zr = Zc + (long long)al * nab + a * nB;
          const double* Dr = Ds + ff * nB;
          double s2 = 0.0;
          for (int bb = 0; bb < nB; ++bb) s2 += Zr[bb] * Dr[bb];
          const long long ci = (long long)(a0 + al) * naf + af;
          g0 += dC[ci] * s2;
          g1 += dC[nc + ci] * s2;
          g2 += dC[2 * nc + ci] * s2;
        }
        g0 = block_sum(g0, red);
        g1 = block_sum(g1, red);
        g2 = block_sum(g2, red);
        if (threadIdx.x == 0) {
          gF[3 * t + 0] += g0;
          gF[3 * t + 1] += g1;
          gF[3 * t + 2] += g2;
          if (a0 == 0) fl += 2.0 * mA * nA * nB * nF;
        }
        __syncthreads();
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      if (gF[3 * t] != 0.0 || gF[3 * t + 1] != 0.0 || gF[3 * t + 2] != 0.0) {
        const int q = q0 + t;
        dev::add_gC(P, 3 * q + 0, -2.0 * gF[3 * t + 0]);
        dev::add_gC(P, 3 * q + 1, -2.0 * gF[3 * t + 1]);
        dev::add_gC(P, 3 * q + 2, -2.0 * gF[3 * t + 2]);
      }
    }
    if (threadIdx.x == 0) atomicAdd(&P.acc[ACC_F2], fl);
  }
}

// ---------------------------------------------------------------- K7: reduce
// Forces F_I += g, F_J -= g for every pair p = (I -> J, R) and the virial
// sum g (x) d.  out = [E, F (n*3), sigma (9)]; E and the virial come from acc.
__global__ void k_reduce_pairs(DevPlan P, double* F) {
  __shared__ double red[kThreads / 32];
  double w[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) w[c] = 0.0;
  const int total = P.nC + P.nV;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int A, j;
    const int* R;
    double g[3];
    if (t < P.nC) {
      A = P.c_home[t];
      j = P.c_j[t];
      R = P.c_R + 3 * t;
      g[0] = dev::get_gC(P, 3LL * t);
      g[1] = dev::get_gC(P, 3LL * t + 1);
      g[2] = dev::get_gC(P, 3LL * t + 2);
    } else {
      const int p = t - P.nC;
      A = P.v_home[p];
      j = P.v_j[p];
      R = P.v_R + 3 * p;
      g[0] = dev::get_gV(P, 3LL * p);
      g[1] = dev::get_gV(P, 3LL * p + 1);
      g[2] = dev::get_gV(P, 3LL * p + 2);
    }
    if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
    double d[3];
    pair_vector(P, A, j, R, d);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (P.fxF) {   // deterministic plan: exact cells, written to F by k_finish
        dev::fx_add(P.fxF + 2 * (3 * A + c), g[c]);
        dev::fx_add(P.fxF + 2 * (3 * j + c), -g[c]);
      } else {
        atomicAdd(&F[3 * A + c], g[c]);
        atomicAdd(&F[3 * j + c], -g[c]);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) w[3 * a + c] += g[a] * d[c];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const double s = block_sum(w[c], red);
    if (threadIdx.x == 0 && s != 0.0) dev::add_W(P, c, s);
  }
}

__global__ void k_finish(DevPlan P, double* out) {
  if (P.fxF)
    for (int i = threadIdx.x; i < 3 * P.N; i += blockDim.x) out[1 + i] = dev::fx_get(P.fxF + 2 * i);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double L[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) L[k] = P.L[k];
  const double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                     L[2] * (L[3] * L[7] - L[4] * L[6]);
  const double vol = fabs(det);
  out[0] = dev::get_E(P);
  double* sig = out + 1 + 3 * P.N;
  for (int c = 0; c < 9; ++c) sig[c] = -dev::get_W(P, c) / vol;
}

// ---------------------------------------------------------------- scans
__device__ __forceinline__ long long scan_value(const int* flag, const long long* size, const unsigned* mask,
                                                const unsigned char* bytes, int mode, int i) {
  switch (mode) {
    case 0: return flag[i] != 0 ? 1 : 0;
    case 1: return flag[i] != 0 ? size[i] : 0;
    case 2: {
      unsigned any = 0u;
      for (int w = 0; w < kMaskWords; ++w) any |= mask[(size_t)i * kMaskWords + w];
      return any ? 1 : 0;
    }
    case 3: return bytes[i] != 0 ? 1 : 0;
    default: return flag[i];
  }
}

constexpr int kScanItems = 4;
constexpr int kScanTile = kThreads * kScanItems;

// Block-local exclusive scan of a tile; writes block totals.
template <bool kFromValues>
__global__ void k_scan_tile(const int* flag, const long long* size, const unsigned* mask,
                            const unsigned char* bytes, int mode, const long long* vin, int n, long long* out,
                            long long* block_tot) {
  __shared__ long long wsum[kThreads / 32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  long long v[kScanItems];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int i = base + k;
    long long x = 0;
    if (i < n) x = kFromValues ? vin[i] : scan_value(flag, size, mask, bytes, mode, i);
    v[k] = s;
    s += x;
  }
  // inclusive warp scan of per-thread sums
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  long long wpre = 0;
  for (int w = 0; w < wid; ++w) wpre += wsum[w];
  const long long excl = wpre + incl - s;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int i = base + k;
    if (i < n) out[i] = excl + v[k];
  }
  if (threadIdx.x == blockDim.x - 1) block_tot[blockIdx.x] = excl + s;
}

__global__ void k_scan_add(long long* out, int n, const long long* block_pre) {
  const int i = blockIdx.x * kScanTile + threadIdx.x;
  const long long a = block_pre[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    const int j = i + k * kThreads;
    if (j < n && j < (blockIdx.x + 1) * kScanTile) out[j] += a;
  }
}

__global__ void k_scan_total(const long long* out, const int* flag, const long long* size, const unsigned* mask,
                             const unsigned char* bytes, int mode, int n, long long* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *total = n > 0 ? out[n - 1] + scan_value(flag, size, mask, bytes, mode, n - 1) : 0;
}

__global__ void k_scatter(const int* flag, const unsigned* mask, const unsigned char* bytes, int mode, int n,
                          const long long* off, int* list, int base) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (scan_value(flag, nullptr, mask, bytes, mode == 1 ? 0 : mode, i)) list[off[i]] = base + i;
}

int grid_for(long long n, int per_block, int cap = 152 * 32) {
  long long g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Recursive exclusive scan of values (block totals) in place into out.
cudaError_t scan_values(long long* vals, int n, long long* out, long long* tmp, size_t tmp_cap, cudaStream_t s) {
  const int nb = (n + kScanTile - 1) / kScanTile;
  if ((size_t)nb > tmp_cap) return cudaErrorInvalidValue;
  ++g_launches;
  k_scan_tile<true><<<nb, kThreads, 0, s>>>(nullptr, nullptr, nullptr, nullptr, 0, vals, n, out, tmp);
  if (nb > 1) {
    cudaError_t e = scan_values(tmp, nb, tmp, tmp + nb, tmp_cap - nb, s);
    if (e != cudaSuccess) return e;
    ++g_launches;
    k_scan_add<<<nb, kThreads, 0, s>>>(out, n, tmp);
  }
  return cudaGetLastError();
}

}  // namespace

long long launch_count() { return g_launches; }

// Block totals plus the levels of the recursive scan fit in 2*nb + 64.
size_t scan_tmp_need(int n) {
  const size_t nb = n > 0 ? ((size_t)n + kScanTile - 1) / kScanTile : 0;
  return 2 * nb + 64;
}

cudaError_t scan_flags(const int* flag, const long long* size, const unsigned* mask, const unsigned char* bytes,
                       int mode, int n, long long* out, long long* total, ScanTmp& tmp, cudaStream_t s) {
  if (n <= 0) {
    cudaError_t e = cudaMemsetAsync(total, 0, sizeof(long long), s);
    return e;
  }
  const int nb = (n + kScanTile - 1) / kScanTile;
  const size_t need = scan_tmp_need(n);
  if (tmp.cap < need) {
    if (tmp.fixed) return cudaErrorMemoryAllocation;
    tmp.mem.put(tmp.buf, tmp.cap * sizeof(long long));
    tmp.buf = nullptr;
    tmp.cap = 0;
    void* p = nullptr;
    cudaError_t e = tmp.mem.get(&p, need * sizeof(long long));
    if (e != cudaSuccess) return e;
    tmp.buf = static_cast<long long*>(p);
    tmp.cap = need;
  }
  ++g_launches;
  k_scan_tile<false><<<nb, kThreads, 0, s>>>(flag, size, mask, bytes, mode, nullptr, n, out, tmp.buf);
  if (nb > 1) {
    cudaError_t e = scan_values(tmp.buf, nb, tmp.buf, tmp.buf + nb, tmp.cap - nb, s);
    if (e != cudaSuccess) return e;
    ++g_launches;
    k_scan_add<<<nb, kThreads, 0, s>>>(out, n, tmp.buf);
  }
  ++g_launches;
  k_scan_total<<<1, 32, 0, s>>>(out, flag, size, mask, bytes, mode, n, total);
  return cudaGetLastError();
}

cudaError_t scatter_list(const int* flag, const unsigned* mask, const unsigned char* bytes, int mode, int n,
                         const long long* off, int* list, int base, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++g_launches;
  k_scatter<<<grid_for(n, kThreads), kThreads, 0, s>>>(flag, mask, bytes, mode, n, off, list, base);
  return cudaGetLastError();
}

cudaError_t launch_dnorm(const DevPlan& P, cudaStream_t s) {
  if (P.n_d == 0) return cudaSuccess;
  ++g_launches;
  k_dnorm<<<grid_for(P.n_d, 1, 152 * 64), kThreads, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_cblocks(const DevPlan& P, int frozen, cudaStream_t s) {
  if (P.nC == 0) return cudaSuccess;
  ++g_launches;
  k_cblocks<<<grid_for(P.nC, 1, 152 * 64), kThreads, 0, s>>>(P, frozen);
  return cudaGetLastError();
}

cudaError_t launch_cnorm(const DevPlan& P, int frozen, cudaStream_t s) {
  if (P.nC == 0) return cudaSuccess;
  ++g_launches;
  k_cnorm<<<grid_for(P.nC, kThreads), kThreads, 0, s>>>(P, frozen);
  return cudaGetLastError();
}

cudaError_t launch_vnorm(const DevPlan& P, int frozen, cudaStream_t s) {
  if (P.nV == 0) return cudaSuccess;
  ++g_launches;
  k_vnorm<<<grid_for(P.nV, kThreads), kThreads, 0, s>>>(P, frozen);
  return cudaGetLastError();
}

cudaError_t launch_yhat(const DevPlan& P, cudaStream_t s) {
  if (P.nY == 0) return cudaSuccess;
  ++g_launches;
  k_yhat<<<grid_for(P.nY, kThreads), kThreads, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_screen(const DevPlan& P, cudaStream_t s) {
  if (P.nV == 0) return cudaSuccess;
  ++g_launches;
  k_screen<<<grid_for(P.nV, kThreads), kThreads, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_vblocks(const DevPlan& P, const int* list, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_launches;
  k_vblocks<<<grid_for(n, 1, 152 * 64), kThreads, 0, s>>>(P, list, n);
  return cudaGetLastError();
}

cudaError_t launch_ybuild(const DevPlan& P, const int* list, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_launches;
  k_ybuild<<<grid_for(n, 1, 152 * 64), kThreads, 0, s>>>(P, list, n);
  return cudaGetLastError();
}

cudaError_t allow_max_dynamic_smem(const void* f) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes a{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, f);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
}

cudaError_t set_kernel_smem_limits() {
  cudaError_t e = allow_max_dynamic_smem((const void*)k_term1);
  if (e != cudaSuccess) return e;
  return allow_max_dynamic_smem((const void*)k_term2);
}

cudaError_t launch_term1(const DevPlan& P, const int* list, int n, int beta_chunk, size_t smem, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_launches;
  k_term1<<<grid_for(n, 1, 152 * 64), kThreads, smem, s>>>(P, list, n, beta_chunk);
  return cudaGetLastError();
}

cudaError_t launch_term2(const DevPlan& P, const int* list, int n, int alpha_chunk, size_t smem, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_launches;
  k_term2<<<grid_for(n, 1, 152 * 64), kThreads, smem, s>>>(P, list, n, alpha_chunk);
  return cudaGetLastError();
}

// ------------------------------------------------------------ LRI fit
// Eq. C_VA and the gradient equation after Eq. V_inverse, per atom pair p of
// a batch (one CTA per pair, grid-stride over the batch):
//   A X = B                       X = the C^I rows, then the C^K rows
//   A dX[c] = dB[c] - dA[c] X     c = x, y, z (gradient in K's position)
// A (n x n, SPD) is factored as L L^T (left-looking Cholesky, L in shared
// memory); each thread then owns RHS columns and runs the forward and back
// substitutions on them in place in the output (row-major [n][w], so the
// threads of a warp touch consecutive columns of one row), reading L by
// broadcast.  A pivot <= 0 (A not positive definite) sets *err and is
// replaced by 1 so that the CTA finishes.
namespace {

__device__ void lri_cholesky(double* L, const double* A, int n, int* err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < n * n; e += blockDim.x) L[e] = A[e];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      double sq = 0.0;
      for (int k = lane; k < j; k += 32) sq += L[j * n + k] * L[j * n + k];
      sq = warp_sum(sq);
      if (lane == 0) {
        double d = L[j * n + j] - sq;
        if (!(d > 0.0)) {
          atomicExch(err, 1);
          d = 1.0;
        }
        L[j * n + j] = sqrt(d);
      }
    }
    __syncthreads();
    const double ljj = L[j * n + j];
    for (int i = j + 1 + tid; i < n; i += blockDim.x) {
      double a = L[i * n + j];
      for (int k = 0; k < j; ++k) a -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = a / ljj;
    }
    __syncthreads();
  }
}

// In-place solve L L^T x = r for the columns this thread owns of the
// row-major n x w array R.
__device__ void lri_substitute(const double* L, double* R, int n, int w) {
  for (int col = threadIdx.x; col < w; col += blockDim.x) {
    for (int i = 0; i < n; ++i) {   // L y = r
      double a = R[(size_t)i * w + col];
      for (int k = 0; k < i; ++k) a -= L[i * n + k] * R[(size_t)k * w + col];
      R[(size_t)i * w + col] = a / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {   // L^T x = y
      double a = R[(size_t)i * w + col];
      for (int k = i + 1; k < n; ++k) a -= L[k * n + i] * R[(size_t)k * w + col];
      R[(size_t)i * w + col] = a / L[i * n + i];
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_lri_fit(int batch, int n, int w, const double* A, const double* B,
                                                     const double* dA, const double* dB, double* X, double* dX,
                                                     int* err) {
  extern __shared__ double L[];   // [n][n]
  const size_t nn = (size_t)n * n, nw = (size_t)n * w;
  for (int p = blockIdx.x; p < batch; p += gridDim.x) {
    __syncthreads();   // the previous pair's L is no longer read
    lri_cholesky(L, A + p * nn, n, err);
    double* Xp = X + p * nw;
    const double* Bp = B + p * nw;
    for (size_t e = threadIdx.x; e < nw; e += blockDim.x) Xp[e] = Bp[e];
    __syncthreads();
    lri_substitute(L, Xp, n, w);
    if (dX == nullptr) continue;
    __syncthreads();   // X complete (each thread solved its own columns; rows mix below)
    for (int c = 0; c < 3; ++c) {
      const double* dAc = dA + (p * 3 + c) * nn;
      const double* dBc = dB + (p * 3 + c) * nw;
      double* R = dX + (p * 3 + c) * nw;
      for (int col = threadIdx.x; col < w; col += blockDim.x)
        for (int i = 0; i < n; ++i) {
          double a = dBc[(size_t)i * w + col];
          for (int j = 0; j < n; ++j) a -= dAc[(size_t)i * n + j] * Xp[(size_t)j * w + col];
          R[(size_t)i * w + col] = a;
        }
      lri_substitute(L, R, n, w);
    }
  }
}

}  // namespace

size_t lri_fit_smem(int n) { return (size_t)n * n * sizeof(double); }

cudaError_t launch_lri_fit(int batch, int n, int w, const double* A, const double* B, const double* dA,
                           const double* dB, double* X, double* dX, int* err, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const size_t smem = lri_fit_smem(n);
  cudaError_t e = allow_max_dynamic_smem((const void*)k_lri_fit);
  if (e != cudaSuccess) return e;
  ++g_launches;
  k_lri_fit<<<grid_for(batch, 1, 152 * 2), kThreads, smem, s>>>(batch, n, w, A, B, dA, dB, X, dX, err);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const DevPlan& P, double* out, cudaStream_t s) {
  double* F = out + 1;
  const int total = P.nC + P.nV;
  ++g_launches;
  k_reduce_pairs<<<grid_for(total, kThreads, 152 * 4), kThreads, 0, s>>>(P, F);
  ++g_launches;
  k_finish<<<1, 32, 0, s>>>(P, out);
  return cudaGetLastError();
}

}  // namespace hfx
