// Split-precision tensor-core kernels of the HFX force/stress hot path.
//
// Every FP64 operand x of a contraction is written as NP bf16 pieces
// x = p0 + p1 (+ p2) + r (p0 = bf16(x), p1 = bf16(x - p0), ...), and each
// product keeps the piece pairs (i, j) with i + j < NP: three warp-level
// MMAs for NP = 2, six for NP = 3 (the BF16x3 / BF16x6 splits of Henry,
// Tang & Heinecke).  Accumulation is FP32 in the MMA and FP64 beyond a
// short run; the screening, the pair gradients, E, F and sigma stay FP64.
//
// Operand stores, written once per evaluation from the FP64 blocks
// (k_cpieces, k_vpieces): per C pair, NP bf16 planes of C [(alpha,a)][rup16(f)]
// and grad C in FP32; per needed V pair, NP bf16 planes of V [alpha][rup16(beta)]
// and V, grad V in FP32.  No FP64 arithmetic runs inside the item loops.
//
// Same factorisation as the FP64 kernels (Eq. exx_expand by the
// distributive law), with the first exchange product organised per
// (A, F) pair so that Q_AF = sum_B V_AB . U_ABF accumulates inside the
// MMA accumulators:
//   Y^{XZ}[alpha][z][x] = sum_W C_XW . D_WZ                (k_ybuild_mma)
//   per (A,F), over its kept B:                             (k_term1_mma)
//     U[(beta,f)][a] = sum_b Y^{BF}[(beta,f)][b] D_AB[a][b]
//     R = C_AF . U^T  -> E += -<V,R>, g^V += -<grad V,R>
//     Q += V_AB . U   -> g^C_AF = -2 <grad C_AF, Q>
//   per (A,B) of the second product:                        (k_term2_mma)
//     R2 = <Y^{AB}, Y^{BA}>;  Z = V_AB . Y^{BA};  Q2_F = Z . D_FB^T
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "hfx_internal.h"

namespace hfx {
namespace {

constexpr int kWarps1 = 16;     // warps per CTA of the term-1 kernel
constexpr int kWarps = 8;       // warps per CTA of the other mixed kernels
constexpr int kQT = 16;         // Q accumulator tiles per warp (term 1)
constexpr int kYT = 4;          // m-tiles per warp per pass (Y build)
constexpr int kFlush = 8;       // B per FP32 run of the Q accumulators
long long g_mix_launches = 0;

__device__ __forceinline__ int rup16(int x) { return (x + 15) & ~15; }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NV doubles (all threads get the sums).  red: >= 32*NV doubles.
template <int NV>
__device__ void block_sum_n(double (&v)[NV], double* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum_d(v[i]);
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * 32 + w] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += red[i * 32 + k];
    v[i] = t;
  }
  __syncthreads();
}

template <int NP>
__device__ __forceinline__ void split_f(float x, uint16_t (&p)[NP]) {
  float r = x;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const __nv_bfloat16 h = __float2bfloat16_rn(r);
    p[i] = __bfloat16_as_ushort(h);
    r -= __bfloat162float(h);
  }
}

__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// All piece products (i, j) with i + j < NP, smallest first.
template <int NP>
__device__ __forceinline__ void mma_split(float (&c)[4], const uint32_t (&a)[NP][4], const uint32_t (&b)[NP][2]) {
  if (NP == 3) {
    mma16816(c, a[1], b[1]);
    mma16816(c, a[0], b[2]);
    mma16816(c, a[2], b[0]);
  }
  if (NP >= 2) {
    mma16816(c, a[0], b[1]);
    mma16816(c, a[1], b[0]);
  }
  mma16816(c, a[0], b[0]);
}

__device__ __forceinline__ void ldm_x4(uint32_t (&r)[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldm_x2(uint32_t (&r)[2], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

__device__ __forceinline__ void ldm_x2_trans(uint32_t (&r)[2], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

__device__ __forceinline__ int ylut_get(const DevPlan& P, int i, int j, int r0, int r1, int r2) {
  if (r0 < -P.HY0 || r0 > P.HY0 || r1 < -P.HY1 || r1 > P.HY1 || r2 < -P.HY2 || r2 > P.HY2) return -1;
  const long long n0 = 2 * P.HY0 + 1, n1 = 2 * P.HY1 + 1, n2 = 2 * P.HY2 + 1;
  const long long idx = (((((long long)i * P.N + j) * n0 + (r0 + P.HY0)) * n1 + (r1 + P.HY1)) * n2) + (r2 + P.HY2);
  return P.ylut[idx];
}

__device__ __forceinline__ int dlut_get(const DevPlan& P, int i, int j, int r0, int r1, int r2) {
  if (r0 < -P.HD0 || r0 > P.HD0 || r1 < -P.HD1 || r1 > P.HD1 || r2 < -P.HD2 || r2 > P.HD2) return -1;
  const long long n0 = 2 * P.HD0 + 1, n1 = 2 * P.HD1 + 1, n2 = 2 * P.HD2 + 1;
  const long long idx = (((((long long)i * P.N + j) * n0 + (r0 + P.HD0)) * n1 + (r1 + P.HD1)) * n2) + (r2 + P.HD2);
  return P.dlut[idx];
}

// ------------------------------------------------------------------ D split
// D block k (n_ao(I) x n_ao(J)) -> NP bf16 planes of rup16(n_ao(I)) x rup16(n_ao(J)), zero padded.
template <int NP>
__global__ void k_dsplit(DevPlan P, MixPlan X) {
  for (long long k = blockIdx.x; k < P.n_d; k += gridDim.x) {
    const int I = P.Didx[5 * k], J = P.Didx[5 * k + 1];
    const int na = P.n_ao[P.species[I]], nb = P.n_ao[P.species[J]];
    const int pa = rup16(na), pb = rup16(nb);
    uint16_t* out = X.Dsp + X.dsp_off[k];
    const double* src = P.Dval + P.Doff[k];
    for (int e = threadIdx.x; e < pa * pb; e += blockDim.x) {
      const int a = e / pb, b = e - a * pb;
      uint16_t pc[NP];
      split_f<NP>((a < na && b < nb) ? (float)src[a * nb + b] : 0.f, pc);
#pragma unroll
      for (int p = 0; p < NP; ++p) out[p * pa * pb + e] = pc[p];
    }
  }
}

// ------------------------------------------------------------------ pieces
// C pair q: NP bf16 planes of C[(alpha,a)][rup16(n_ao(F))] then grad C (FP32).
template <int NP>
__global__ void k_cpieces(DevPlan P, MixPlan X) {
  for (int q = blockIdx.x; q < P.nC; q += gridDim.x) {
    if (!P.c_keep[q]) continue;
    const int A = P.c_home[q], f = P.c_j[q];
    const int sA = P.species[A], sF = P.species[f];
    const int rows = P.n_abf[sA] * P.n_ao[sA], nF = P.n_ao[sF], pF = rup16(nF);
    const double* C = P.Cst + P.c_off[q];
    const double* dC = P.dCst + 3 * P.c_off[q];
    uint16_t* out = X.Cm + X.cm_off[q];
    for (int e = threadIdx.x; e < rows * pF; e += blockDim.x) {
      const int r = e / pF, c = e - r * pF;
      uint16_t pc[NP];
      split_f<NP>(c < nF ? (float)C[r * nF + c] : 0.f, pc);
#pragma unroll
      for (int p = 0; p < NP; ++p) out[p * rows * pF + e] = pc[p];
    }
    float* g = reinterpret_cast<float*>(out + NP * rows * pF);
    for (int e = threadIdx.x; e < 3 * rows * nF; e += blockDim.x) g[e] = (float)dC[e];
  }
}

// needed V pair p: NP bf16 planes of V[alpha][rup16(n_abf(B))] then V, grad V (FP32).
template <int NP>
__global__ void k_vpieces(DevPlan P, MixPlan X, const int* list, int n_list) {
  for (int k = blockIdx.x; k < n_list; k += gridDim.x) {
    const int p = list[k];
    const int mA = P.n_abf[P.species[P.v_home[p]]], mB = P.n_abf[P.species[P.v_j[p]]];
    const int MB = rup16(mB);
    const double* V = P.Vst + P.v_off[p];
    uint16_t* out = X.Vm + X.vm_off[p];
    for (int e = threadIdx.x; e < mA * MB; e += blockDim.x) {
      const int al = e / MB, be = e - al * MB;
      uint16_t pc[NP];
      split_f<NP>(be < mB ? (float)V[al * mB + be] : 0.f, pc);
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) out[pp * mA * MB + e] = pc[pp];
    }
    float* v32 = reinterpret_cast<float*>(out + NP * mA * MB);
    for (int e = threadIdx.x; e < 4 * mA * mB; e += blockDim.x) v32[e] = (float)V[e];
  }
}

// ------------------------------------------------------------------ Y build
// One CTA per needed key (X; Z).  Rows (alpha, x), columns z, K = (W, w):
// Y[(alpha,x)][z] = sum_W sum_w C_XW[(alpha,x)][w] D_WZ[w][z].  The B
// fragments come from the mirror block D_ZW = D_WZ^T (row z, column w).
// Output: NP planes of [alpha][z][rup16(n_ao(X))], x padding zeroed.
template <int NP, int NTM>
__global__ void __launch_bounds__(kWarps * 32, 2) k_ybuild_mma(DevPlan P, MixPlan X, const int* list, int n_list) {
  __shared__ int dsel[kMaxCPerAtom];   // mirror D block (index into Dsp) per C slot, -1 = none
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  for (int kk = blockIdx.x; kk < n_list; kk += gridDim.x) {
    const int y = list[kk];
    const int Xa = P.y_home[y], z = P.y_j[y];
    const int* Rz = P.y_R + 3 * y;
    const int q0 = P.c_ptr[Xa], nq = P.c_ptr[Xa + 1] - q0;
    __syncthreads();
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      const int q = q0 + t;
      int sel = -1;
      if (P.c_keep[q]) {
        const int* Rw = P.c_R + 3 * q;
        const int w = P.c_j[q];
        const int di = dlut_get(P, w, z, Rz[0] - Rw[0], Rz[1] - Rw[1], Rz[2] - Rw[2]);
        if (di >= 0 && P.Dkept[di] != 0.0) sel = dlut_get(P, z, w, Rw[0] - Rz[0], Rw[1] - Rz[1], Rw[2] - Rz[2]);
      }
      dsel[t] = sel;
    }
    __syncthreads();
    const int sX = P.species[Xa], sZ = P.species[z];
    const int mX = P.n_abf[sX], nX = P.n_ao[sX], nZ = P.n_ao[sZ];
    const int pX = rup16(nX), pZ = rup16(nZ);
    const int rows = mX * nX;
    const int MT = (rows + 15) >> 4;
    const int NT = pZ >> 3;                 // <= NTM
    uint16_t* Yo = X.Ysp + P.y_off[y];
    const long long plane = (long long)mX * nZ * pX;
    for (int mbase = 0; mbase < MT; mbase += kYT * kWarps) {
    float acc[kYT][NTM][4];
#pragma unroll
    for (int i = 0; i < kYT; ++i)
#pragma unroll
      for (int j = 0; j < NTM; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
    for (int t = 0; t < nq; ++t) {
      const int sel = dsel[t];
      if (sel < 0) continue;
      const int q = q0 + t;
      const int nW = P.n_ao[P.species[P.c_j[q]]];
      const int pW = rup16(nW);
      const uint16_t* Cq = X.Cm + X.cm_off[q];          // planes [(alpha,x)][pW]
      const long long cplane = (long long)rows * pW;
      const uint16_t* Dm = X.Dsp + X.dsp_off[sel];   // mirror block, [z][w] planes of pZ x pW
      for (int k0 = 0; k0 < pW; k0 += 16) {
        uint32_t bf[NTM][NP][2];
#pragma unroll
        for (int nt = 0; nt < NTM; ++nt) {
          if (nt < NT) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              const uint16_t* Db = Dm + p * pZ * pW + (nt * 8 + gid) * pW + k0 + 2 * tig;
              bf[nt][p][0] = *reinterpret_cast<const uint32_t*>(Db);
              bf[nt][p][1] = *reinterpret_cast<const uint32_t*>(Db + 8);
            }
          }
        }
#pragma unroll
        for (int i = 0; i < kYT; ++i) {
          const int mt = mbase + warp + i * kWarps;
          if (mt >= MT) break;
          uint32_t af[NP][4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int r = mt * 16 + gid + ((h & 1) ? 8 : 0);
            const int kc = k0 + 2 * tig + ((h & 2) ? 8 : 0);
#pragma unroll
            for (int p = 0; p < NP; ++p)
              af[p][h] = r < rows ? *reinterpret_cast<const uint32_t*>(Cq + p * cplane + (long long)r * pW + kc) : 0u;
          }
#pragma unroll
          for (int nt = 0; nt < NTM; ++nt)
            if (nt < NT) mma_split<NP>(acc[i][nt], af, bf[nt]);
        }
      }
    }
    // store Y planes [alpha][z][x], x padding zeroed
#pragma unroll
    for (int i = 0; i < kYT; ++i) {
      const int mt = mbase + warp + i * kWarps;
      if (mt >= MT) break;
#pragma unroll
      for (int nt = 0; nt < NTM; ++nt) {
        if (nt >= NT) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int r = mt * 16 + gid + ((c & 2) ? 8 : 0);
          const int zc = nt * 8 + 2 * tig + (c & 1);
          if (r < rows && zc < nZ) {
            const int al = r / nX, x = r - al * nX;
            uint16_t pc[NP];
            split_f<NP>(acc[i][nt][c], pc);
            const long long o = ((long long)al * nZ + zc) * pX + x;
#pragma unroll
            for (int p = 0; p < NP; ++p) Yo[p * plane + o] = pc[p];
          }
        }
      }
    }
    }  // m-tile groups
    if (pX > nX) {
      for (long long e = threadIdx.x; e < (long long)mX * nZ * (pX - nX); e += blockDim.x) {
        const long long rz = e / (pX - nX);
        const int x = nX + (int)(e - rz * (pX - nX));
#pragma unroll
        for (int p = 0; p < NP; ++p) Yo[p * plane + rz * pX + x] = 0;
      }
    }
    if (threadIdx.x == 0) {
      double fl = 0.0;
      for (int t = 0; t < nq; ++t)
        if (dsel[t] >= 0) fl += 2.0 * rows * nZ * P.n_ao[P.species[P.c_j[q0 + t]]];
      atomicAdd(&P.acc[ACC_FY], fl);
    }
  }
}

// --------------------------------------------------- term-1 transposed lists
// Per home atom A: for every C slot of A, the V pairs (A,B) whose item list
// keeps it, in V-pair order (deterministic).
__global__ void k_t1_count(DevPlan P, MixPlan X) {
  const int A = blockIdx.x;
  const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
  for (int s = threadIdx.x; s < nq; s += blockDim.x) {
    int cnt = 0;
    for (int p = P.v_ptr[A]; p < P.v_ptr[A + 1]; ++p)
      cnt += (P.v_mask[(size_t)p * kMaskWords + (s >> 5)] >> (s & 31)) & 1u;
    X.qcnt[q0 + s] = cnt;
  }
}

__global__ void k_t1_fill(DevPlan P, MixPlan X) {
  const int A = blockIdx.x;
  const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
  for (int s = threadIdx.x; s < nq; s += blockDim.x) {
    long long o = X.qoff[q0 + s];
    for (int p = P.v_ptr[A]; p < P.v_ptr[A + 1]; ++p)
      if ((P.v_mask[(size_t)p * kMaskWords + (s >> 5)] >> (s & 31)) & 1u) X.blist[o++] = p;
  }
}

// ------------------------------------------------------------------ term 1
// One CTA (16 warps) per (A,F) with kept B.  Shared memory (bf16 planes):
//   Cs[NP][MA][KS]  C_AF, rows alpha, K = (a,f) (row stride KS)
//   Us[NP][MB][KS]  U of the current B, rows beta, K = (a,f)
//   Vs[NP][MA][VS]  V_AB of the current B, rows alpha, K = beta
template <int NP>
__global__ void __launch_bounds__(kWarps1 * 32) k_term1_mma(DevPlan P, MixPlan X, const int* qlist, int n_list,
                                                            int MAmax, int MBmax, int KSmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 4];
  __shared__ double sacc[4];    // E and g^V partials of the current triplet (E over the item)
  __shared__ int sprev;         // V pair whose g^V partials are in sacc[1..3]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  uint16_t* Cs = reinterpret_cast<uint16_t*>(smem);
  uint16_t* Us = Cs + (size_t)NP * MAmax * KSmax;
  uint16_t* Vs = Us + (size_t)NP * MBmax * KSmax;
  const int VS = MBmax + 8;
  for (int kk = blockIdx.x; kk < n_list; kk += gridDim.x) {
    const int q = qlist[kk];
    const int A = P.c_home[q], f = P.c_j[q];
    const int* Rf = P.c_R + 3 * q;
    const int sA = P.species[A], sF = P.species[f];
    const int nA = P.n_ao[sA], nF = P.n_ao[sF], mA = P.n_abf[sA];
    const int pA = rup16(nA);
    const int KAF = nA * nF, KP = rup16(KAF), KS = KP + 8, MA = rup16(mA);
    const int MT = MA >> 4, NTq = (KAF + 7) >> 3;
    __syncthreads();
    if (threadIdx.x == 0) {
      sacc[0] = sacc[1] = sacc[2] = sacc[3] = 0.0;
      sprev = -1;
    }
    // C_AF pieces -> Cs[alpha][a*nF + f] (zero padded)
    const int pF = rup16(nF);
    const uint16_t* Cq = X.Cm + X.cm_off[q];
    const long long cplane = (long long)mA * nA * pF;
    {
      for (int e = threadIdx.x; e < MA * KS; e += blockDim.x) {
        const int al = e / KS, k = e - al * KS;
        const bool in = al < mA && k < KAF;
        const int a = in ? k / nF : 0, ff = in ? k - a * nF : 0;
#pragma unroll
        for (int p = 0; p < NP; ++p)
          Cs[(size_t)p * MA * KS + e] = in ? Cq[p * cplane + ((long long)al * nA + a) * pF + ff] : (uint16_t)0;
      }
    }
    float qacc[kQT][4];
#pragma unroll
    for (int i = 0; i < kQT; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) qacc[i][c] = 0.f;
    double g[3] = {0.0, 0.0, 0.0};
    const float* dC = reinterpret_cast<const float*>(Cq + NP * cplane);   // grad C, FP32
    const long long ncq = (long long)mA * KAF;
    const long long b0i = X.qoff[q], b1i = b0i + X.qcnt[q];
    unsigned long long fl = 0ull;
    for (long long bi = b0i; bi < b1i; ++bi) {
      const int p = X.blist[bi];
      const int b = P.v_j[p];
      const int* Rb = P.v_R + 3 * p;
      const int sB = P.species[b];
      const int nB = P.n_ao[sB], mB = P.n_abf[sB];
      const int pB = rup16(nB);
      const int MB = rup16(mB);
      const int yc = ylut_get(P, b, f, Rf[0] - Rb[0], Rf[1] - Rb[1], Rf[2] - Rb[2]);
      const uint16_t* Y = X.Ysp + P.y_off[yc];             // [beta][f][pB] planes
      const long long yplane = (long long)mB * nF * pB;
      const uint16_t* Dab = X.Dsp + X.dsp_off[P.v_didx[p]];  // [a][pB] planes of pA x pB
      const uint16_t* Vp = X.Vm + X.vm_off[p];                // V pieces [alpha][MB]
      const float* V = reinterpret_cast<const float*>(Vp + NP * mA * MB);   // V, grad V (FP32)
      const int nvb = mA * mB;
      __syncthreads();   // previous B done with Us / Vs and with sacc
      if (threadIdx.x == 0) {
        if (sprev >= 0) {
          atomicAdd(&P.gV[3 * sprev + 0], -sacc[1]);
          atomicAdd(&P.gV[3 * sprev + 1], -sacc[2]);
          atomicAdd(&P.gV[3 * sprev + 2], -sacc[3]);
        }
        sacc[1] = sacc[2] = sacc[3] = 0.0;
        sprev = p;
        fl += 2ull * mB * nA * nB * nF + 4ull * mA * mB * nA * nF;
      }
      // V_AB pieces -> Vs
      for (int e = threadIdx.x; e < MA * MB; e += blockDim.x) {
        const int al = e / MB, be = e - al * MB;
#pragma unroll
        for (int pp = 0; pp < NP; ++pp)
          Vs[(size_t)pp * MA * VS + al * VS + be] = al < mA ? Vp[pp * mA * MB + e] : (uint16_t)0;
      }
      // zero the Us rows beyond mB (their K range is never written by U)
      for (int e = threadIdx.x; e < (MB - mB) * KS; e += blockDim.x) {
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) Us[(size_t)pp * MB * KS + (size_t)mB * KS + e] = 0;
      }
      // columns KAF..KS of the valid rows
      for (int e = threadIdx.x; e < mB * (KS - KAF); e += blockDim.x) {
        const int be = e / (KS - KAF), k = KAF + (e - be * (KS - KAF));
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) Us[(size_t)pp * MB * KS + (size_t)be * KS + k] = 0;
      }
      // U[(beta,f)][a] = sum_b Y[(beta,f)][b] D_AB[a][b]  ->  Us[beta][a*nF + f]
      {
        const int rowsU = mB * nF;
        const int MTU = (rowsU + 15) >> 4;
        const int NTU = pA >> 3;   // <= 4
        for (int mt = warp; mt < MTU; mt += kWarps1) {
          float acc[4][4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[j][c] = 0.f;
          for (int k0 = 0; k0 < pB; k0 += 16) {
            uint32_t af[NP][4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int r = mt * 16 + gid + ((h & 1) ? 8 : 0);
              const int kc = k0 + 2 * tig + ((h & 2) ? 8 : 0);
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                af[pp][h] = r < rowsU ? *reinterpret_cast<const uint32_t*>(Y + pp * yplane + (long long)r * pB + kc) : 0u;
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              if (nt >= NTU) break;
              uint32_t bf[NP][2];
#pragma unroll
              for (int pp = 0; pp < NP; ++pp) {
                const uint16_t* Db = Dab + pp * pA * pB + (nt * 8 + gid) * pB + k0 + 2 * tig;
                bf[pp][0] = *reinterpret_cast<const uint32_t*>(Db);
                bf[pp][1] = *reinterpret_cast<const uint32_t*>(Db + 8);
              }
              mma_split<NP>(acc[nt], af, bf);
            }
          }
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            if (nt >= NTU) break;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int r = mt * 16 + gid + ((c & 2) ? 8 : 0);
              const int a = nt * 8 + 2 * tig + (c & 1);
              if (r < rowsU && a < nA) {
                const int be = r / nF, ff = r - be * nF;
                uint16_t pc[NP];
                split_f<NP>(acc[nt][c], pc);
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) Us[(size_t)pp * MB * KS + (size_t)be * KS + a * nF + ff] = pc[pp];
              }
            }
          }
        }
      }
      __syncthreads();
      // R_t = C_AF . U^T (M = alpha, N = beta, K = (a,f)); dotted with V and grad V
      float evf[4] = {0.f, 0.f, 0.f, 0.f};
      {
        const int NTR = MB >> 3;
        const int nt_tiles = MT * NTR;
        for (int t = warp; t < nt_tiles; t += kWarps1) {
          const int mt = t / NTR, nt = t - mt * NTR;
          float acc[4] = {0.f, 0.f, 0.f, 0.f};
          for (int k0 = 0; k0 < KP; k0 += 16) {
            uint32_t af[NP][4], bf[NP][2];
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
              ldm_x4(af[pp], Cs + (size_t)pp * MA * KS + (size_t)(mt * 16 + (lane & 15)) * KS + k0 + ((lane >> 4) << 3));
              ldm_x2(bf[pp], Us + (size_t)pp * MB * KS + (size_t)(nt * 8 + (lane & 7)) * KS + k0 + (((lane >> 3) & 1) << 3));
            }
            mma_split<NP>(acc, af, bf);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
            const int be = nt * 8 + 2 * tig + (c & 1);
            if (al < mA && be < mB) {
              const int o = al * mB + be;
              const float r = acc[c];
              evf[0] = fmaf(V[o], r, evf[0]);
              evf[1] = fmaf(V[nvb + o], r, evf[1]);
              evf[2] = fmaf(V[2 * nvb + o], r, evf[2]);
              evf[3] = fmaf(V[3 * nvb + o], r, evf[3]);
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float w = warp_sum_f(evf[c]);
        if (lane == 0) atomicAdd(&sacc[c], (double)w);
      }
      // Q += V_AB . U (M = alpha, N = (a,f), K = beta)
      {
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
          const int t = warp + i * kWarps1;
          if (t >= MT * NTq) continue;
          const int mt = t / NTq, nt = t - mt * NTq;
          for (int k0 = 0; k0 < MB; k0 += 16) {
            uint32_t af[NP][4], bf[NP][2];
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
              ldm_x4(af[pp], Vs + (size_t)pp * MA * VS + (size_t)(mt * 16 + (lane & 15)) * VS + k0 + ((lane >> 4) << 3));
              ldm_x2_trans(bf[pp], Us + (size_t)pp * MB * KS + (size_t)(k0 + (lane & 15)) * KS + nt * 8);
            }
            mma_split<NP>(qacc[i], af, bf);
          }
        }
      }
      // flush the FP32 run of Q into the FP64 gradient dot
      if (((bi - b0i) % kFlush) == kFlush - 1 || bi + 1 == b1i) {
        float gf[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
          const int t = warp + i * kWarps1;
          if (t >= MT * NTq) continue;
          const int mt = t / NTq, nt = t - mt * NTq;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
            const int n = nt * 8 + 2 * tig + (c & 1);
            if (al < mA && n < KAF) {
              const long long o = (long long)al * KAF + n;
              const float v = qacc[i][c];
              gf[0] = fmaf(dC[o], v, gf[0]);
              gf[1] = fmaf(dC[ncq + o], v, gf[1]);
              gf[2] = fmaf(dC[2 * ncq + o], v, gf[2]);
            }
            qacc[i][c] = 0.f;
          }
        }
        g[0] += (double)gf[0];
        g[1] += (double)gf[1];
        g[2] += (double)gf[2];
      }
    }
    block_sum_n<3>(g, red);   // once per (A,F) item; also orders sacc
    if (threadIdx.x == 0) {
      atomicAdd(&P.gC[3 * q + 0], -2.0 * g[0]);
      atomicAdd(&P.gC[3 * q + 1], -2.0 * g[1]);
      atomicAdd(&P.gC[3 * q + 2], -2.0 * g[2]);
      if (sprev >= 0) {
        atomicAdd(&P.gV[3 * sprev + 0], -sacc[1]);
        atomicAdd(&P.gV[3 * sprev + 1], -sacc[2]);
        atomicAdd(&P.gV[3 * sprev + 2], -sacc[3]);
      }
      atomicAdd(&P.acc[ACC_E], -sacc[0]);
      atomicAdd(&P.acc[ACC_F1], (double)fl);
    }
  }
}

// ------------------------------------------------------------------ term 2
// One CTA per (A,B) of the second product.  Shared memory: Zs[NP][(alpha,a)][ZS]
// (bf16 planes, K = b, row stride ZS = rup16(n_ao(B)) + 8) and gF[nq][3].
template <int NP>
__global__ void __launch_bounds__(kWarps * 32) k_term2_mma(DevPlan P, MixPlan X, const int* list, int n_list,
                                                           int ZROWS) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  for (int kk = blockIdx.x; kk < n_list; kk += gridDim.x) {
    const int p = list[kk];
    const int A = P.v_home[p], b = P.v_j[p];
    const int* Rb = P.v_R + 3 * p;
    const int sA = P.species[A], sB = P.species[b];
    const int nA = P.n_ao[sA], nB = P.n_ao[sB], mA = P.n_abf[sA], mB = P.n_abf[sB];
    const int pA = rup16(nA), pB = rup16(nB);
    const int MA = rup16(mA), MB = rup16(mB);
    const int y1 = ylut_get(P, A, b, Rb[0], Rb[1], Rb[2]);
    const int y2 = ylut_get(P, b, A, -Rb[0], -Rb[1], -Rb[2]);
    const uint16_t* Yab = X.Ysp + P.y_off[y1];   // [alpha][b][pA]
    const uint16_t* Yba = X.Ysp + P.y_off[y2];   // [beta][a][pB]
    const long long pl_ab = (long long)mA * nB * pA, pl_ba = (long long)mB * nA * pB;
    const uint16_t* Vp = X.Vm + X.vm_off[p];                               // V pieces [alpha][MB]
    const float* V = reinterpret_cast<const float*>(Vp + NP * mA * MB);    // V, grad V (FP32)
    const int nvb = mA * mB;
    const int ZS = pB + 8;
    uint16_t* Zs = reinterpret_cast<uint16_t*>(smem);
    double* gF = reinterpret_cast<double*>(Zs + (size_t)NP * ZROWS * ZS);
    const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * nq; t += blockDim.x) gF[t] = 0.0;
    // R2[alpha][beta] = sum_{b,a} Yab[alpha][b][a] Yba[beta][a][b]; dotted with V, grad V
    float evf[4] = {0.f, 0.f, 0.f, 0.f};
    {
      const int MT = MA >> 4, NT = MB >> 3;
      for (int t = warp; t < MT * NT; t += kWarps) {
        const int mt = t / NT, nt = t - mt * NT;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int bb = 0; bb < nB; ++bb) {
          for (int k0 = 0; k0 < pA; k0 += 16) {
            uint32_t af[NP][4], bf[NP][2];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int al = mt * 16 + gid + ((h & 1) ? 8 : 0);
              const int kc = k0 + 2 * tig + ((h & 2) ? 8 : 0);
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                af[pp][h] = al < mA ? *reinterpret_cast<const uint32_t*>(Yab + pp * pl_ab + ((long long)al * nB + bb) * pA + kc)
                                    : 0u;
            }
            const int be = nt * 8 + gid;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int a0 = k0 + 2 * tig + h * 8;
#pragma unroll
              for (int pp = 0; pp < NP; ++pp) {
                uint16_t lo = 0, hi = 0;
                if (be < mB) {
                  const uint16_t* Yb = Yba + pp * pl_ba + (long long)be * nA * pB + bb;
                  if (a0 < nA) lo = Yb[(long long)a0 * pB];
                  if (a0 + 1 < nA) hi = Yb[(long long)(a0 + 1) * pB];
                }
                bf[pp][h] = pack2(lo, hi);
              }
            }
            mma_split<NP>(acc, af, bf);
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
          const int be = nt * 8 + 2 * tig + (c & 1);
          if (al < mA && be < mB) {
            const int o = al * mB + be;
            const float r = acc[c];
            evf[0] = fmaf(V[o], r, evf[0]);
            evf[1] = fmaf(V[nvb + o], r, evf[1]);
            evf[2] = fmaf(V[2 * nvb + o], r, evf[2]);
            evf[3] = fmaf(V[3 * nvb + o], r, evf[3]);
          }
        }
      }
    }
    double ev[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float w = warp_sum_f(evf[c]);
      ev[c] = lane == 0 ? (double)w : 0.0;
    }
    block_sum_n<4>(ev, red);
    if (threadIdx.x == 0) {
      atomicAdd(&P.acc[ACC_E], -ev[0]);
      atomicAdd(&P.gV[3 * p + 0], -ev[1]);
      atomicAdd(&P.gV[3 * p + 1], -ev[2]);
      atomicAdd(&P.gV[3 * p + 2], -ev[3]);
    }
    // Z[alpha][a][b] = sum_beta V[alpha][beta] Yba[beta][a][b]  ->  Zs[(alpha,a)][b]
    {
      const int MT = MA >> 4;
      const int NZ = nA * pB;         // columns (a, b)
      const int NT = NZ >> 3;
      for (int t = warp; t < MT * NT; t += kWarps) {
        const int mt = t / NT, nt = t - mt * NT;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k0 = 0; k0 < MB; k0 += 16) {
          uint32_t af[NP][4], bf[NP][2];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int al = mt * 16 + gid + ((h & 1) ? 8 : 0);
            const int kc = k0 + 2 * tig + ((h & 2) ? 8 : 0);
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
              af[pp][h] = al < mA ? *reinterpret_cast<const uint32_t*>(Vp + pp * mA * MB + al * MB + kc) : 0u;
          }
          const int col = nt * 8 + gid;    // (a, b) flattened, b fastest (pB)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int be0 = k0 + 2 * tig + h * 8;
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
              uint16_t lo = 0, hi = 0;
              const uint16_t* Yb = Yba + pp * pl_ba + col;
              if (be0 < mB) lo = Yb[(long long)be0 * nA * pB];
              if (be0 + 1 < mB) hi = Yb[(long long)(be0 + 1) * nA * pB];
              bf[pp][h] = pack2(lo, hi);
            }
          }
          mma_split<NP>(acc, af, bf);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
          const int col = nt * 8 + 2 * tig + (c & 1);
          if (al < mA) {
            const int a = col / pB, bb = col - a * pB;
            uint16_t pc[NP];
            split_f<NP>(acc[c], pc);
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) Zs[(size_t)pp * ZROWS * ZS + (size_t)(al * nA + a) * ZS + bb] = pc[pp];
          }
        }
      }
      // zero rows beyond mA*nA up to the m-tile boundary
      const int rowsZ = mA * nA, rowsZp = rup16(rowsZ);
      for (int e = threadIdx.x; e < (rowsZp - rowsZ) * ZS; e += blockDim.x)
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) Zs[(size_t)pp * ZROWS * ZS + (size_t)rowsZ * ZS + e] = 0;
    }
    __syncthreads();
    // Q2_F[(alpha,a)][f] = sum_b Z[(alpha,a)][b] D_FB[f][b], dotted with grad C_AF
    unsigned long long fl = 4ull * mA * mB * nA * nB;
    {
      const int rowsZ = mA * nA;
      const int MTZ = (rowsZ + 15) >> 4;
      for (int t = 0; t < nq; ++t) {
        const int q = q0 + t;
        if (!P.c_keep[q]) continue;
        const int f = P.c_j[q];
        const int* Rf = P.c_R + 3 * q;
        const int di = dlut_get(P, f, b, Rb[0] - Rf[0], Rb[1] - Rf[1], Rb[2] - Rf[2]);
        if (di < 0 || P.Dkept[di] == 0.0) continue;
        const int nF = P.n_ao[P.species[f]];
        const int pF = rup16(nF);
        const uint16_t* Dfb = X.Dsp + X.dsp_off[di];   // [f][pB] planes pF x pB
        const float* dC = reinterpret_cast<const float*>(X.Cm + X.cm_off[q] + (long long)NP * mA * nA * pF);
        const int KAF = nA * nF;
        const long long ncq = (long long)mA * KAF;
        float gf[3] = {0.f, 0.f, 0.f};
        const int NTF = pF >> 3;
        for (int mt = warp; mt < MTZ; mt += kWarps) {
          float acc[4][4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[j][c] = 0.f;
          for (int k0 = 0; k0 < pB; k0 += 16) {
            uint32_t af[NP][4];
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
              ldm_x4(af[pp], Zs + (size_t)pp * ZROWS * ZS + (size_t)(mt * 16 + (lane & 15)) * ZS + k0 + ((lane >> 4) << 3));
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              if (nt >= NTF) break;
              uint32_t bf[NP][2];
#pragma unroll
              for (int pp = 0; pp < NP; ++pp) {
                const uint16_t* Db = Dfb + pp * pF * pB + (nt * 8 + gid) * pB + k0 + 2 * tig;
                bf[pp][0] = *reinterpret_cast<const uint32_t*>(Db);
                bf[pp][1] = *reinterpret_cast<const uint32_t*>(Db + 8);
              }
              mma_split<NP>(acc[nt], af, bf);
            }
          }
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            if (nt >= NTF) break;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int r = mt * 16 + gid + ((c & 2) ? 8 : 0);
              const int ff = nt * 8 + 2 * tig + (c & 1);
              if (r < rowsZ && ff < nF) {
                const int al = r / nA, a = r - al * nA;
                const long long o = (long long)al * KAF + a * nF + ff;
                const float v = acc[nt][c];
                gf[0] = fmaf(dC[o], v, gf[0]);
                gf[1] = fmaf(dC[ncq + o], v, gf[1]);
                gf[2] = fmaf(dC[2 * ncq + o], v, gf[2]);
              }
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float w = warp_sum_f(gf[c]);
          if (lane == 0 && w != 0.f) atomicAdd(&gF[3 * t + c], (double)w);
        }
        if (threadIdx.x == 0) fl += 2ull * mA * nA * nB * nF;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      if (gF[3 * t] != 0.0 || gF[3 * t + 1] != 0.0 || gF[3 * t + 2] != 0.0) {
        const int q = q0 + t;
        atomicAdd(&P.gC[3 * q + 0], -2.0 * gF[3 * t + 0]);
        atomicAdd(&P.gC[3 * q + 1], -2.0 * gF[3 * t + 1]);
        atomicAdd(&P.gC[3 * q + 2], -2.0 * gF[3 * t + 2]);
      }
    }
    if (threadIdx.x == 0) atomicAdd(&P.acc[ACC_F2], (double)fl);
  }
}

int grid_for(long long n, int cap) {
  long long g = n < 1 ? 1 : n;
  return (int)(g > cap ? cap : g);
}

}  // namespace

long long mixed_launch_count() { return g_mix_launches; }

cudaError_t launch_dsplit(const DevPlan& P, const MixPlan& X, int np, cudaStream_t s) {
  if (P.n_d == 0) return cudaSuccess;
  ++g_mix_launches;
  if (np == 2) k_dsplit<2><<<grid_for(P.n_d, 152 * 64), 256, 0, s>>>(P, X);
  else k_dsplit<3><<<grid_for(P.n_d, 152 * 64), 256, 0, s>>>(P, X);
  return cudaGetLastError();
}

cudaError_t launch_cpieces(const DevPlan& P, const MixPlan& X, int np, cudaStream_t s) {
  if (P.nC == 0) return cudaSuccess;
  ++g_mix_launches;
  if (np == 2) k_cpieces<2><<<grid_for(P.nC, 152 * 32), 256, 0, s>>>(P, X);
  else k_cpieces<3><<<grid_for(P.nC, 152 * 32), 256, 0, s>>>(P, X);
  return cudaGetLastError();
}

cudaError_t launch_vpieces(const DevPlan& P, const MixPlan& X, int np, const int* list, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_mix_launches;
  if (np == 2) k_vpieces<2><<<grid_for(n, 152 * 32), 256, 0, s>>>(P, X, list, n);
  else k_vpieces<3><<<grid_for(n, 152 * 32), 256, 0, s>>>(P, X, list, n);
  return cudaGetLastError();
}

cudaError_t launch_ybuild_mma(const DevPlan& P, const MixPlan& X, int np, const int* list, int n, int wide,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_mix_launches;
  const int g = grid_for(n, 152 * 32);
  if (np == 2 && !wide) k_ybuild_mma<2, 2><<<g, kWarps * 32, 0, s>>>(P, X, list, n);
  else if (np == 2) k_ybuild_mma<2, 4><<<g, kWarps * 32, 0, s>>>(P, X, list, n);
  else if (!wide) k_ybuild_mma<3, 2><<<g, kWarps * 32, 0, s>>>(P, X, list, n);
  else k_ybuild_mma<3, 4><<<g, kWarps * 32, 0, s>>>(P, X, list, n);
  return cudaGetLastError();
}

cudaError_t launch_t1_lists(const DevPlan& P, const MixPlan& X, int phase, cudaStream_t s) {
  ++g_mix_launches;
  if (phase == 0) k_t1_count<<<P.N, 256, 0, s>>>(P, X);
  else k_t1_fill<<<P.N, 256, 0, s>>>(P, X);
  return cudaGetLastError();
}

size_t term1_mma_smem(int np, int MAmax, int MBmax, int KSmax) {
  return (size_t)np * (MAmax * KSmax + MBmax * KSmax + MAmax * (MBmax + 8)) * sizeof(uint16_t);
}

size_t term2_mma_smem(int np, int zrows, int zs) {
  return (size_t)np * zrows * zs * sizeof(uint16_t) + 3 * kMaxCPerAtom * sizeof(double);
}

cudaError_t set_mixed_smem_limits(int np, size_t t1, size_t t2) {
  cudaError_t e;
  if (np == 2) {
    e = cudaFuncSetAttribute(k_term1_mma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t1);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_term2_mma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t2);
  }
  e = cudaFuncSetAttribute(k_term1_mma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t1);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_term2_mma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t2);
}

cudaError_t launch_term1_mma(const DevPlan& P, const MixPlan& X, int np, const int* qlist, int n, int MAmax, int MBmax,
                             int KSmax, size_t smem, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_mix_launches;
  if (np == 2)
    k_term1_mma<2><<<grid_for(n, 152 * 16), kWarps1 * 32, smem, s>>>(P, X, qlist, n, MAmax, MBmax, KSmax);
  else
    k_term1_mma<3><<<grid_for(n, 152 * 16), kWarps1 * 32, smem, s>>>(P, X, qlist, n, MAmax, MBmax, KSmax);
  return cudaGetLastError();
}

cudaError_t launch_term2_mma(const DevPlan& P, const MixPlan& X, int np, const int* list, int n, int zrows,
                             size_t smem, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_mix_launches;
  if (np == 2) k_term2_mma<2><<<grid_for(n, 152 * 32), kWarps * 32, smem, s>>>(P, X, list, n, zrows);
  else k_term2_mma<3><<<grid_for(n, 152 * 32), kWarps * 32, smem, s>>>(P, X, list, n, zrows);
  return cudaGetLastError();
}

}  // namespace hfx
